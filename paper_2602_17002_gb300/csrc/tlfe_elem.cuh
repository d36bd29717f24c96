// Parent-element data for the CUDA path: shape-function gradients on the
// parent element, quadrature points, and the normalised consistent-mass tables
// of affine elements. Written from the element definitions, not from any
// other implementation:
//   T4 : linear barycentric tetrahedron, L1 = 1 - xi - eta - zeta, L2..L4 = xi, eta, zeta
//   T10: quadratic barycentric tetrahedron (App. A.1): corners L_k (2 L_k - 1),
//        edge nodes 4 L_a L_b on edges (1,2) (2,3) (1,3) (1,4) (2,4) (3,4)
//   H8 : trilinear brick on {-1,1}^3, node i + 2j + 4k (tensor order of App. A.2)
#pragma once

#include "tlfe_math.cuh"

namespace tlfe {

// edge (a, b) of the six T10 mid-edge nodes 5..10, as barycentric indices
__host__ __device__ inline void t10_edge(int e, int &a, int &b)
{
    const int A[6] = {0, 1, 0, 0, 1, 2};
    const int B[6] = {1, 2, 2, 3, 3, 3};
    a = A[e];
    b = B[e];
}

// d s_i / d xi_k in double, g[i*3 + k]
__host__ __device__ inline void parent_grad(int et, const double xi[3], double *g)
{
    if (et == ET_T4 || et == ET_T10) {
        const double L[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
        // dL_k / dxi: L1 -> (-1,-1,-1), L2 -> e1, L3 -> e2, L4 -> e3
        double dL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        if (et == ET_T4) {
            for (int k = 0; k < 4; ++k)
                for (int c = 0; c < 3; ++c) g[k * 3 + c] = dL[k][c];
            return;
        }
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) g[k * 3 + c] = (4.0 * L[k] - 1.0) * dL[k][c];
        for (int e = 0; e < 6; ++e) {
            int a, b;
            t10_edge(e, a, b);
            for (int c = 0; c < 3; ++c) g[(4 + e) * 3 + c] = 4.0 * (L[b] * dL[a][c] + L[a] * dL[b][c]);
        }
        return;
    }
    // H8
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                const double sx = i ? 1.0 : -1.0, sy = j ? 1.0 : -1.0, sz = k ? 1.0 : -1.0;
                const double nx = 0.5 * (1.0 + sx * xi[0]), ny = 0.5 * (1.0 + sy * xi[1]),
                             nz = 0.5 * (1.0 + sz * xi[2]);
                const int n = i + 2 * j + 4 * k;
                g[n * 3 + 0] = 0.5 * sx * ny * nz;
                g[n * 3 + 1] = nx * 0.5 * sy * nz;
                g[n * 3 + 2] = nx * ny * 0.5 * sz;
            }
}

// Quadrature point q of the (et, nq) rule: parent coordinates and weight.
// Tetrahedra (parent volume 1/6): 1-point centroid; 4-point degree-2 rule with
// barycentric (a, b, b, b), a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20, w = 1/24;
// 5-point degree-3 rule: centroid with w = -2/15, and (1/2, 1/6, 1/6, 1/6)
// permutations with w = 3/40. Bricks: 2x2x2 Gauss-Legendre (+-1/sqrt3, w = 1),
// or the 1-point centre rule (w = 8).
__host__ __device__ inline bool quad_point(int et, int nq, int q, double xi[3], double &w)
{
    if (et == ET_T4 || et == ET_T10) {
        double L[4];
        if (nq == 1) {
            L[0] = L[1] = L[2] = L[3] = 0.25;
            w = 1.0 / 6.0;
        } else if (nq == 4) {
            const double s5 = sqrt(5.0);
            const double a = (5.0 + 3.0 * s5) / 20.0, b = (5.0 - s5) / 20.0;
            for (int k = 0; k < 4; ++k) L[k] = (k == q) ? a : b;
            w = 1.0 / 24.0;
        } else if (nq == 5) {
            if (q == 0) {
                L[0] = L[1] = L[2] = L[3] = 0.25;
                w = -2.0 / 15.0;
            } else {
                for (int k = 0; k < 4; ++k) L[k] = (k == q - 1) ? 0.5 : 1.0 / 6.0;
                w = 3.0 / 40.0;
            }
        } else {
            return false;
        }
        xi[0] = L[1];
        xi[1] = L[2];
        xi[2] = L[3];
        return true;
    }
    if (et == ET_H8) {
        if (nq == 1) {
            xi[0] = xi[1] = xi[2] = 0.0;
            w = 8.0;
            return true;
        }
        if (nq == 8) {
            const double g = 1.0 / sqrt(3.0);
            xi[0] = (q & 1) ? g : -g;
            xi[1] = (q & 2) ? g : -g;
            xi[2] = (q & 4) ? g : -g;
            w = 1.0;
            return true;
        }
    }
    return false;
}

// Normalised consistent mass of an affine element, Mhat_ij = (1/V) int s_i s_j dV,
// so that m_ij = rho V Mhat_ij (Sec. 4.1). Closed forms from the barycentric
// integral int L1^a L2^b L3^c L4^d dV = a! b! c! d! 3! V / (a+b+c+d+3)!:
//   T4 : (1 + delta_ij) / 20
//   T10 (units of 1/420): corner-corner 6 (i = j) or 1; corner-edge -4 when the
//        edge holds the corner, else -6; edge-edge 32 (same edge), 16 (one
//        shared corner), 8 (disjoint)
//   H8 (parallelepiped): prod_d (1/3 if the d-th tensor indices agree, else 1/6)
__host__ __device__ inline double mass_hat(int et, int i, int j)
{
    if (et == ET_T4) return (i == j ? 2.0 : 1.0) / 20.0;
    if (et == ET_H8) {
        double m = 1.0;
        for (int d = 0; d < 3; ++d) m *= (((i >> d) & 1) == ((j >> d) & 1)) ? 1.0 / 3.0 : 1.0 / 6.0;
        return m;
    }
    // T10
    const bool ci = i < 4, cj = j < 4;
    if (ci && cj) return (i == j ? 6.0 : 1.0) / 420.0;
    if (ci != cj) {
        const int c = ci ? i : j, e = ci ? j - 4 : i - 4;
        int a, b;
        t10_edge(e, a, b);
        return (a == c || b == c ? -4.0 : -6.0) / 420.0;
    }
    int a1, b1, a2, b2;
    t10_edge(i - 4, a1, b1);
    t10_edge(j - 4, a2, b2);
    const int shared = (a1 == a2) + (a1 == b2) + (b1 == a2) + (b1 == b2);
    return (shared == 2 ? 32.0 : (shared == 1 ? 16.0 : 8.0)) / 420.0;
}

// v_i / V = (1/V) int s_i dV of an affine element (row sums of Mhat)
__host__ __device__ inline double vol_hat(int et, int i)
{
    double s = 0.0;
    const int n = nodes_per_elem(et);
    for (int j = 0; j < n; ++j) s += mass_hat(et, i, j);
    return s;
}

}  // namespace tlfe
