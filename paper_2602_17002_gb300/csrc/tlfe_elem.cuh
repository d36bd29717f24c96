// Parent-element data for the CUDA path: shape-function gradients on the
// parent element, quadrature points, and the normalised consistent-mass tables
// of affine elements. Written from the element definitions, not from any
// other implementation:
//   T4 : linear barycentric tetrahedron, L1 = 1 - xi - eta - zeta, L2..L4 = xi, eta, zeta
//   T10: quadratic barycentric tetrahedron (App. A.1): corners L_k (2 L_k - 1),
//        edge nodes 4 L_a L_b on edges (1,2) (2,3) (1,3) (1,4) (2,4) (3,4)
//   H8 : trilinear brick on {-1,1}^3, node i + 2j + 4k (tensor order of App. A.2)
//   Q27: triquadratic brick (App. A, Q27 element): node i + 3j + 9k at
//        (xi, eta, zeta) = (i - 1, j - 1, k - 1), shape function
//        l_i(xi) l_j(eta) l_k(zeta) with the 1D quadratic Lagrange polynomials
//        l_0 = x (x - 1)/2, l_1 = 1 - x^2, l_2 = x (x + 1)/2 on the nodes -1, 0, 1
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

// 1D quadratic Lagrange polynomials on the nodes -1, 0, 1 and their derivatives
__host__ __device__ inline void lagrange2(double x, double l[3], double dl[3])
{
    l[0] = 0.5 * x * (x - 1.0);
    l[1] = (1.0 - x) * (1.0 + x);
    l[2] = 0.5 * x * (x + 1.0);
    dl[0] = x - 0.5;
    dl[1] = -2.0 * x;
    dl[2] = x + 0.5;
}

// d s_i / d xi_k in double, g[i*3 + k]
__host__ __device__ inline void parent_grad(int et, const double xi[3], double *g)
{
    if (et == ET_Q27) {
        double l[3][3], dl[3][3];
        for (int d = 0; d < 3; ++d) lagrange2(xi[d], l[d], dl[d]);
        for (int n = 0; n < 27; ++n) {
            const int a = n % 3, b = (n / 3) % 3, c = n / 9;
            g[n * 3 + 0] = dl[0][a] * l[1][b] * l[2][c];
            g[n * 3 + 1] = l[0][a] * dl[1][b] * l[2][c];
            g[n * 3 + 2] = l[0][a] * l[1][b] * dl[2][c];
        }
        return;
    }
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

// s_i(xi) in double: T4 barycentric; T10 corners L (2 L - 1), mid-edge nodes
// 4 L_a L_b; H8 trilinear tensor products
__host__ __device__ inline void shape_fn(int et, const double xi[3], double *sh)
{
    if (et == ET_Q27) {
        double l[3][3], dl[3][3];
        for (int d = 0; d < 3; ++d) lagrange2(xi[d], l[d], dl[d]);
        for (int n = 0; n < 27; ++n) sh[n] = l[0][n % 3] * l[1][(n / 3) % 3] * l[2][n / 9];
        return;
    }
    if (et == ET_T4 || et == ET_T10) {
        const double L[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
        if (et == ET_T4) {
            for (int k = 0; k < 4; ++k) sh[k] = L[k];
            return;
        }
        for (int k = 0; k < 4; ++k) sh[k] = L[k] * (2.0 * L[k] - 1.0);
        for (int e = 0; e < 6; ++e) {
            int a, b;
            t10_edge(e, a, b);
            sh[4 + e] = 4.0 * L[a] * L[b];
        }
        return;
    }
    for (int n = 0; n < 8; ++n) {
        double v = 1.0;
        for (int d = 0; d < 3; ++d) v *= 0.5 * (1.0 + (((n >> d) & 1) ? xi[d] : -xi[d]));
        sh[n] = v;
    }
}

// Quadrature point q of the (et, nq) rule: parent coordinates and weight.
// Tetrahedra (parent volume 1/6): 1-point centroid; 4-point degree-2 rule with
// barycentric (a, b, b, b), a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20, w = 1/24;
// 5-point degree-3 rule: centroid with w = -2/15, and (1/2, 1/6, 1/6, 1/6)
// permutations with w = 3/40. H8: 2x2x2 Gauss-Legendre (+-1/sqrt3, w = 1), or
// the 1-point centre rule (w = 8). Q27: 3x3x3 Gauss-Legendre (0, +-sqrt(3/5);
// 8/9, 5/9 per direction), point q = i + 3j + 9k.
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
    if (et == ET_Q27 && nq == 27) {
        const int id[3] = {q % 3, (q / 3) % 3, q / 9};
        const double r = sqrt(0.6);
        w = 1.0;
        for (int d = 0; d < 3; ++d) {
            xi[d] = id[d] == 0 ? -r : (id[d] == 1 ? 0.0 : r);
            w *= id[d] == 1 ? 8.0 / 9.0 : 5.0 / 9.0;
        }
        return true;
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
//   Q27 (parallelepiped): prod_d m[i_d][j_d] with the normalised 1D quadratic
//        mass m = [[4, 2, -1], [2, 16, 2], [-1, 2, 4]] / 30
__host__ __device__ inline double mass_hat(int et, int i, int j)
{
    if (et == ET_Q27) {
        const double m1[3][3] = {{4.0, 2.0, -1.0}, {2.0, 16.0, 2.0}, {-1.0, 2.0, 4.0}};
        return m1[i % 3][j % 3] * m1[(i / 3) % 3][(j / 3) % 3] * m1[i / 9][j / 9] / 27000.0;
    }
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

// ---------------------------------------------------------------------------
// Affine elements (Sec. 6, affine case): with du/dxi = J constant, the
// reference gradients are h_i = J^{-T} dS_i/dxi(xi_q) and the quadrature
// weight is w_q det J. The element kernels then stream J^{-1} and det J per
// element instead of h_i per point, and evaluate the parent gradients at each
// point from the point's coordinates. ParentGrad<ET, NQ, R> gives the entry
// g(i, k) = dS_i/dxi_k at the current point; nz(i, k) is false where the entry
// vanishes identically, so that fully unrolled loops skip those terms.
// ---------------------------------------------------------------------------

// barycentric gradients dL_j/dxi_k of the tetrahedron: L1 -> (-1,-1,-1), L2..L4 -> unit vectors
__host__ __device__ constexpr int tet_dL(int j, int k) { return j == 0 ? -1 : (k == j - 1 ? 1 : 0); }
__host__ __device__ constexpr int t10_ea(int e) { return e == 0 ? 0 : (e == 1 ? 1 : (e == 2 ? 0 : (e == 3 ? 0 : (e == 4 ? 1 : 2)))); }
__host__ __device__ constexpr int t10_eb(int e) { return e == 0 ? 1 : (e == 1 ? 2 : (e == 2 ? 2 : 3)); }

template <int ET, int NQ, typename R> struct ParentGrad;

// T4: constant gradients dS_i/dxi = dL_i/dxi
template <int NQ, typename R> struct ParentGrad<ET_T4, NQ, R> {
    __device__ __forceinline__ void at(int) {}
    __host__ __device__ static constexpr bool nz(int i, int k) { return tet_dL(i, k) != 0; }
    __device__ __forceinline__ R g(int i, int k) const { return tet_dL(i, k) > 0 ? R(1) : R(-1); }
};

// T10: corners L_i (2 L_i - 1) -> (4 L_i - 1) dL_i; edge (a, b): 4 L_a L_b -> 4 (L_b dL_a + L_a dL_b).
// The point is held as L4 = 4 L.
template <int NQ, typename R> struct ParentGrad<ET_T10, NQ, R> {
    R L4[4];
    __device__ __forceinline__ void at(int q)
    {
        if constexpr (NQ == 5) {  // centroid, then (1/2, 1/6, 1/6, 1/6) permutations
#pragma unroll
            for (int j = 0; j < 4; ++j) L4[j] = q == 0 ? R(1) : (j == q - 1 ? R(2) : R(2.0 / 3.0));
        } else if constexpr (NQ == 4) {  // (a, b, b, b) permutations, a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20
            const R a4 = R(0.58541019662496845446 * 4.0), b4 = R(0.13819660112501051518 * 4.0);
#pragma unroll
            for (int j = 0; j < 4; ++j) L4[j] = j == q ? a4 : b4;
        } else {  // centroid
#pragma unroll
            for (int j = 0; j < 4; ++j) L4[j] = R(1);
        }
    }
    __host__ __device__ static constexpr bool nz(int i, int k)
    {
        return i < 4 ? tet_dL(i, k) != 0 : (tet_dL(t10_ea(i - 4), k) != 0 || tet_dL(t10_eb(i - 4), k) != 0);
    }
    __device__ __forceinline__ R g(int i, int k) const
    {
        if (i < 4) {
            const R c = L4[i] - R(1);
            return tet_dL(i, k) > 0 ? c : -c;
        }
        const int a = t10_ea(i - 4), b = t10_eb(i - 4);
        const int da = tet_dL(a, k), db = tet_dL(b, k);
        const R ta = da > 0 ? L4[b] : -L4[b];  // 4 L_b dL_a
        const R tb = db > 0 ? L4[a] : -L4[a];  // 4 L_a dL_b
        if (da != 0 && db != 0) return ta + tb;
        return da != 0 ? ta : tb;
    }
};

// H8 (parallelepiped): dS_n/dxi_k = (s_k / 2) prod_{j != k} (1 + s_j xi_j) / 2 with
// s_j = -1 / +1 from bit j of n; the point is held as the six factors (1 +- xi_j) / 2.
template <int NQ, typename R> struct ParentGrad<ET_H8, NQ, R> {
    R f[3][2];  // f[j][s] = (1 + (2s - 1) xi_j) / 2
    __device__ __forceinline__ void at(int q)
    {
        const R gp = R(0.57735026918962576451);  // 1/sqrt(3)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const R x = NQ == 8 ? (((q >> j) & 1) ? gp : -gp) : R(0);
            f[j][0] = R(0.5) * (R(1) - x);
            f[j][1] = R(0.5) * (R(1) + x);
        }
    }
    __host__ __device__ static constexpr bool nz(int, int) { return true; }
    __device__ __forceinline__ R g(int n, int k) const
    {
        const int j1 = (k + 1) % 3, j2 = (k + 2) % 3;
        const R p = R(0.5) * f[j1][(n >> j1) & 1] * f[j2][(n >> j2) & 1];
        return ((n >> k) & 1) ? p : -p;
    }
};

// Q27 (parallelepiped): dS_n/dxi_k = l'_{n_k}(xi_k) prod_{j != k} l_{n_j}(xi_j)
// with the tensor indices (n_0, n_1, n_2) = (n % 3, (n / 3) % 3, n / 9). The 81
// entries at each of the 27 Gauss points are tabulated once, at compile time,
// in constant memory: every lane of a warp reads the same point's row, a
// broadcast, in place of 108 multiplications per use.
template <typename R> struct Q27Table {
    R g[27][81];
};
__host__ __device__ constexpr double q27_l(int a, double x)
{
    return a == 0 ? 0.5 * x * (x - 1.0) : (a == 1 ? (1.0 - x) * (1.0 + x) : 0.5 * x * (x + 1.0));
}
__host__ __device__ constexpr double q27_dl(int a, double x) { return a == 0 ? x - 0.5 : (a == 1 ? -2.0 * x : x + 0.5); }
template <typename R> constexpr Q27Table<R> make_q27_table()
{
    Q27Table<R> t{};
    const double r = 0.77459666924148337704;  // sqrt(3/5)
    for (int q = 0; q < 27; ++q) {
        const int qi[3] = {q % 3, (q / 3) % 3, q / 9};
        double x[3] = {0, 0, 0};
        for (int j = 0; j < 3; ++j) x[j] = qi[j] == 0 ? -r : (qi[j] == 1 ? 0.0 : r);
        for (int n = 0; n < 27; ++n) {
            const int a[3] = {n % 3, (n / 3) % 3, n / 9};
            for (int k = 0; k < 3; ++k) {
                double v = 1.0;
                for (int j = 0; j < 3; ++j) v *= j == k ? q27_dl(a[j], x[j]) : q27_l(a[j], x[j]);
                t.g[q][n * 3 + k] = R(v);
            }
        }
    }
    return t;
}
static __constant__ Q27Table<float> kQ27F = make_q27_table<float>();
static __constant__ Q27Table<double> kQ27D = make_q27_table<double>();
template <int NQ, typename R> struct ParentGrad<ET_Q27, NQ, R> {
    const R *row;
    __device__ __forceinline__ void at(int q)
    {
        if constexpr (sizeof(R) == 4) row = kQ27F.g[q];
        else row = kQ27D.g[q];
    }
    __host__ __device__ static constexpr bool nz(int, int) { return true; }
    __device__ __forceinline__ R g(int n, int k) const { return row[n * 3 + k]; }
};

// quadrature weight w_q of point q (parent measure), matching quad_point
template <int ET, int NQ, typename R> __device__ __forceinline__ R quad_weight(int q)
{
    if constexpr (ET == ET_Q27) {
        const R w1 = R(5.0 / 9.0), w0 = R(8.0 / 9.0);
        return ((q % 3) == 1 ? w0 : w1) * (((q / 3) % 3) == 1 ? w0 : w1) * ((q / 9) == 1 ? w0 : w1);
    }
    if constexpr (ET == ET_H8) return NQ == 8 ? R(1) : R(8);
    if constexpr (NQ == 5) return q == 0 ? R(-2.0 / 15.0) : R(3.0 / 40.0);
    if constexpr (NQ == 4) return R(1.0 / 24.0);
    return R(1.0 / 6.0);
}

}  // namespace tlfe
