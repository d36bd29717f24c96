// Mesh set-up kernels: the reference precompute of Section 6 and one round
// of the Jones-Plassmann conflict colouring.
#include "tlfe_elem.cuh"
#include "tlfe_internal.h"

namespace tlfe {

// Affine element (Sec. 6, affine case): the map from the parent element is
// u(xi) = A xi + b. Holds for every T4; for T10 when the mid-edge nodes sit at
// their edge midpoints; for H8 when the brick is a parallelepiped; for Q27
// when the nodes sit at X_0 + (i/2)(X_2 - X_0) + (j/2)(X_6 - X_0) + (k/2)(X_18 - X_0)
// (node i + 3j + 9k). Tolerance 1e-10 of the element extent.
__device__ bool element_is_affine(int et, int npe, const double Xe[27][3])
{
    bool affine = true;
    double ext = 0.0;
    for (int i = 1; i < npe; ++i)
        for (int a = 0; a < 3; ++a) ext = fmax(ext, fabs(Xe[i][a] - Xe[0][a]));
    const double tol = 1e-10 * ext;
    if (et == ET_T10) {
        for (int m = 0; m < 6; ++m) {
            int a, b;
            t10_edge(m, a, b);
            for (int d = 0; d < 3; ++d)
                if (fabs(Xe[4 + m][d] - 0.5 * (Xe[a][d] + Xe[b][d])) > tol) affine = false;
        }
    } else if (et == ET_H8) {
        for (int n = 0; n < 8; ++n)
            for (int d = 0; d < 3; ++d) {
                const double p = Xe[0][d] + ((n & 1) ? Xe[1][d] - Xe[0][d] : 0.0) +
                                 ((n & 2) ? Xe[2][d] - Xe[0][d] : 0.0) + ((n & 4) ? Xe[4][d] - Xe[0][d] : 0.0);
                if (fabs(Xe[n][d] - p) > tol) affine = false;
            }
    } else if (et == ET_Q27) {
        for (int n = 0; n < 27; ++n)
            for (int d = 0; d < 3; ++d) {
                const double p = Xe[0][d] + 0.5 * (n % 3) * (Xe[2][d] - Xe[0][d]) +
                                 0.5 * ((n / 3) % 3) * (Xe[6][d] - Xe[0][d]) + 0.5 * (n / 9) * (Xe[18][d] - Xe[0][d]);
                if (fabs(Xe[n][d] - p) > tol) affine = false;
            }
    }
    return affine;
}

// Jp = U Hp(xi) evaluated as sum_{i>0} (X_i - X_0) dS_i/dxi^T (the parent
// gradients sum to zero); relative coordinates keep the digits that large
// absolute coordinates would cancel away. Returns det Jp and Jp^{-1} = cof^T / det.
__device__ double parent_jacobian_inv(int et, int npe, const double Xe[27][3], const double *g, double Ji[9])
{
    double J[9];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int i = 1; i < npe; ++i) s += (Xe[i][a] - Xe[0][a]) * g[i * 3 + k];
            J[a * 3 + k] = s;
        }
    const double c00 = J[4] * J[8] - J[5] * J[7];
    const double c01 = J[5] * J[6] - J[3] * J[8];
    const double c02 = J[3] * J[7] - J[4] * J[6];
    const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    Ji[0] = c00 / det;
    Ji[3] = c01 / det;
    Ji[6] = c02 / det;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    return det;
}

// One thread per (tile, lane): for each quadrature point,
//   Jp = U Hp(xi_q)  (U = [X_1 .. X_n]),  h_i^T = dS_i/dxi Jp^{-1},
//   wJ = w_q det(Jp)                               (Sec. 6, H = Hp (U Hp)^{-1}, J_p)
// in FP64, stored in the mesh precision as the slab
//   slab[tile][q][r][lane], r = 3 i + c for (h_i)_c and r = 3 npe for wJ,
// so that one quadrature point of one tile is a contiguous slice. Also
// records the element volume sum_q wJ and whether the element is affine
// (straight edges / parallelepiped), which the consistent-mass shortcut
// m_ij = rho V Mhat_ij needs.
template <typename R>
__global__ void k_precompute(int et, int nq, int npe, int n_tiles, const int32_t *__restrict__ eid,
                             const int32_t *__restrict__ conn, int elem_base,
                             const double *__restrict__ X, R *__restrict__ slab,
                             R *__restrict__ evol, int *affine_flag, int *status)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_tiles * 32) return;
    const int64_t t = idx >> 5;
    const int lane = (int)(idx & 31);
    const int e = eid[idx];
    const int rows = npe * 3 + 1;
    if (e < 0) {
        for (int q = 0; q < nq; ++q)
            for (int k = 0; k < rows; ++k) slab[((t * nq + q) * rows + k) * 32 + lane] = R(0);
        evol[idx] = R(0);
        return;
    }
    const int64_t el = (int64_t)e - elem_base;
    double Xe[27][3];
    for (int i = 0; i < npe; ++i) {
        const int64_t n = conn[el * npe + i];
        for (int a = 0; a < 3; ++a) Xe[i][a] = X[n * 3 + a];
    }
    double vol = 0.0, jmin = 1e300, jmax = -1e300;
    int inverted = 0;
    for (int q = 0; q < nq; ++q) {
        double xi[3], w, g[81];
        quad_point(et, nq, q, xi, w);
        parent_grad(et, xi, g);
        double Ji[9];
        const double det = parent_jacobian_inv(et, npe, Xe, g, Ji);
        jmin = fmin(jmin, det);
        jmax = fmax(jmax, det);
        const bool ok = det > 0.0;
        if (!ok) inverted = 1;
        for (int i = 0; i < npe; ++i)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += g[i * 3 + k] * Ji[k * 3 + c];
                slab[((t * nq + q) * rows + i * 3 + c) * 32 + lane] = ok ? R(s) : R(0);
            }
        const double wj = ok ? w * det : 0.0;
        slab[((t * nq + q) * rows + npe * 3) * 32 + lane] = R(wj);
        vol += wj;
    }
    evol[idx] = R(vol);
    if (inverted) atomicAdd(status + ST_INVERTED, 1);
    const bool affine = element_is_affine(et, npe, Xe);
    (void)jmin;
    (void)jmax;
    if (!affine) atomicAnd(affine_flag, 0);
}

cudaError_t launch_precompute(int et, int nq, int precision, int n_tiles, const int32_t *eid,
                              const int32_t *conn_elem, int elem_base, const double *X, void *slab,
                              void *evol, int *affine_flag, int *status, cudaStream_t s)
{
    const int npe = nodes_per_elem(et);
    const int64_t n = (int64_t)n_tiles * 32;
    const int tpb = 128;
    const unsigned grid = (unsigned)((n + tpb - 1) / tpb);
    if (grid == 0) return cudaSuccess;
    if (precision == TLFE_FP32)
        k_precompute<float><<<grid, tpb, 0, s>>>(et, nq, npe, n_tiles, eid, conn_elem, elem_base, X,
                                                 (float *)slab, (float *)evol, affine_flag, status);
    else
        k_precompute<double><<<grid, tpb, 0, s>>>(et, nq, npe, n_tiles, eid, conn_elem, elem_base, X,
                                                  (double *)slab, (double *)evol, affine_flag, status);
    return cudaGetLastError();
}

// Affine path (Sec. 6, affine case): one thread per (tile, lane) writes
//   aff[tile][r][lane], r = 0..8: J^{-1} (row-major), r = 9: det J
// with J = du/dxi constant over the element (evaluated at the centroid, in
// FP64, relative coordinates), the element volume det J * |parent| into evol,
// and clears *affine_flag when an element of the block is not affine.
// det J <= 0 counts as an inverted element.
template <typename R>
__global__ void k_precompute_affine(int et, int npe, int n_tiles, const int32_t *__restrict__ eid,
                                    const int32_t *__restrict__ conn, int elem_base,
                                    const double *__restrict__ X, R *__restrict__ aff, R *__restrict__ evol,
                                    int *affine_flag, int *status)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_tiles * 32) return;
    const int64_t t = idx >> 5;
    const int lane = (int)(idx & 31);
    const int e = eid[idx];
    if (e < 0) {
        for (int r = 0; r < 10; ++r) aff[(t * 10 + r) * 32 + lane] = R(0);
        evol[idx] = R(0);
        return;
    }
    const int64_t el = (int64_t)e - elem_base;
    double Xe[27][3];
    for (int i = 0; i < npe; ++i) {
        const int64_t n = conn[el * npe + i];
        for (int a = 0; a < 3; ++a) Xe[i][a] = X[n * 3 + a];
    }
    double xi[3], g[81];
    if (et == ET_H8 || et == ET_Q27) {
        xi[0] = xi[1] = xi[2] = 0.0;
    } else {
        xi[0] = xi[1] = xi[2] = 0.25;
    }
    parent_grad(et, xi, g);
    double Ji[9];
    const double det = parent_jacobian_inv(et, npe, Xe, g, Ji);
    const bool ok = det > 0.0;
    for (int r = 0; r < 9; ++r) aff[(t * 10 + r) * 32 + lane] = ok ? R(Ji[r]) : R(0);
    aff[(t * 10 + 9) * 32 + lane] = ok ? R(det) : R(0);
    evol[idx] = ok ? R(det * ((et == ET_H8 || et == ET_Q27) ? 8.0 : 1.0 / 6.0)) : R(0);
    if (!ok) atomicAdd(status + ST_INVERTED, 1);
    if (!element_is_affine(et, npe, Xe)) atomicAnd(affine_flag, 0);
}

cudaError_t launch_precompute_affine(int et, int precision, int n_tiles, const int32_t *eid,
                                     const int32_t *conn_elem, int elem_base, const double *X, void *aff,
                                     void *evol, int *affine_flag, int *status, cudaStream_t s)
{
    const int npe = nodes_per_elem(et);
    const int64_t n = (int64_t)n_tiles * 32;
    const int tpb = 128;
    const unsigned grid = (unsigned)((n + tpb - 1) / tpb);
    if (grid == 0) return cudaSuccess;
    if (precision == TLFE_FP32)
        k_precompute_affine<float><<<grid, tpb, 0, s>>>(et, npe, n_tiles, eid, conn_elem, elem_base, X,
                                                        (float *)aff, (float *)evol, affine_flag, status);
    else
        k_precompute_affine<double><<<grid, tpb, 0, s>>>(et, npe, n_tiles, eid, conn_elem, elem_base, X,
                                                         (double *)aff, (double *)evol, affine_flag, status);
    return cudaGetLastError();
}

// per-element (mu, lambda) from a device array in global element order into the
// block's AoSoA copy [tile][2][32]
template <typename R>
__global__ void k_set_elam(int n_slots, const int32_t *__restrict__ eid, const double *__restrict__ src,
                           R *__restrict__ elam)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_slots) return;
    const int t = idx >> 5, lane = idx & 31;
    const int e = eid[idx];
    elam[((size_t)t * 2 + 0) * 32 + lane] = e >= 0 ? R(src[(size_t)e * 2 + 0]) : R(0);
    elam[((size_t)t * 2 + 1) * 32 + lane] = e >= 0 ? R(src[(size_t)e * 2 + 1]) : R(0);
}

cudaError_t launch_set_elam(int precision, int n_tiles, const int32_t *eid, const double *src, void *elam,
                            cudaStream_t s)
{
    const int n = n_tiles * 32;
    if (n == 0) return cudaSuccess;
    if (precision == TLFE_FP32)
        k_set_elam<float><<<(n + 255) / 256, 256, 0, s>>>(n, eid, src, (float *)elam);
    else
        k_set_elam<double><<<(n + 255) / 256, 256, 0, s>>>(n, eid, src, (double *)elam);
    return cudaGetLastError();
}

// splitmix64 finaliser (Steele, Lea and Flood 2014) applied to x + golden gamma
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One Jones-Plassmann round over the elements of one block. An uncoloured
// element whose uncoloured conflicting neighbours (sharing a node) all have
// lower priority takes the smallest colour not held by its coloured
// neighbours. Coloured neighbours are exactly the higher-priority ones, so the
// result equals greedy colouring in descending priority, whatever the order in
// which elements of one round finish.
__global__ void k_color_round(int n_elem, int npe, const int32_t *__restrict__ conn,
                              const int32_t *__restrict__ inc_off, const int32_t *__restrict__ inc,
                              uint64_t seed, int32_t *color, int *n_left, int *overflow)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    volatile int32_t *vc = color;
    if (vc[e] >= 0) return;
    const uint64_t pe = splitmix64((uint64_t)e ^ seed);
    uint32_t used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < npe; ++i) {
        const int nd = conn[(int64_t)e * npe + i];
        for (int k = inc_off[nd]; k < inc_off[nd + 1]; ++k) {
            const int o = inc[k];
            if (o == e) continue;
            const int c = vc[o];
            if (c < 0) {
                if (splitmix64((uint64_t)o ^ seed) > pe) return;
            } else if (c < 256) {
                used[c >> 5] |= 1u << (c & 31);
            } else {
                atomicExch(overflow, 1);
            }
        }
    }
    int c = 0;
    while (c < 256 && (used[c >> 5] >> (c & 31)) & 1u) ++c;
    if (c >= 256) {
        atomicExch(overflow, 1);
        c = 255;
    }
    vc[e] = c;
    atomicSub(n_left, 1);
}

cudaError_t launch_color_round(int n_elem, int npe, const int32_t *conn, const int32_t *inc_off,
                               const int32_t *inc, const int32_t *, uint64_t seed, int, int32_t *color,
                               int *n_left, int *overflow, cudaStream_t s)
{
    const int tpb = 256;
    const int grid = (n_elem + tpb - 1) / tpb;
    if (grid == 0) return cudaSuccess;
    k_color_round<<<grid, tpb, 0, s>>>(n_elem, npe, conn, inc_off, inc, seed, color, n_left, overflow);
    return cudaGetLastError();
}

}  // namespace tlfe
