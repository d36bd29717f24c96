// External loads of Sec. 4: pointwise forces distributed through the shape
// functions (Eq. virtual_work_point_force_discrete) and nominal surface
// tractions integrated over loaded element faces by boundary quadrature
// (Eq. virtual_work_traction_discrete). FP64 throughout; results are added
// into a caller-owned FP64 node array with atomics.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "tlfe_elem.cuh"
#include "tlfe_mesh.h"

namespace tlfe {

// f[conn_i] += s_i(xi_k) force_k for the loads k whose global element lies in
// [elem_base, elem_base + n_elem)
__global__ void k_point_loads(int et, int npe, int elem_base, int n_elem, const int32_t *__restrict__ conn,
                              int n, const int32_t *__restrict__ elem, const double *__restrict__ xi,
                              const double *__restrict__ force, double *f, int *bad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int e = elem[k] - elem_base;
    if (e < 0 || e >= n_elem) return;
    const double x[3] = {xi[3 * k], xi[3 * k + 1], xi[3 * k + 2]};
    if (!(std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2]))) {
        atomicAdd(bad, 1);
        return;
    }
    double sh[27];
    shape_fn(et, x, sh);
    for (int i = 0; i < npe; ++i) {
        const int64_t nd = conn[(int64_t)e * npe + i];
        for (int a = 0; a < 3; ++a) atomicAdd(f + 3 * nd + a, sh[i] * force[3 * k + a]);
    }
}

// Parent face `face` as (a, b) -> xi with tangents: tetrahedra, face k opposite
// barycentric vertex k, L_p = 1 - a - b, L_q = a, L_r = b for the other
// vertices p < q < r; bricks (H8, Q27), face 2 d + s at xi_d = +-1 with (a, b)
// the other coordinates in increasing order.
__device__ void face_point(int et, int face, double a, double b, double xi[3], double ta[3], double tb[3])
{
    if (et == ET_T4 || et == ET_T10) {
        int v[3], m = 0;
        for (int j = 0; j < 4; ++j)
            if (j != face) v[m++] = j;
        double L[4] = {0, 0, 0, 0}, La[4] = {0, 0, 0, 0}, Lb[4] = {0, 0, 0, 0};
        L[v[0]] = 1.0 - a - b;
        L[v[1]] = a;
        L[v[2]] = b;
        La[v[0]] = -1.0;
        La[v[1]] = 1.0;
        Lb[v[0]] = -1.0;
        Lb[v[2]] = 1.0;
        for (int c = 0; c < 3; ++c) {
            xi[c] = L[c + 1];
            ta[c] = La[c + 1];
            tb[c] = Lb[c + 1];
        }
        return;
    }
    const int d = face / 2, s = face % 2;
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    for (int c = 0; c < 3; ++c) ta[c] = tb[c] = 0.0;
    xi[d] = s ? 1.0 : -1.0;
    xi[d1] = a;
    xi[d2] = b;
    ta[d1] = 1.0;
    tb[d2] = 1.0;
}

// Gauss-Legendre nodes and weights on [-1, 1]: 3 points (0, +-sqrt(3/5); 8/9,
// 5/9) and 4 points (+-sqrt(3/7 -+ 2/7 sqrt(6/5)); (18 +- sqrt(30)) / 36)
__device__ void gauss3(int i, double &x, double &w)
{
    const double r = sqrt(0.6);
    x = i == 0 ? -r : (i == 1 ? 0.0 : r);
    w = i == 1 ? 8.0 / 9.0 : 5.0 / 9.0;
}
__device__ void gauss4(int i, double &x, double &w)
{
    const double s = 2.0 / 7.0 * sqrt(1.2);
    const double xi_in = sqrt(3.0 / 7.0 - s), xi_out = sqrt(3.0 / 7.0 + s);
    const double w_in = (18.0 + sqrt(30.0)) / 36.0, w_out = (18.0 - sqrt(30.0)) / 36.0;
    const bool inner = i == 1 || i == 2;
    x = (i < 2 ? -1.0 : 1.0) * (inner ? xi_in : xi_out);
    w = inner ? w_in : w_out;
}

// One thread per (loaded face, face quadrature point): triangle faces take the
// 4 x 4 collapsed Gauss rule (a, b) = (u, (1 - u) v) with weight (1 - u) on the
// unit triangle, quadrilateral faces the 3 x 3 Gauss rule (exact for the
// biquadratic Q27 face functions on a flat face); dA0 = |X_a x X_b|.
__global__ void k_surface_traction(int et, int npe, int elem_base, int n_elem, const int32_t *__restrict__ conn,
                                   const double *__restrict__ X, int n, const int32_t *__restrict__ elem,
                                   const int32_t *__restrict__ face, const double *__restrict__ t0, double *f,
                                   int *bad)
{
    const bool tet = et == ET_T4 || et == ET_T10;
    const int nqf = tet ? 16 : 9;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * nqf) return;
    const int k = (int)(idx / nqf), q = (int)(idx % nqf);
    const int e = elem[k] - elem_base;
    if (e < 0 || e >= n_elem) return;
    const int fc = face[k];
    if (fc < 0 || fc >= (tet ? 4 : 6)) {
        if (q == 0) atomicAdd(bad, 1);
        return;
    }
    double a, b, w;
    if (tet) {
        double xu, wu, xv, wv;
        gauss4(q / 4, xu, wu);
        gauss4(q % 4, xv, wv);
        const double u = 0.5 * (xu + 1.0), v = 0.5 * (xv + 1.0);
        a = u;
        b = (1.0 - u) * v;
        w = 0.25 * wu * wv * (1.0 - u);
    } else {
        double wa, wb;
        gauss3(q / 3, a, wa);
        gauss3(q % 3, b, wb);
        w = wa * wb;
    }
    double xi[3], ta[3], tb[3], sh[27], g[81];
    face_point(et, fc, a, b, xi, ta, tb);
    shape_fn(et, xi, sh);
    parent_grad(et, xi, g);
    double Xa[3] = {0, 0, 0}, Xb[3] = {0, 0, 0};
    for (int i = 0; i < npe; ++i) {
        const int64_t nd = conn[(int64_t)e * npe + i];
        const double ga = g[i * 3] * ta[0] + g[i * 3 + 1] * ta[1] + g[i * 3 + 2] * ta[2];
        const double gb = g[i * 3] * tb[0] + g[i * 3 + 1] * tb[1] + g[i * 3 + 2] * tb[2];
        for (int c = 0; c < 3; ++c) {
            Xa[c] += X[3 * nd + c] * ga;
            Xb[c] += X[3 * nd + c] * gb;
        }
    }
    const double nx = Xa[1] * Xb[2] - Xa[2] * Xb[1], ny = Xa[2] * Xb[0] - Xa[0] * Xb[2],
                 nz = Xa[0] * Xb[1] - Xa[1] * Xb[0];
    const double dA = sqrt(nx * nx + ny * ny + nz * nz) * w;
    for (int i = 0; i < npe; ++i) {
        const int64_t nd = conn[(int64_t)e * npe + i];
        for (int c = 0; c < 3; ++c) atomicAdd(f + 3 * nd + c, sh[i] * t0[3 * k + c] * dA);
    }
}

}  // namespace tlfe

using namespace tlfe;

static tlfe_status loads_check(tlfe_mesh *m, int n, std::initializer_list<const void *> req)
{
    if (!m) return fail(TLFE_E_INVALID, "mesh is NULL");
    if (n < 0) return fail(TLFE_E_INVALID, "negative load count");
    if (n == 0) return TLFE_OK;
    for (const void *p : req)
        if (!p) return fail(TLFE_E_INVALID, "required array pointer is NULL");
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_point_loads(tlfe_mesh *m, int32_t n, const int32_t *elem, const double *xi,
                                        const double *force, double *f, void *stream)
{
    TLFE_TRACE("tlfe_point_loads");
    tlfe_status st = loads_check(m, n, {elem, xi, force, f});
    if (st != TLFE_OK || n == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (const BlockStore &B : m->blocks) {
        if (B.n_elem == 0) continue;
        k_point_loads<<<(n + 127) / 128, 128, 0, s>>>(B.et, B.npe, B.elem_base, B.n_elem, B.d_conn, n, elem, xi,
                                                      force, f, m->d_status + ST_NONFINITE);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "tlfe_point_loads");
    }
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_surface_traction(tlfe_mesh *m, int32_t n, const int32_t *elem, const int32_t *face,
                                             const double *t0, double *f, void *stream)
{
    TLFE_TRACE("tlfe_surface_traction");
    tlfe_status st = loads_check(m, n, {elem, face, t0, f});
    if (st != TLFE_OK || n == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (const BlockStore &B : m->blocks) {
        if (B.n_elem == 0) continue;
        const int nqf = (B.et == ET_T4 || B.et == ET_T10) ? 16 : 9;
        const int64_t work = (int64_t)n * nqf;
        k_surface_traction<<<(unsigned)((work + 127) / 128), 128, 0, s>>>(B.et, B.npe, B.elem_base, B.n_elem,
                                                                          B.d_conn, m->d_X, n, elem, face, t0, f,
                                                                          m->d_status + ST_NONFINITE);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "tlfe_surface_traction");
    }
    return TLFE_OK;
}
