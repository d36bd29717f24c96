// Bilateral constraint primitives of Sec. 3 (DP1, DP2, DIST, CD): point
// evaluation through the shape functions, c(q), and the actions of
// C_q = dc/dq and C_q^T through the element-level blocks (no global C_q is
// formed). FP64 throughout. Used by the tlfe_constraint_* calls and by the
// augmented-Lagrangian Newton step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "tlfe_elem.cuh"
#include "tlfe_mesh.h"

namespace tlfe {

__device__ __forceinline__ int con_npoints(int type) { return (type == 2 || type == 3) ? 4 : 2; }

// per (constraint, point): shape-function values and node ids of the host
// element, found in the block table by global element id
__global__ void k_con_prepare(int n, const tlfe_constraint *__restrict__ cons, ConBlocks bt, double *sh,
                              int32_t *nd, int *bad)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * 4) return;
    const int k = idx / 4, p = idx % 4;
    const tlfe_constraint &c = cons[k];
    double *s = sh + (size_t)idx * CON_MAXN;
    int32_t *d = nd + (size_t)idx * CON_MAXN;
    for (int i = 0; i < CON_MAXN; ++i) {
        s[i] = 0.0;
        d[i] = -1;
    }
    if (c.type < 0 || c.type > 3) {
        if (p == 0) atomicAdd(bad, 1);
        return;
    }
    if (p >= con_npoints(c.type) || c.elem[p] < 0) return;
    const int e = c.elem[p];
    for (int b = 0; b < bt.n; ++b) {
        if (e >= bt.base[b] && e < bt.base[b] + bt.ne[b]) {
            const double xi[3] = {c.xi[p][0], c.xi[p][1], c.xi[p][2]};
            double v[27];
            shape_fn(bt.et[b], xi, v);
            const int npe = nodes_per_elem(bt.et[b]);
            for (int i = 0; i < npe; ++i) {
                s[i] = v[i];
                d[i] = bt.conn[b][(size_t)(e - bt.base[b]) * npe + i];
            }
            return;
        }
    }
    atomicAdd(bad, 1);  // element id outside every block
}

// positions r_p = sum_i s_i (X_i + u_i) of the points of constraint k (u may
// be NULL: the reference configuration); ground points at their coordinates
__device__ void con_positions(int k, const tlfe_constraint &c, const double *__restrict__ sh,
                              const int32_t *__restrict__ nd, const double *__restrict__ X,
                              const double *__restrict__ u, double r[4][3])
{
    const int np = con_npoints(c.type);
    for (int p = 0; p < 4; ++p) {
        for (int a = 0; a < 3; ++a) r[p][a] = 0.0;
        if (p >= np) continue;
        if (c.elem[p] < 0) {
            for (int a = 0; a < 3; ++a) r[p][a] = c.xi[p][a];
            continue;
        }
        const double *s = sh + ((size_t)k * 4 + p) * CON_MAXN;
        const int32_t *d = nd + ((size_t)k * 4 + p) * CON_MAXN;
        for (int i = 0; i < CON_MAXN; ++i) {
            if (d[i] < 0) continue;
            for (int a = 0; a < 3; ++a) r[p][a] += s[i] * (X[3 * (int64_t)d[i] + a] + (u ? u[3 * (int64_t)d[i] + a] : 0.0));
        }
    }
}

// c_k and dc_k/dr_p at q = X + u:
//   CD  : c = d.(r_Q - r_P) - f,        dc/dr_P = -d, dc/dr_Q = d
//   DIST: c = (a.a - f^2)/2, a = r_Q - r_P; dc/dr_P = -a, dc/dr_Q = a
//   DP1 / DP2: c = a.b - f, b = r_T - r_R;  dc/dr_P = -b, dc/dr_Q = b, dc/dr_R = -a, dc/dr_T = a
// times the row weight wrow[k] when wrow is given (the normalised rows of the
// step, Eq. rev_normalized)
__global__ void k_con_eval(int n, const tlfe_constraint *__restrict__ cons, const double *__restrict__ sh,
                           const int32_t *__restrict__ nd, const double *__restrict__ X, const double *__restrict__ u,
                           const double *__restrict__ wrow, double *cval, double *gp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const tlfe_constraint &c = cons[k];
    double r[4][3];
    con_positions(k, c, sh, nd, X, u, r);
    double A[3], B[3], g[4][3];
    for (int a = 0; a < 3; ++a) {
        A[a] = r[1][a] - r[0][a];
        B[a] = r[3][a] - r[2][a];
        for (int p = 0; p < 4; ++p) g[p][a] = 0.0;
    }
    double val;
    if (c.type == 0) {
        val = c.d[0] * A[0] + c.d[1] * A[1] + c.d[2] * A[2] - c.f;
        for (int a = 0; a < 3; ++a) {
            g[0][a] = -c.d[a];
            g[1][a] = c.d[a];
        }
    } else if (c.type == 1) {
        val = 0.5 * (A[0] * A[0] + A[1] * A[1] + A[2] * A[2] - c.f * c.f);
        for (int a = 0; a < 3; ++a) {
            g[0][a] = -A[a];
            g[1][a] = A[a];
        }
    } else {
        val = A[0] * B[0] + A[1] * B[1] + A[2] * B[2] - c.f;
        for (int a = 0; a < 3; ++a) {
            g[0][a] = -B[a];
            g[1][a] = B[a];
            g[2][a] = -A[a];
            g[3][a] = A[a];
        }
    }
    const double w = wrow ? wrow[k] : 1.0;
    cval[k] = w * val;
    for (int p = 0; p < 4; ++p)
        for (int a = 0; a < 3; ++a) gp[((size_t)k * 4 + p) * 3 + a] = w * g[p][a];
}

// Row weights of Eq. row_weights, from the reference configuration: a DP1 row
// (c = a.b - f) gets 1 / sqrt(|a_0|^2 + |b_0|^2), with a_0 = r_Q - r_P and
// b_0 = r_T - r_R at q = X; every other row (CD, DIST, DP2) gets 1, as does a
// DP1 row whose reference directions both vanish.
__global__ void k_con_row_weights(int n, const tlfe_constraint *__restrict__ cons, const double *__restrict__ sh,
                                  const int32_t *__restrict__ nd, const double *__restrict__ X, double *wrow)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const tlfe_constraint &c = cons[k];
    double w = 1.0;
    if (c.type == TLFE_CON_DP1) {
        double r[4][3];
        con_positions(k, c, sh, nd, X, nullptr, r);
        double s2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double A = r[1][a] - r[0][a], B = r[3][a] - r[2][a];
            s2 += A * A + B * B;
        }
        if (s2 > 0.0) w = 1.0 / sqrt(s2);
    }
    wrow[k] = w;
}

// f += scale * C_q^T w, one thread per (constraint, point)
template <typename R>
__global__ void k_con_jt(int n, const double *__restrict__ sh, const int32_t *__restrict__ nd,
                         const double *__restrict__ gp, const double *__restrict__ w, double scale, R *f)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * 4) return;
    const int k = idx / 4;
    const double wk = scale * w[k];
    const double *s = sh + (size_t)idx * CON_MAXN;
    const int32_t *d = nd + (size_t)idx * CON_MAXN;
    const double *g = gp + (size_t)idx * 3;
    for (int i = 0; i < CON_MAXN; ++i) {
        if (d[i] < 0) continue;
        for (int a = 0; a < 3; ++a) atomicAdd(f + 3 * (int64_t)d[i] + a, R(wk * s[i] * g[a]));
    }
}

// out_k = (C_q v)_k (v in FP64, or the FP32 search direction of an FP32 mesh)
template <typename V>
__global__ void k_con_j(int n, const double *__restrict__ sh, const int32_t *__restrict__ nd,
                        const double *__restrict__ gp, const V *__restrict__ v, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double acc = 0.0;
    for (int p = 0; p < 4; ++p) {
        const double *s = sh + ((size_t)k * 4 + p) * CON_MAXN;
        const int32_t *d = nd + ((size_t)k * 4 + p) * CON_MAXN;
        const double *g = gp + ((size_t)k * 4 + p) * 3;
        for (int i = 0; i < CON_MAXN; ++i) {
            if (d[i] < 0) continue;
            for (int a = 0; a < 3; ++a) acc += g[a] * s[i] * v[3 * (int64_t)d[i] + a];
        }
    }
    out[k] = acc;
}

// D += alpha diag(C_q^T C_q) restricted to one point's terms (the Jacobi
// preconditioner of the Gauss-Newton term)
template <typename R>
__global__ void k_con_diag(int n, const double *__restrict__ sh, const int32_t *__restrict__ nd,
                           const double *__restrict__ gp, double alpha, R *D)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * 4) return;
    const double *s = sh + (size_t)idx * CON_MAXN;
    const int32_t *d = nd + (size_t)idx * CON_MAXN;
    const double *g = gp + (size_t)idx * 3;
    for (int i = 0; i < CON_MAXN; ++i) {
        if (d[i] < 0) continue;
        for (int a = 0; a < 3; ++a) atomicAdd(D + 3 * (int64_t)d[i] + a, R(alpha * s[i] * s[i] * g[a] * g[a]));
    }
}

// lam += rho c; w = h (lam + rho c) for the residual term
__global__ void k_con_weights(int n, const double *__restrict__ lam, const double *__restrict__ c, double rho,
                              double h, double *w)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) w[k] = h * (lam[k] + rho * c[k]);
}
__global__ void k_con_lam_update(int n, double *lam, const double *__restrict__ c, double rho)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) lam[k] += rho * c[k];
}

static unsigned grid_of(int64_t n) { return (unsigned)((n + 127) / 128); }

ConBlocks con_blocks(const tlfe_mesh *m)
{
    ConBlocks bt;
    memset(&bt, 0, sizeof(bt));
    for (const BlockStore &B : m->blocks) {
        if (B.n_elem == 0) continue;
        if (bt.n == CON_MAXB) {
            bt.n = -1;
            return bt;
        }
        bt.et[bt.n] = B.et;
        bt.base[bt.n] = B.elem_base;
        bt.ne[bt.n] = B.n_elem;
        bt.conn[bt.n] = B.d_conn;
        ++bt.n;
    }
    return bt;
}

cudaError_t con_prepare(const ConBlocks &bt, int n, const tlfe_constraint *cons, double *sh, int32_t *nd, int *bad,
                        cudaStream_t s)
{
    if (n > 0) k_con_prepare<<<grid_of(4 * (int64_t)n), 128, 0, s>>>(n, cons, bt, sh, nd, bad);
    return cudaGetLastError();
}
cudaError_t con_eval(int n, const tlfe_constraint *cons, const double *sh, const int32_t *nd, const double *X,
                     const double *u, const double *wrow, double *c, double *gp, cudaStream_t s)
{
    if (n > 0) k_con_eval<<<grid_of(n), 128, 0, s>>>(n, cons, sh, nd, X, u, wrow, c, gp);
    return cudaGetLastError();
}
cudaError_t con_row_weights(int n, const tlfe_constraint *cons, const double *sh, const int32_t *nd, const double *X,
                            double *wrow, cudaStream_t s)
{
    if (n > 0) k_con_row_weights<<<grid_of(n), 128, 0, s>>>(n, cons, sh, nd, X, wrow);
    return cudaGetLastError();
}
template <typename R>
cudaError_t con_jt(int n, const double *sh, const int32_t *nd, const double *gp, const double *w, double scale, R *f,
                   cudaStream_t s)
{
    if (n > 0) k_con_jt<R><<<grid_of(4 * (int64_t)n), 128, 0, s>>>(n, sh, nd, gp, w, scale, f);
    return cudaGetLastError();
}
template cudaError_t con_jt<float>(int, const double *, const int32_t *, const double *, const double *, double, float *,
                                   cudaStream_t);
template cudaError_t con_jt<double>(int, const double *, const int32_t *, const double *, const double *, double,
                                    double *, cudaStream_t);
template <typename V>
cudaError_t con_j(int n, const double *sh, const int32_t *nd, const double *gp, const V *v, double *out,
                  cudaStream_t s)
{
    if (n > 0) k_con_j<V><<<grid_of(n), 128, 0, s>>>(n, sh, nd, gp, v, out);
    return cudaGetLastError();
}
template cudaError_t con_j<float>(int, const double *, const int32_t *, const double *, const float *, double *,
                                  cudaStream_t);
template cudaError_t con_j<double>(int, const double *, const int32_t *, const double *, const double *, double *,
                                   cudaStream_t);
template <typename R>
cudaError_t con_diag(int n, const double *sh, const int32_t *nd, const double *gp, double alpha, R *D, cudaStream_t s)
{
    if (n > 0) k_con_diag<R><<<grid_of(4 * (int64_t)n), 128, 0, s>>>(n, sh, nd, gp, alpha, D);
    return cudaGetLastError();
}
template cudaError_t con_diag<float>(int, const double *, const int32_t *, const double *, double, float *, cudaStream_t);
template cudaError_t con_diag<double>(int, const double *, const int32_t *, const double *, double, double *,
                                      cudaStream_t);
cudaError_t con_weights(int n, const double *lam, const double *c, double rho, double h, double *w, cudaStream_t s)
{
    if (n > 0) k_con_weights<<<grid_of(n), 128, 0, s>>>(n, lam, c, rho, h, w);
    return cudaGetLastError();
}
cudaError_t con_lam_update(int n, double *lam, const double *c, double rho, cudaStream_t s)
{
    if (n > 0) k_con_lam_update<<<grid_of(n), 128, 0, s>>>(n, lam, c, rho);
    return cudaGetLastError();
}

}  // namespace tlfe

using namespace tlfe;

// scratch of a standalone call: point data, coefficients and values of the
// mesh handle's constraint scratch (grown by con_setup, freed with the handle;
// every standalone call synchronises its stream before returning, so the next
// call reuses it only after the previous one's kernels have ended)
namespace {
struct ConScratch {
    double *sh = nullptr, *gp = nullptr, *c = nullptr;
    int32_t *nd = nullptr;
    int *bad = nullptr;
};

tlfe_status con_reserve(tlfe_mesh *m, int n)
{
    if (n <= m->con_cap) return TLFE_OK;
    cudaFree(m->d_con_sh);
    cudaFree(m->d_con_nd);
    cudaFree(m->d_con_gp);
    cudaFree(m->d_con_c);
    cudaFree(m->d_con_bad);
    m->d_con_sh = m->d_con_gp = m->d_con_c = nullptr;
    m->d_con_nd = nullptr;
    m->d_con_bad = nullptr;
    m->con_cap = 0;
    const size_t cap = std::max<size_t>((size_t)n, 64);
    if (cudaMalloc(&m->d_con_sh, sizeof(double) * 4 * CON_MAXN * cap) != cudaSuccess ||
        cudaMalloc(&m->d_con_nd, sizeof(int32_t) * 4 * CON_MAXN * cap) != cudaSuccess ||
        cudaMalloc(&m->d_con_gp, sizeof(double) * 12 * cap) != cudaSuccess ||
        cudaMalloc(&m->d_con_c, sizeof(double) * cap) != cudaSuccess ||
        cudaMalloc(&m->d_con_bad, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(TLFE_E_OOM, "constraint scratch");
    }
    m->con_cap = (int)cap;
    return TLFE_OK;
}
}  // namespace

static tlfe_status con_setup(tlfe_mesh *m, int n, const tlfe_constraint *cons, const double *u, ConScratch &cs,
                             cudaStream_t s)
{
    const ConBlocks bt = con_blocks(m);
    if (bt.n < 0) return fail(TLFE_E_UNSUPPORTED, "constraints support at most 16 element blocks");
    tlfe_status st = con_reserve(m, n);
    if (st != TLFE_OK) return st;
    cs.sh = m->d_con_sh;
    cs.nd = m->d_con_nd;
    cs.gp = m->d_con_gp;
    cs.c = m->d_con_c;
    cs.bad = m->d_con_bad;
    cudaError_t e = cudaMemsetAsync(cs.bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = con_prepare(bt, n, cons, cs.sh, cs.nd, cs.bad, s);
    if (e == cudaSuccess) e = con_eval(n, cons, cs.sh, cs.nd, m->d_X, u, nullptr, cs.c, cs.gp, s);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, cs.bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "constraint set-up");
    if (bad) return fail(TLFE_E_INVALID, "constraint with a bad type or an element outside the mesh");
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_constraint_eval(tlfe_mesh *m, int32_t n, const tlfe_constraint *cons, const double *u,
                                            double *c, void *stream)
{
    TLFE_TRACE("tlfe_constraint_eval");
    if (!m || n < 0 || (n > 0 && (!cons || !u || !c))) return fail(TLFE_E_INVALID, "bad constraint arguments");
    if (n == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ConScratch cs;
    tlfe_status st = con_setup(m, n, cons, u, cs, s);
    if (st != TLFE_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c, cs.c, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? TLFE_OK : cuda_fail(e, "tlfe_constraint_eval");
}

extern "C" tlfe_status tlfe_constraint_jt(tlfe_mesh *m, int32_t n, const tlfe_constraint *cons, const double *u,
                                          const double *w, double *f, void *stream)
{
    TLFE_TRACE("tlfe_constraint_jt");
    if (!m || n < 0 || (n > 0 && (!cons || !u || !w || !f))) return fail(TLFE_E_INVALID, "bad constraint arguments");
    if (n == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ConScratch cs;
    tlfe_status st = con_setup(m, n, cons, u, cs, s);
    if (st != TLFE_OK) return st;
    cudaError_t e = con_jt<double>(n, cs.sh, cs.nd, cs.gp, w, 1.0, f, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? TLFE_OK : cuda_fail(e, "tlfe_constraint_jt");
}

extern "C" tlfe_status tlfe_constraint_j(tlfe_mesh *m, int32_t n, const tlfe_constraint *cons, const double *u,
                                         const double *v, double *out, void *stream)
{
    TLFE_TRACE("tlfe_constraint_j");
    if (!m || n < 0 || (n > 0 && (!cons || !u || !v || !out))) return fail(TLFE_E_INVALID, "bad constraint arguments");
    if (n == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ConScratch cs;
    tlfe_status st = con_setup(m, n, cons, u, cs, s);
    if (st != TLFE_OK) return st;
    cudaError_t e = con_j(n, cs.sh, cs.nd, cs.gp, v, out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? TLFE_OK : cuda_fail(e, "tlfe_constraint_j");
}
