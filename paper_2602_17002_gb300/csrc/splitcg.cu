// Vector kernels of the backward-Euler step of Sec. 7 for one body whose
// elements are split across GPUs (slabs whose interface nodes are held by
// two ranks each).
//
// The host drives the inexact Newton / Jacobi-PCG loop of the step (the same
// iteration as tlfe_newton_step): each operator application on a rank gives
// partial rows at its interface nodes, which the ranks sum through a compact
// buffer (tlfe_gather_nodes, an all-reduce, tlfe_scatter_nodes); each sum over
// rows (a residual norm, the CG dots p.q, r.z, r.r) is a partial sum over the
// rows the rank owns, all-reduced in FP64 by the caller. The kernels here do
// the per-rank vector work between those exchanges:
//
//   tlfe_split_prep      u = u_n + h v, w = v - v_n - h b0 (so that
//                        M/h w = M/h (v - v_n) - f_ff, f_ff = M b0, Sec. 4.2)
//   tlfe_split_residual  g = f_int + M/h w, clamped rows zeroed (Eq. residual)
//   tlfe_split_velocity  v = v_base (+ x), clamped rows zeroed
//   tlfe_split_dot       partial sum of a . b over the owned rows
//   tlfe_split_cg_*      the Jacobi-PCG updates with their partial dots
//
// Sums are FP64 and deterministic: every CTA reduces one chunk of 4096 values
// in a fixed order into the caller's work array, and one warp per sum adds the
// chunk partials in a fixed order.
#include <cuda_runtime.h>

#include <string>

#include "tlfe_mesh.h"

namespace tlfe {

constexpr int SP_CHUNK = 4096;  // values per partial sum (one CTA each)
constexpr int SP_THREADS = 256;

__host__ __device__ inline int sp_chunks(int64_t nv) { return (int)((nv + SP_CHUNK - 1) / SP_CHUNK); }

__device__ __forceinline__ bool sp_fixed(const uint8_t *fixed, int64_t row) { return fixed && fixed[row]; }
__device__ __forceinline__ bool sp_own(const uint8_t *own, int64_t row) { return !own || own[row]; }

// CTA sums of a0 and a1 (fixed order) into work[blockIdx.x], work[nc + blockIdx.x]
__device__ __forceinline__ void sp_store(double a0, double a1, double *work, int nc)
{
    __shared__ double sh[2][SP_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = a0;
        sh[1][w] = a1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < SP_THREADS / 32; ++k) {
            s0 += sh[0][k];
            s1 += sh[1][k];
        }
        work[blockIdx.x] = s0;
        work[nc + blockIdx.x] = s1;
    }
}

// dots[k] = sum of work[k nc + c] over c, k < nd: lane l adds c = l, l + 32,
// ... in order, then a fixed butterfly combines the lanes (one warp per sum)
__global__ void k_sp_finish(const double *__restrict__ work, int nc, int nd, double *__restrict__ dots)
{
    const int k = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (k >= nd) return;
    double s = 0.0;
    for (int c = l; c < nc; c += 32) s += work[(size_t)k * nc + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) dots[k] = s;
}

#define SP_LOOP(i)                                                                       \
    const int64_t sp_b0 = (int64_t)blockIdx.x * SP_CHUNK;                                \
    const int64_t sp_b1 = sp_b0 + SP_CHUNK < nv ? sp_b0 + SP_CHUNK : nv;                 \
    for (int64_t i = sp_b0 + threadIdx.x; i < sp_b1; i += SP_THREADS)

__global__ void k_sp_prep(int64_t nv, double h, double gx, double gy, double gz, const double *__restrict__ u_n,
                          const double *__restrict__ v_n, const double *__restrict__ v, double *__restrict__ u,
                          double *__restrict__ w)
{
    SP_LOOP(i)
    {
        const int c = (int)(i % 3);
        const double b0 = c == 0 ? gx : (c == 1 ? gy : gz);
        const double vi = v[i];
        u[i] = u_n[i] + h * vi;
        w[i] = (vi - v_n[i]) - h * b0;
    }
}

__global__ void k_sp_residual(int64_t nv, const double *__restrict__ f, const double *__restrict__ y,
                              const uint8_t *__restrict__ fixed, double *__restrict__ g)
{
    SP_LOOP(i) g[i] = sp_fixed(fixed, i / 3) ? 0.0 : f[i] + y[i];
}

template <typename R>
__global__ void k_sp_velocity(int64_t nv, const double *__restrict__ vb, const R *__restrict__ x,
                              const uint8_t *__restrict__ fixed, double *__restrict__ v)
{
    SP_LOOP(i) v[i] = sp_fixed(fixed, i / 3) ? 0.0 : vb[i] + (x ? (double)x[i] : 0.0);
}

// the caller's copy of the velocity in the operator's precision (its udot)
template <typename R> __global__ void k_sp_cast(int64_t nv, const double *__restrict__ v, R *__restrict__ out)
{
    SP_LOOP(i) out[i] = (R)v[i];
}

template <typename A>
__global__ void k_sp_dot(int64_t nv, const A *__restrict__ a, const A *__restrict__ b, const uint8_t *__restrict__ own,
                         double *__restrict__ work, int nc)
{
    double s = 0.0;
    SP_LOOP(i)
    {
        if (sp_own(own, i / 3)) s += (double)a[i] * (double)b[i];
    }
    sp_store(s, 0.0, work, nc);
}

template <typename R>
__global__ void k_sp_dinv(int64_t nv, const R *__restrict__ D, const uint8_t *__restrict__ fixed, R *__restrict__ dinv)
{
    SP_LOOP(i)
    {
        const R d = D[i];
        dinv[i] = (sp_fixed(fixed, i / 3) || d == R(0)) ? R(0) : R(1) / d;
    }
}

// x = 0, r = -g (clamped rows 0), p = z = dinv r; partial r.z and r.r
template <typename R>
__global__ void k_sp_start(int64_t nv, const double *__restrict__ g, const R *__restrict__ dinv,
                           const uint8_t *__restrict__ fixed, const uint8_t *__restrict__ own, R *__restrict__ x,
                           R *__restrict__ r, R *__restrict__ p, double *__restrict__ work, int nc)
{
    double rz = 0.0, rr = 0.0;
    SP_LOOP(i)
    {
        const int64_t row = i / 3;
        const R ri = sp_fixed(fixed, row) ? R(0) : (R)(-g[i]);
        const R zi = dinv[i] * ri;
        x[i] = R(0);
        r[i] = ri;
        p[i] = zi;
        if (sp_own(own, row)) {
            rz += (double)ri * (double)zi;
            rr += (double)ri * (double)ri;
        }
    }
    sp_store(rz, rr, work, nc);
}

// q = A p with its clamped rows zeroed; partial p.q
template <typename R>
__global__ void k_sp_pq(int64_t nv, const R *__restrict__ p, R *__restrict__ q, const uint8_t *__restrict__ fixed,
                        const uint8_t *__restrict__ own, double *__restrict__ work, int nc)
{
    double pq = 0.0;
    SP_LOOP(i)
    {
        const int64_t row = i / 3;
        if (sp_fixed(fixed, row)) {
            q[i] = R(0);
        } else if (sp_own(own, row)) {
            pq += (double)p[i] * (double)q[i];
        }
    }
    sp_store(pq, 0.0, work, nc);
}

// x += alpha p, r -= alpha q; partial r.z (z = dinv r) and r.r
template <typename R>
__global__ void k_sp_update(int64_t nv, double alpha, const R *__restrict__ p, const R *__restrict__ q,
                            const R *__restrict__ dinv, const uint8_t *__restrict__ own, R *__restrict__ x,
                            R *__restrict__ r, double *__restrict__ work, int nc)
{
    const R a = (R)alpha;
    double rz = 0.0, rr = 0.0;
    SP_LOOP(i)
    {
        x[i] += a * p[i];
        const R ri = r[i] - a * q[i];
        r[i] = ri;
        if (sp_own(own, i / 3)) {
            const R zi = dinv[i] * ri;
            rz += (double)ri * (double)zi;
            rr += (double)ri * (double)ri;
        }
    }
    sp_store(rz, rr, work, nc);
}

// p = dinv r + beta p
template <typename R>
__global__ void k_sp_direction(int64_t nv, double beta, const R *__restrict__ r, const R *__restrict__ dinv,
                               R *__restrict__ p)
{
    const R b = (R)beta;
    SP_LOOP(i) p[i] = dinv[i] * r[i] + b * p[i];
}

#undef SP_LOOP

static tlfe_status sp_check(const tlfe_split_cg *c, const char *what, bool vecs)
{
    if (!c || c->n_rows < 0 || (c->precision != TLFE_FP32 && c->precision != TLFE_FP64))
        return fail(TLFE_E_INVALID, std::string(what) + ": bad tlfe_split_cg");
    if (vecs && c->n_rows > 0 && (!c->x || !c->r || !c->p || !c->q || !c->dinv))
        return fail(TLFE_E_INVALID, std::string(what) + ": a CG vector is NULL");
    return TLFE_OK;
}

static tlfe_status sp_sums(const tlfe_split_cg *c, const char *what)
{
    if (!c->work || !c->dots) return fail(TLFE_E_INVALID, std::string(what) + ": work or dots is NULL");
    return TLFE_OK;
}

static tlfe_status sp_launched(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TLFE_OK : cuda_fail(e, what);
}

// grid of one CTA per chunk (at least one, so that an empty share still
// writes zero partials), then the fixed-order finish of nd sums
template <typename K> static tlfe_status sp_reduce(const tlfe_split_cg *c, int nd, cudaStream_t s, const char *what,
                                                   K launch)
{
    const int64_t nv = 3 * (int64_t)c->n_rows;
    const int nc = sp_chunks(nv) > 0 ? sp_chunks(nv) : 1;
    launch(nc);
    k_sp_finish<<<1, 64, 0, s>>>(c->work, nc, nd, c->dots);
    return sp_launched(what);
}

}  // namespace tlfe

using namespace tlfe;

extern "C" int64_t tlfe_split_work_doubles(int64_t n_rows)
{
    const int nc = n_rows > 0 ? sp_chunks(3 * n_rows) : 1;
    return 2 * (int64_t)nc;
}

extern "C" tlfe_status tlfe_split_prep(const tlfe_split_cg *c, double h, const double *gravity_host,
                                       const double *u_n, const double *v_n, const double *v, double *u_out,
                                       double *w_out, void *v_op_out, void *stream)
{
    TLFE_TRACE("tlfe_split_prep");
    tlfe_status st = sp_check(c, "tlfe_split_prep", false);
    if (st != TLFE_OK) return st;
    if (!(h > 0.0) || !gravity_host || (c->n_rows > 0 && (!u_n || !v_n || !v || !u_out || !w_out)))
        return fail(TLFE_E_INVALID, "tlfe_split_prep: bad arguments");
    const int64_t nv = 3 * (int64_t)c->n_rows;
    if (nv == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_sp_prep<<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, h, gravity_host[0], gravity_host[1], gravity_host[2], u_n, v_n,
                                                    v, u_out, w_out);
    if (v_op_out) {
        if (c->precision == TLFE_FP32)
            k_sp_cast<float><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, v, (float *)v_op_out);
        else
            k_sp_cast<double><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, v, (double *)v_op_out);
    }
    return sp_launched("tlfe_split_prep");
}

extern "C" tlfe_status tlfe_split_residual(const tlfe_split_cg *c, const double *f, const double *y, double *g,
                                           void *stream)
{
    TLFE_TRACE("tlfe_split_residual");
    tlfe_status st = sp_check(c, "tlfe_split_residual", false);
    if (st != TLFE_OK) return st;
    if (c->n_rows > 0 && (!f || !y || !g)) return fail(TLFE_E_INVALID, "tlfe_split_residual: bad arguments");
    const int64_t nv = 3 * (int64_t)c->n_rows;
    if (nv == 0) return TLFE_OK;
    k_sp_residual<<<sp_chunks(nv), SP_THREADS, 0, (cudaStream_t)stream>>>(nv, f, y, c->fixed, g);
    return sp_launched("tlfe_split_residual");
}

extern "C" tlfe_status tlfe_split_velocity(const tlfe_split_cg *c, const double *v_base, int32_t add_x, double *v_out,
                                           void *stream)
{
    TLFE_TRACE("tlfe_split_velocity");
    tlfe_status st = sp_check(c, "tlfe_split_velocity", false);
    if (st != TLFE_OK) return st;
    if (c->n_rows > 0 && (!v_base || !v_out || (add_x && !c->x)))
        return fail(TLFE_E_INVALID, "tlfe_split_velocity: bad arguments");
    const int64_t nv = 3 * (int64_t)c->n_rows;
    if (nv == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->precision == TLFE_FP32)
        k_sp_velocity<float><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, v_base, add_x ? (const float *)c->x : nullptr,
                                                                   c->fixed, v_out);
    else
        k_sp_velocity<double><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, v_base, add_x ? (const double *)c->x : nullptr,
                                                                    c->fixed, v_out);
    return sp_launched("tlfe_split_velocity");
}

extern "C" tlfe_status tlfe_split_dot(const tlfe_split_cg *c, const double *a, const double *b, void *stream)
{
    TLFE_TRACE("tlfe_split_dot");
    tlfe_status st = sp_check(c, "tlfe_split_dot", false);
    if (st == TLFE_OK) st = sp_sums(c, "tlfe_split_dot");
    if (st != TLFE_OK) return st;
    if (c->n_rows > 0 && (!a || !b)) return fail(TLFE_E_INVALID, "tlfe_split_dot: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nv = 3 * (int64_t)c->n_rows;
    return sp_reduce(c, 1, s, "tlfe_split_dot", [&](int nc) {
        k_sp_dot<double><<<nc, SP_THREADS, 0, s>>>(nv, a, b, c->own, c->work, nc);
    });
}

extern "C" tlfe_status tlfe_split_cg_dinv(const tlfe_split_cg *c, const void *D, void *stream)
{
    TLFE_TRACE("tlfe_split_cg_dinv");
    tlfe_status st = sp_check(c, "tlfe_split_cg_dinv", true);
    if (st != TLFE_OK) return st;
    if (c->n_rows > 0 && !D) return fail(TLFE_E_INVALID, "tlfe_split_cg_dinv: D is NULL");
    const int64_t nv = 3 * (int64_t)c->n_rows;
    if (nv == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->precision == TLFE_FP32)
        k_sp_dinv<float><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, (const float *)D, c->fixed, (float *)c->dinv);
    else
        k_sp_dinv<double><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, (const double *)D, c->fixed, (double *)c->dinv);
    return sp_launched("tlfe_split_cg_dinv");
}

extern "C" tlfe_status tlfe_split_cg_start(const tlfe_split_cg *c, const double *g, void *stream)
{
    TLFE_TRACE("tlfe_split_cg_start");
    tlfe_status st = sp_check(c, "tlfe_split_cg_start", true);
    if (st == TLFE_OK) st = sp_sums(c, "tlfe_split_cg_start");
    if (st != TLFE_OK) return st;
    if (c->n_rows > 0 && !g) return fail(TLFE_E_INVALID, "tlfe_split_cg_start: g is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nv = 3 * (int64_t)c->n_rows;
    return sp_reduce(c, 2, s, "tlfe_split_cg_start", [&](int nc) {
        if (c->precision == TLFE_FP32)
            k_sp_start<float><<<nc, SP_THREADS, 0, s>>>(nv, g, (const float *)c->dinv, c->fixed, c->own,
                                                         (float *)c->x, (float *)c->r, (float *)c->p, c->work, nc);
        else
            k_sp_start<double><<<nc, SP_THREADS, 0, s>>>(nv, g, (const double *)c->dinv, c->fixed, c->own,
                                                          (double *)c->x, (double *)c->r, (double *)c->p, c->work, nc);
    });
}

extern "C" tlfe_status tlfe_split_cg_pq(const tlfe_split_cg *c, void *stream)
{
    TLFE_TRACE("tlfe_split_cg_pq");
    tlfe_status st = sp_check(c, "tlfe_split_cg_pq", true);
    if (st == TLFE_OK) st = sp_sums(c, "tlfe_split_cg_pq");
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nv = 3 * (int64_t)c->n_rows;
    return sp_reduce(c, 1, s, "tlfe_split_cg_pq", [&](int nc) {
        if (c->precision == TLFE_FP32)
            k_sp_pq<float><<<nc, SP_THREADS, 0, s>>>(nv, (const float *)c->p, (float *)c->q, c->fixed, c->own, c->work,
                                                      nc);
        else
            k_sp_pq<double><<<nc, SP_THREADS, 0, s>>>(nv, (const double *)c->p, (double *)c->q, c->fixed, c->own,
                                                       c->work, nc);
    });
}

extern "C" tlfe_status tlfe_split_cg_update(const tlfe_split_cg *c, double alpha, void *stream)
{
    TLFE_TRACE("tlfe_split_cg_update");
    tlfe_status st = sp_check(c, "tlfe_split_cg_update", true);
    if (st == TLFE_OK) st = sp_sums(c, "tlfe_split_cg_update");
    if (st != TLFE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nv = 3 * (int64_t)c->n_rows;
    return sp_reduce(c, 2, s, "tlfe_split_cg_update", [&](int nc) {
        if (c->precision == TLFE_FP32)
            k_sp_update<float><<<nc, SP_THREADS, 0, s>>>(nv, alpha, (const float *)c->p, (const float *)c->q,
                                                          (const float *)c->dinv, c->own, (float *)c->x, (float *)c->r,
                                                          c->work, nc);
        else
            k_sp_update<double><<<nc, SP_THREADS, 0, s>>>(nv, alpha, (const double *)c->p, (const double *)c->q,
                                                           (const double *)c->dinv, c->own, (double *)c->x,
                                                           (double *)c->r, c->work, nc);
    });
}

extern "C" tlfe_status tlfe_split_cg_direction(const tlfe_split_cg *c, double beta, void *stream)
{
    TLFE_TRACE("tlfe_split_cg_direction");
    tlfe_status st = sp_check(c, "tlfe_split_cg_direction", true);
    if (st != TLFE_OK) return st;
    const int64_t nv = 3 * (int64_t)c->n_rows;
    if (nv == 0) return TLFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->precision == TLFE_FP32)
        k_sp_direction<float><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, beta, (const float *)c->r,
                                                                    (const float *)c->dinv, (float *)c->p);
    else
        k_sp_direction<double><<<sp_chunks(nv), SP_THREADS, 0, s>>>(nv, beta, (const double *)c->r,
                                                                     (const double *)c->dinv, (double *)c->p);
    return sp_launched("tlfe_split_cg_direction");
}
