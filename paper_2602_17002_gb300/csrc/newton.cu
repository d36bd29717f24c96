// Backward-Euler step of Section 7 (no constraint terms), batched over bodies.
//
//   q(v) = q_n + h v                                   (Eq. step_map_velocity_level)
//   g(v) = M/h (v - v_n) + f_int(q(v), v) - f_ff       (Eq. residual, f_ext = 0)
//
// Inexact Newton: each iteration solves (M/h + h K^e + C) dv = -g, the
// symmetric part of dg/dv = M/h + h K_t + C (the Newton matrix of Sec. 2.2
// without constraint terms, plus the Kelvin-Voigt damping C), by
// Jacobi-preconditioned CG, then v += dv. Bodies are independent: every body
// has its own CG scalars and convergence masks, all bodies advance in
// lockstep, and each stops when ||g_b|| <= newton_rtol ||g_b(v_n)||.
//
// Precision: the residual, the CG vectors, dots and updates are FP64; the
// operator product and the Jacobi diagonal use the mesh precision. For an FP32
// mesh the residual is evaluated on an FP64 twin of the mesh (same description,
// FP64 slab), built on the first call.
//
// Per-body reductions are deterministic: the DOFs of every body (which must
// own one contiguous node range) are cut into fixed chunks; one CTA reduces a
// chunk into a partial, and one thread per body sums its partials in order.
//
// The whole step is one CUDA graph with two nested conditional WHILE nodes
// (Newton outside, CG inside), captured on the first call for a given
// parameter set and replayed afterwards; use_graph = 0 runs the same kernels
// from a host loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tlfe_mesh.h"

namespace tlfe {

constexpr int CHUNK = 4096;  // DOFs per reduction chunk
constexpr int RT = 256;      // threads per chunk CTA
constexpr int UNR = 4;       // DOFs a thread of the CG vector kernels loads before it uses them

enum {
    S_G0 = 0,   // ||g_b(v_n)||
    S_GN,       // ||g_b||
    S_NACT,     // Newton active (1/0)
    S_RZ,       // r . z
    S_R0,       // ||r_0||
    S_RN,       // ||r||
    S_ALPHA,
    S_BETA,
    S_CACT,     // CG active (1/0)
    S_NIT,      // Newton iterations of the body
    S_COUNT
};
enum { I_NEWTON = 0, I_CG, I_CG_TOTAL, I_ANY_N, I_ANY_C, I_COUNT };

struct NewtonState {
    // parameters the captured graph was built for
    double h = 0, grav[3] = {0, 0, 0}, nrtol = 0, crtol = 0;
    int max_newton = 0, max_cg = 0;
    const void *fixed_user = nullptr;
    int use_graph = -1;
    // body / chunk tables
    int nb = 0, n_chunks = 0;
    int32_t *chunk_start = nullptr, *chunk_end = nullptr, *chunk_body = nullptr, *body_chunk_off = nullptr;
    // FP64 vectors [3N] (x, r, p, Dinv: the CG state of an FP64 mesh)
    double *u_n = nullptr, *v_n = nullptr, *v = nullptr, *u_cur = nullptr, *dv = nullptr, *g = nullptr,
           *fff = nullptr, *fgrav = nullptr, *y1 = nullptr, *y2 = nullptr, *x = nullptr, *r = nullptr, *p = nullptr,
           *Dinv = nullptr, *gv = nullptr, *Dd = nullptr;
    // mesh-precision vectors [3N]
    float *ud32 = nullptr, *p32 = nullptr, *Ap32 = nullptr, *D32 = nullptr;
    float *x32 = nullptr, *r32 = nullptr, *Dinv32 = nullptr;  // CG state of an FP32 mesh (p32: its direction)
    uint8_t *fixed = nullptr;  // [N], 1 = clamped (nodes outside every element included)
    double *partials = nullptr;  // [2][n_chunks]
    double *sc = nullptr;        // [S_COUNT][nb]
    int *it = nullptr;           // [I_COUNT]
    tlfe_mesh *twin = nullptr;   // FP64 mesh for the residual (FP32 meshes only)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle hN = 0, hC = 0;
    cudaStream_t s_main = nullptr, s_body = nullptr, s_cg = nullptr;  // capture streams
    std::vector<void *> allocs;
    // augmented-Lagrangian constraints (Sec. 7): one coupled system when present
    int coupled = 0;             // 1: every body in one convergence group
    int n_cons = 0, cap_cons = 0;
    double rho = 0;
    tlfe_constraint *cons = nullptr;               // [cap] copy of the caller's set
    double *con_sh = nullptr, *con_gp = nullptr;   // [cap][4][CON_MAXN], [cap][4][3]
    int32_t *con_nd = nullptr;                     // [cap][4][CON_MAXN]
    double *con_c = nullptr, *con_w = nullptr, *lam = nullptr;  // [cap]
    double *con_wrow = nullptr;                    // [cap] row weights (Eq. row_weights)
    int *con_bad = nullptr;
    int *alm = nullptr;          // [2]: keep the first residual norm as reference; start from the current v
    double *g0keep = nullptr;    // [nb] residual norms of the first Newton solve of the step
};

// ---------------------------------------------------------------------------
// kernels (grid = n_chunks CTAs of RT threads; CTA c owns DOFs [start_c, end_c)
// of body chunk_body[c])
// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    return s;  // valid in thread 0
}

// Sum of the chunk partials k0 <= k < k1 of one body by one warp: lane l adds
// partials k0 + l, k0 + l + 32, ... in that order, then a fixed butterfly
// combines the lanes; every lane returns the same value, and the order does
// not depend on anything but k0 and k1 (deterministic).
__device__ __forceinline__ double warp_body_sum(const double *partials, int k0, int k1)
{
    const int l = threadIdx.x & 31;
    double s = 0.0;
    for (int k = k0 + l; k < k1; k += 32) s += partials[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

struct ChunkArgs {
    const int32_t *start, *end, *body;
    int n_chunks;
};

// u_cur = u_n + h v, dv = v - v_n, and the mesh-precision copies
template <typename R>
__global__ void k_prep(ChunkArgs c, double h, const double *u_n, const double *v, const double *v_n, double *u_cur,
                       double *dv, R *dv_lo, R *ud_lo)
{
    const int ch = blockIdx.x;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) {
        const double uc = u_n[i] + h * v[i];
        u_cur[i] = uc;
        dv[i] = v[i] - v_n[i];
        if (dv_lo) dv_lo[i] = R(dv[i]);
        if (ud_lo) ud_lo[i] = R(v[i]);
    }
}

// g = y1 + y2 - f_ff on free DOFs, 0 on clamped ones (in FP64, y1 and y2 in
// either precision); partial of g.g
template <typename T>
__global__ void k_residual(ChunkArgs c, const T *y1, const T *y2, const double *fff, const uint8_t *fixed,
                           double *g, double *partials)
{
    __shared__ double sh[32];
    const int ch = blockIdx.x;
    double acc = 0.0;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) {
        const double gi = fixed[i / 3] ? 0.0 : double(y1[i]) + double(y2[i]) - fff[i];
        g[i] = gi;
        acc += gi * gi;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[ch] = s;
}

// c = a + b (FP64 node arrays)
__global__ void k_add(int64_t n, const double *a, const double *b, double *c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] + b[i];
}

// Newton convergence test per body; sets the Newton WHILE condition
// (alm[0]: later solves of an augmented-Lagrangian step keep the first
// solve's reference norm g0keep). With low_first, the first residual of the
// solve was evaluated in FP32: it sets the reference norm and the first
// Newton right-hand side but cannot certify convergence, so every body with
// g0 > 0 takes at least one Newton iteration and an FP64 residual decides.
__global__ void k_newton_check(int nb, const int32_t *boff, const double *partials, double *sc, int *it, double rtol,
                               int max_newton, cudaGraphConditionalHandle hN, int use_handle, const int *alm,
                               double *g0keep, int low_first)
{
    int any = 0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int b = threadIdx.x >> 5; b < nb; b += nw) {  // one warp per body
        const double gn = sqrt(warp_body_sum(partials, boff[b], boff[b + 1]));
        if (lane != 0) continue;
        if (it[I_NEWTON] == 0) {
            if (alm[0]) {
                sc[S_G0 * nb + b] = g0keep[b];
            } else {
                sc[S_G0 * nb + b] = gn;
                g0keep[b] = gn;
            }
        }
        sc[S_GN * nb + b] = gn;
        const double g0 = sc[S_G0 * nb + b];
        const bool uncertified = low_first && it[I_NEWTON] == 0;
        const int act = (g0 > 0.0 && (gn > rtol * g0 || uncertified) && it[I_NEWTON] < max_newton) ? 1 : 0;
        sc[S_NACT * nb + b] = act;
        any |= act;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        it[I_ANY_N] = any;
        if (use_handle) cudaGraphSetConditional(hN, any ? 1u : 0u);
    }
}

// Sum of products for the CG dots, per thread, in the vector type V of the CG
// state. FP64 state: a plain FP64 sum. FP32 state: an unevaluated FP32 pair
// (hi, lo), each product split exactly into its rounded value and error by
// one FMA and added with Knuth's two-sum (error-free transformations; the
// sum carries about 44 significant bits), so that the dots keep FP64-class
// accuracy while running on the FP32 pipes (GB300's FP64 rate is about 1/64
// of its FP32 rate, and these kernels would be bound by it). The intrinsics
// keep the compiler from fusing the products into the sums.
template <typename V> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s += a * b; }
    __device__ double value() const { return s; }
};
template <> struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);            // a b = p + e exactly
        const float t = __fadd_rn(hi, p);          // two-sum: hi + p = t + err exactly
        const float bv = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ double value() const { return double(hi) + double(lo); }
};

// Jacobi inverse on free DOFs of Newton-active bodies, in the type of the CG state
template <typename R>
__global__ void k_dinv(ChunkArgs c, const R *D, const uint8_t *fixed, const double *sc, int nb, R *Dinv)
{
    const int ch = blockIdx.x;
    const int b = c.body[ch];
    const bool act = sc[S_NACT * nb + b] != 0.0;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) {
        const R d = D[i];
        Dinv[i] = (act && !fixed[i / 3] && d != R(0)) ? R(1) / d : R(0);
    }
}

// The CG state (x, r, p, Dinv) is held in the mesh precision R: FP64 for an
// FP64 mesh; FP32 for an FP32 mesh, whose operator runs in FP32 anyway. The
// Newton residual g, the step's update v += x and the chunk / body sums of
// the dots stay in FP64; each CG solve only needs the relative tolerance
// cg_rtol, and the Newton iteration corrects the rounding of its solution.

// x = 0, r = -g (active bodies), z = Dinv r, p = z; partials of r.z and r.r
template <typename R>
__global__ void k_cg_init(ChunkArgs c, const double *g, const R *Dinv, const double *sc, int nb, R *x, R *r, R *p,
                          double *partials)
{
    __shared__ double sh[32];
    const int ch = blockIdx.x;
    const int b = c.body[ch];
    const bool act = sc[S_NACT * nb + b] != 0.0;
    DotAcc<R> rz, rr;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) {
        const R ri = act ? R(-g[i]) : R(0);
        const R zi = Dinv[i] * ri;
        x[i] = R(0);
        r[i] = ri;
        p[i] = zi;
        rz.add(ri, zi);
        rr.add(ri, ri);
    }
    const double s1 = block_sum(rz.value(), sh);
    if (threadIdx.x == 0) partials[ch] = s1;
    const double s2 = block_sum(rr.value(), sh);
    if (threadIdx.x == 0) partials[c.n_chunks + ch] = s2;
}

__global__ void k_cg_init_finish(int nb, const int32_t *boff, const double *partials, int n_chunks, double *sc,
                                 int *it, int max_cg, cudaGraphConditionalHandle hC, int use_handle)
{
    int any = 0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int b = threadIdx.x >> 5; b < nb; b += nw) {  // one warp per body
        const double rz = warp_body_sum(partials, boff[b], boff[b + 1]);
        const double rr = warp_body_sum(partials + n_chunks, boff[b], boff[b + 1]);
        if (lane != 0) continue;
        const double r0 = sqrt(rr);
        sc[S_RZ * nb + b] = rz;
        sc[S_R0 * nb + b] = r0;
        sc[S_RN * nb + b] = r0;
        const int act = (sc[S_NACT * nb + b] != 0.0 && r0 > 0.0 && rz > 0.0 && max_cg > 0) ? 1 : 0;
        sc[S_CACT * nb + b] = act;
        any |= act;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        it[I_CG] = 0;
        it[I_ANY_C] = any;
        if (use_handle) cudaGraphSetConditional(hC, any ? 1u : 0u);
    }
}

// partial of p.Ap, Ap the operator product with the clamped DOFs zero
// (k_cg_xr forms the same values again). Each thread loads UNR DOFs before
// it uses them; its sum runs over its DOFs in plain strided order.
template <typename R>
__global__ void k_cg_pap(ChunkArgs c, const R *__restrict__ Ap, const uint8_t *__restrict__ fixed,
                         const R *__restrict__ p, double *partials)
{
    __shared__ double sh[32];
    const int ch = blockIdx.x;
    const int i1 = c.end[ch];
    DotAcc<R> acc;
    for (int i0 = c.start[ch] + threadIdx.x; i0 < i1; i0 += UNR * RT) {
        R a[UNR], q[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int i = i0 + k * RT;
            const bool in = i < i1;
            a[k] = in && !fixed[i / 3] ? Ap[i] : R(0);
            q[k] = in ? p[i] : R(0);
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) acc.add(q[k], a[k]);
    }
    const double s = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[ch] = s;
}

__global__ void k_cg_alpha(int nb, const int32_t *boff, const double *partials, double *sc)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int b = threadIdx.x >> 5; b < nb; b += nw) {  // one warp per body
        const double pap = warp_body_sum(partials, boff[b], boff[b + 1]);
        if (lane != 0) continue;
        const bool act = sc[S_CACT * nb + b] != 0.0 && pap > 0.0;
        if (sc[S_CACT * nb + b] != 0.0 && !(pap > 0.0)) sc[S_CACT * nb + b] = 0.0;  // not SPD here: stop this body
        sc[S_ALPHA * nb + b] = act ? sc[S_RZ * nb + b] / pap : 0.0;
    }
}

// x += alpha p, r -= alpha Ap; partials of r.r and r.z with z = Dinv r (z is
// not stored: k_cg_p forms it again). Ap with the clamped DOFs zeroed, as in
// k_cg_pap.
template <typename R>
__global__ void k_cg_xr(ChunkArgs c, const double *sc, int nb, const R *__restrict__ p, const R *__restrict__ Ap,
                        const uint8_t *__restrict__ fixed, const R *__restrict__ Dinv, R *__restrict__ x,
                        R *__restrict__ r, double *partials)
{
    __shared__ double sh[32];
    const int ch = blockIdx.x;
    const int b = c.body[ch];
    const int i1 = c.end[ch];
    const R alpha = R(sc[S_ALPHA * nb + b]);
    DotAcc<R> rr, rz;
    for (int i0 = c.start[ch] + threadIdx.x; i0 < i1; i0 += UNR * RT) {
        R api[UNR], pi[UNR], xi[UNR], ri[UNR], di[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int i = i0 + k * RT;
            const bool in = i < i1;
            api[k] = in && !fixed[i / 3] ? Ap[i] : R(0);
            pi[k] = in ? p[i] : R(0);
            xi[k] = in ? x[i] : R(0);
            ri[k] = in ? r[i] : R(0);
            di[k] = in ? Dinv[i] : R(0);
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int i = i0 + k * RT;
            const R xn = xi[k] + alpha * pi[k];
            const R rn = ri[k] - alpha * api[k];
            const R zn = di[k] * rn;
            if (i < i1) {
                x[i] = xn;
                r[i] = rn;
            }
            rr.add(rn, rn);
            rz.add(rn, zn);
        }
    }
    const double s1 = block_sum(rr.value(), sh);
    if (threadIdx.x == 0) partials[ch] = s1;
    const double s2 = block_sum(rz.value(), sh);
    if (threadIdx.x == 0) partials[c.n_chunks + ch] = s2;
}

__global__ void k_cg_beta(int nb, const int32_t *boff, const double *partials, int n_chunks, double *sc, int *it,
                          double rtol, int max_cg, cudaGraphConditionalHandle hC, int use_handle)
{
    int any = 0;
    const int itn = it[I_CG] + 1;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int b = threadIdx.x >> 5; b < nb; b += nw) {  // one warp per body
        const double rr = warp_body_sum(partials, boff[b], boff[b + 1]);
        const double rz = warp_body_sum(partials + n_chunks, boff[b], boff[b + 1]);
        if (lane != 0) continue;
        const double rn = sqrt(rr);
        int act = sc[S_CACT * nb + b] != 0.0 ? 1 : 0;
        if (act) {
            sc[S_RN * nb + b] = rn;
            const double rz_old = sc[S_RZ * nb + b];
            sc[S_BETA * nb + b] = rz_old != 0.0 ? rz / rz_old : 0.0;
            sc[S_RZ * nb + b] = rz;
            if (!(rn > rtol * sc[S_R0 * nb + b]) || itn >= max_cg) act = 0;
            sc[S_CACT * nb + b] = act;
        }
        any |= act;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        it[I_CG] = itn;
        it[I_CG_TOTAL] += 1;
        it[I_ANY_C] = any;
        if (use_handle) cudaGraphSetConditional(hC, any ? 1u : 0u);
    }
}

// p = z + beta p with z = Dinv r, on CG-active bodies (unchanged bodies keep
// theirs); p is the operator's next input
template <typename R>
__global__ void k_cg_p(ChunkArgs c, const double *sc, int nb, const R *__restrict__ r, const R *__restrict__ Dinv,
                       R *__restrict__ p)
{
    const int ch = blockIdx.x;
    const int b = c.body[ch];
    if (sc[S_CACT * nb + b] == 0.0) return;
    const R beta = R(sc[S_BETA * nb + b]);
    const int i1 = c.end[ch];
    for (int i0 = c.start[ch] + threadIdx.x; i0 < i1; i0 += UNR * RT) {
        R zi[UNR], pi[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int i = i0 + k * RT;
            const bool in = i < i1;
            zi[k] = in ? Dinv[i] * r[i] : R(0);
            pi[k] = in ? p[i] : R(0);
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const int i = i0 + k * RT;
            if (i < i1) p[i] = zi[k] + beta * pi[k];
        }
    }
}

// v += x on Newton-active bodies (x is zero elsewhere)
template <typename R>
__global__ void k_v_update(ChunkArgs c, const double *sc, int nb, const R *x, double *v)
{
    const int ch = blockIdx.x;
    const int b = c.body[ch];
    if (sc[S_NACT * nb + b] == 0.0) return;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) v[i] += double(x[i]);
}

__global__ void k_newton_count(int nb, double *sc, int *it)
{
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (sc[S_NACT * nb + b] != 0.0) sc[S_NIT * nb + b] += 1.0;
    if (threadIdx.x == 0) it[I_NEWTON] += 1;
}

// v = v_n with clamped DOFs zeroed; counters reset
__global__ void k_start(ChunkArgs c, const uint8_t *fixed, const double *v_n, double *v, const int *alm)
{
    if (alm[1]) return;  // augmented-Lagrangian re-solve: start from the current v
    const int ch = blockIdx.x;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) v[i] = fixed[i / 3] ? 0.0 : v_n[i];
}

__global__ void k_reset(int nb, double *sc, int *it)
{
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int k = 0; k < S_COUNT; ++k) sc[k * nb + b] = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < I_COUNT; ++k) it[k] = 0;
}

// gravity vector field b0 at every node (f_ff = M b0, since sum_j s_j = 1)
__global__ void k_fill_grav(int64_t n_nodes, double gx, double gy, double gz, double *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    out[3 * k] = gx;
    out[3 * k + 1] = gy;
    out[3 * k + 2] = gz;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

#define NCK(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return tlfe::cuda_fail(e_, #call);     \
    } while (0)

template <typename T> static tlfe_status nalloc(NewtonState *ns, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (newton workspace)");
    ns->allocs.push_back(q);
    *p = (T *)q;
    return TLFE_OK;
}

void destroy_newton(tlfe_mesh *m)
{
    NewtonState *ns = m->newton;
    if (!ns) return;
    if (ns->exec) cudaGraphExecDestroy(ns->exec);
    if (ns->graph) cudaGraphDestroy(ns->graph);
    if (ns->s_main) cudaStreamDestroy(ns->s_main);
    if (ns->s_body) cudaStreamDestroy(ns->s_body);
    if (ns->s_cg) cudaStreamDestroy(ns->s_cg);
    for (void *q : ns->allocs) cudaFree(q);
    if (ns->twin) tlfe_destroy_mesh(ns->twin);
    delete ns;
    m->newton = nullptr;
}

// bodies must own contiguous node ranges; builds the chunk tables
static tlfe_status setup_newton(tlfe_mesh *m, cudaStream_t s, int coupled)
{
    NewtonState *ns = new NewtonState();
    m->newton = ns;
    ns->coupled = coupled;
    const int N = m->n_nodes;
    std::vector<int> nstart(m->n_bodies, -1), nend(m->n_bodies, -1);
    int prev = -2;
    std::vector<char> seen(m->n_bodies, 0);
    for (int k = 0; k < N; ++k) {
        const int b = m->node_body[k];
        if (b < 0) {
            prev = -2;
            continue;
        }
        if (b != prev) {
            if (seen[b]) return fail(TLFE_E_UNSUPPORTED, "newton step needs every body to own one contiguous node range");
            seen[b] = 1;
            nstart[b] = k;
        }
        nend[b] = k + 1;
        prev = b;
    }
    // every element's nodes must belong to its own body (bodies do not share nodes)
    for (size_t bi = 0; bi < m->h_conn.size(); ++bi) {
        const int npe = nodes_per_elem(m->h_blocks[bi].type);
        for (size_t e = 0; e < m->h_body[bi].size(); ++e)
            for (int i = 0; i < npe; ++i)
                if (m->node_body[m->h_conn[bi][e * npe + i]] != m->h_body[bi][e])
                    return fail(TLFE_E_UNSUPPORTED, "newton step needs bodies that share no node");
    }
    // convergence groups: one per body, or a single group when constraints
    // may couple bodies
    ns->nb = coupled ? 1 : m->n_bodies;
    std::vector<int32_t> cs, ce, cb, boff(ns->nb + 1, 0);
    for (int b = 0; b < m->n_bodies; ++b) {
        const int grp = coupled ? 0 : b;
        if (nstart[b] >= 0)
            for (int64_t d = 3 * (int64_t)nstart[b]; d < 3 * (int64_t)nend[b]; d += CHUNK) {
                cs.push_back((int32_t)d);
                ce.push_back((int32_t)std::min<int64_t>(d + CHUNK, 3 * (int64_t)nend[b]));
                cb.push_back(grp);
            }
        boff[grp + 1] = (int32_t)cs.size();
    }
    ns->n_chunks = (int)cs.size();
    if (ns->n_chunks == 0) return fail(TLFE_E_INVALID, "no body owns any node");
    const size_t N3 = 3 * (size_t)N;
    tlfe_status st = TLFE_OK;
#define NA(ptr, n)                              \
    if ((st = nalloc(ns, &(ptr), (n))) != TLFE_OK) return st;
    NA(ns->chunk_start, ns->n_chunks);
    NA(ns->chunk_end, ns->n_chunks);
    NA(ns->chunk_body, ns->n_chunks);
    NA(ns->body_chunk_off, ns->nb + 1);
    for (double **q : {&ns->u_n, &ns->v_n, &ns->v, &ns->u_cur, &ns->dv, &ns->g, &ns->fff, &ns->fgrav, &ns->y1, &ns->y2,
                       &ns->gv, &ns->Dd})
        NA(*q, N3);
    for (float **q : {&ns->ud32, &ns->p32, &ns->Ap32, &ns->D32}) NA(*q, N3);
    // the CG state in the mesh precision
    if (m->precision == TLFE_FP32) {
        for (float **q : {&ns->x32, &ns->r32, &ns->Dinv32}) NA(*q, N3);
    } else {
        for (double **q : {&ns->x, &ns->r, &ns->p, &ns->Dinv}) NA(*q, N3);
    }
    NA(ns->fixed, (size_t)N);
    NA(ns->partials, 2 * (size_t)ns->n_chunks);
    NA(ns->sc, (size_t)S_COUNT * ns->nb);
    NA(ns->it, (size_t)I_COUNT);
    NA(ns->alm, 2);
    NA(ns->g0keep, (size_t)ns->nb);
    NA(ns->con_bad, 1);
#undef NA
    NCK(cudaMemcpyAsync(ns->chunk_start, cs.data(), 4 * cs.size(), cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(ns->chunk_end, ce.data(), 4 * ce.size(), cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(ns->chunk_body, cb.data(), 4 * cb.size(), cudaMemcpyHostToDevice, s));
    NCK(cudaMemcpyAsync(ns->body_chunk_off, boff.data(), 4 * boff.size(), cudaMemcpyHostToDevice, s));
    NCK(cudaStreamSynchronize(s));
    NCK(cudaStreamCreateWithFlags(&ns->s_main, cudaStreamNonBlocking));
    NCK(cudaStreamCreateWithFlags(&ns->s_body, cudaStreamNonBlocking));
    NCK(cudaStreamCreateWithFlags(&ns->s_cg, cudaStreamNonBlocking));
    // FP64 twin for the residual of an FP32 mesh
    if (m->precision == TLFE_FP32) {
        tlfe_mesh_desc d;
        memset(&d, 0, sizeof(d));
        d.n_nodes = m->n_nodes;
        d.X_ref = m->h_X.data();
        std::vector<tlfe_block> blocks = m->h_blocks;
        for (size_t bi = 0; bi < blocks.size(); ++bi) {
            blocks[bi].conn = m->h_conn[bi].data();
            blocks[bi].body = m->h_body[bi].data();
        }
        d.n_blocks = (int)blocks.size();
        d.blocks = blocks.data();
        d.n_bodies = m->n_bodies;
        d.body_mat = m->h_mats.data();
        d.elem_mu_lambda = m->h_elam.empty() ? nullptr : m->h_elam.data();
        d.precision = TLFE_FP64;
        d.scatter = m->scatter;
        d.color_seed = m->color_seed;
        d.element_path = m->element_path;
        d.patch_layout = m->patch_layout;
        st = tlfe_create_mesh(&d, s, &ns->twin);
        if (st != TLFE_OK) return st;
    }
    return TLFE_OK;
}

struct StepCtx {
    tlfe_mesh *m;
    NewtonState *ns;
    ChunkArgs c;
    int use_handle;
};

// --- building blocks, all stream-ordered on s --------------------------------

// Residual g(v) of Eq. residual at the current v, its per-body norms and the
// Newton test. Evaluated with the FP64 twin mesh (FP64 element arithmetic), so
// that it can certify relative residuals near 1e-8; with `first` on an FP32
// mesh without constraints, the step's first residual is evaluated with the
// FP32 kernels instead (it only sets g0 and the first right-hand side, which
// CG solves to cg_rtol anyway; k_newton_check then does not accept it as
// converged). Scratch for that FP32 evaluation: p32 (v - v_n), Ap32 (mass
// product), D32 (force), all set later by the CG set-up.
static tlfe_status enq_residual(const StepCtx &x, cudaStream_t s, bool first)
{
    NewtonState *ns = x.ns;
    tlfe_mesh *m64 = ns->twin ? ns->twin : x.m;
    const int nc = ns->n_chunks;
    const bool low = first && x.m->precision == TLFE_FP32 && ns->n_cons == 0;
    if (x.m->precision == TLFE_FP32)
        k_prep<float><<<nc, RT, 0, s>>>(x.c, ns->h, ns->u_n, ns->v, ns->v_n, ns->u_cur, ns->dv, low ? ns->p32 : nullptr,
                                        ns->ud32);
    else
        k_prep<double><<<nc, RT, 0, s>>>(x.c, ns->h, ns->u_n, ns->v, ns->v_n, ns->u_cur, ns->dv, nullptr, nullptr);
    NCK(cudaGetLastError());
    tlfe_status st;
    if (low) {
        st = run_op<OP_MATVEC, float>(x.m, ns->u_cur, ns->ud32, ns->p32, ns->Ap32, nullptr, nullptr, 1.0 / ns->h, 0.0,
                                      0.0, 0, s);
        if (st != TLFE_OK) return st;
        st = run_op<OP_FORCE, float>(x.m, ns->u_cur, ns->ud32, nullptr, ns->D32, nullptr, nullptr, 0.0, 1.0, 0.0, 0, s);
        if (st != TLFE_OK) return st;
        k_residual<float><<<nc, RT, 0, s>>>(x.c, ns->Ap32, ns->D32, ns->fff, ns->fixed, ns->g, ns->partials);
    } else {
        st = run_op<OP_MATVEC, double>(m64, ns->u_cur, ns->v, ns->dv, ns->y1, nullptr, nullptr, 1.0 / ns->h, 0.0, 0.0, 0,
                                       s);
        if (st != TLFE_OK) return st;
        st = run_op<OP_FORCE, double>(m64, ns->u_cur, ns->v, nullptr, ns->y2, nullptr, nullptr, 0.0, 1.0, 0.0, 0, s);
        if (st != TLFE_OK) return st;
        if (ns->n_cons > 0) {
            // + h C_q^T (lambda + rho c) at q(v) (Eq. residual)
            NCK(con_eval(ns->n_cons, ns->cons, ns->con_sh, ns->con_nd, x.m->d_X, ns->u_cur, ns->con_wrow, ns->con_c,
                         ns->con_gp, s));
            NCK(con_weights(ns->n_cons, ns->lam, ns->con_c, ns->rho, ns->h, ns->con_w, s));
            NCK(con_jt<double>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, ns->con_w, 1.0, ns->y2, s));
        }
        k_residual<double><<<nc, RT, 0, s>>>(x.c, ns->y1, ns->y2, ns->fff, ns->fixed, ns->g, ns->partials);
    }
    k_newton_check<<<1, 1024, 0, s>>>(ns->nb, ns->body_chunk_off, ns->partials, ns->sc, ns->it, ns->nrtol,
                                       ns->max_newton, ns->hN, x.use_handle, ns->alm, ns->g0keep, low ? 1 : 0);
    NCK(cudaGetLastError());
    return TLFE_OK;
}

static tlfe_status enq_cg_init(const StepCtx &x, cudaStream_t s)
{
    NewtonState *ns = x.ns;
    const int nc = ns->n_chunks;
    const double h = ns->h;
    tlfe_status st;
    if (x.m->precision == TLFE_FP32) {
        st = run_op<OP_DIAG, float>(x.m, ns->u_cur, ns->ud32, nullptr, ns->D32, nullptr, nullptr, 1.0 / h, h, 1.0, 1, s);
        if (st != TLFE_OK) return st;
        if (ns->n_cons > 0)
            NCK(con_diag<float>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, h * h * ns->rho, ns->D32, s));
        k_dinv<float><<<nc, RT, 0, s>>>(x.c, ns->D32, ns->fixed, ns->sc, ns->nb, ns->Dinv32);
    } else {
        st = run_op<OP_DIAG, double>(x.m, ns->u_cur, ns->v, nullptr, ns->Dd, nullptr, nullptr, 1.0 / h, h, 1.0, 1, s);
        if (st != TLFE_OK) return st;
        if (ns->n_cons > 0)
            NCK(con_diag<double>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, h * h * ns->rho, ns->Dd, s));
        k_dinv<double><<<nc, RT, 0, s>>>(x.c, ns->Dd, ns->fixed, ns->sc, ns->nb, ns->Dinv);
    }
    if (x.m->precision == TLFE_FP32)
        k_cg_init<float><<<nc, RT, 0, s>>>(x.c, ns->g, ns->Dinv32, ns->sc, ns->nb, ns->x32, ns->r32, ns->p32,
                                           ns->partials);
    else
        k_cg_init<double><<<nc, RT, 0, s>>>(x.c, ns->g, ns->Dinv, ns->sc, ns->nb, ns->x, ns->r, ns->p, ns->partials);
    k_cg_init_finish<<<1, 1024, 0, s>>>(ns->nb, ns->body_chunk_off, ns->partials, nc, ns->sc, ns->it, ns->max_cg,
                                         ns->hC, x.use_handle);
    NCK(cudaGetLastError());
    return TLFE_OK;
}

static tlfe_status enq_cg_iter(const StepCtx &x, cudaStream_t s)
{
    NewtonState *ns = x.ns;
    const int nc = ns->n_chunks;
    const double h = ns->h;
    tlfe_status st;
    if (x.m->precision == TLFE_FP32) {  // p32: the FP32 search direction, kept by k_cg_init / k_cg_p
        st = run_op<OP_MATVEC, float>(x.m, ns->u_cur, ns->ud32, ns->p32, ns->Ap32, nullptr, nullptr, 1.0 / h, h, 1.0,
                                      1, s);
        if (st != TLFE_OK) return st;
        if (ns->n_cons > 0) {  // + h^2 rho C_q^T C_q p (Gauss-Newton)
            NCK(con_j<float>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, ns->p32, ns->con_w, s));
            NCK(con_jt<float>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, ns->con_w, h * h * ns->rho, ns->Ap32, s));
        }
        k_cg_pap<float><<<nc, RT, 0, s>>>(x.c, ns->Ap32, ns->fixed, ns->p32, ns->partials);
    } else {
        st = run_op<OP_MATVEC, double>(x.m, ns->u_cur, ns->v, ns->p, ns->y1, nullptr, nullptr, 1.0 / h, h, 1.0, 1, s);
        if (st != TLFE_OK) return st;
        if (ns->n_cons > 0) {
            NCK(con_j<double>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, ns->p, ns->con_w, s));
            NCK(con_jt<double>(ns->n_cons, ns->con_sh, ns->con_nd, ns->con_gp, ns->con_w, h * h * ns->rho, ns->y1, s));
        }
        k_cg_pap<double><<<nc, RT, 0, s>>>(x.c, ns->y1, ns->fixed, ns->p, ns->partials);
    }
    k_cg_alpha<<<1, 1024, 0, s>>>(ns->nb, ns->body_chunk_off, ns->partials, ns->sc);
    if (x.m->precision == TLFE_FP32)
        k_cg_xr<float><<<nc, RT, 0, s>>>(x.c, ns->sc, ns->nb, ns->p32, ns->Ap32, ns->fixed, ns->Dinv32, ns->x32,
                                         ns->r32, ns->partials);
    else
        k_cg_xr<double><<<nc, RT, 0, s>>>(x.c, ns->sc, ns->nb, ns->p, ns->y1, ns->fixed, ns->Dinv, ns->x, ns->r,
                                          ns->partials);
    k_cg_beta<<<1, 1024, 0, s>>>(ns->nb, ns->body_chunk_off, ns->partials, nc, ns->sc, ns->it, ns->crtol, ns->max_cg,
                                  ns->hC, x.use_handle);
    if (x.m->precision == TLFE_FP32)
        k_cg_p<float><<<nc, RT, 0, s>>>(x.c, ns->sc, ns->nb, ns->r32, ns->Dinv32, ns->p32);
    else
        k_cg_p<double><<<nc, RT, 0, s>>>(x.c, ns->sc, ns->nb, ns->r, ns->Dinv, ns->p);
    NCK(cudaGetLastError());
    return TLFE_OK;
}

static tlfe_status enq_newton_tail(const StepCtx &x, cudaStream_t s)
{
    NewtonState *ns = x.ns;
    if (x.m->precision == TLFE_FP32)
        k_v_update<float><<<ns->n_chunks, RT, 0, s>>>(x.c, ns->sc, ns->nb, ns->x32, ns->v);
    else
        k_v_update<double><<<ns->n_chunks, RT, 0, s>>>(x.c, ns->sc, ns->nb, ns->x, ns->v);
    k_newton_count<<<1, 1024, 0, s>>>(ns->nb, ns->sc, ns->it);
    NCK(cudaGetLastError());
    return enq_residual(x, s, false);
}

static tlfe_status enq_prologue(const StepCtx &x, cudaStream_t s)
{
    NewtonState *ns = x.ns;
    k_reset<<<1, 1024, 0, s>>>(ns->nb, ns->sc, ns->it);
    k_start<<<ns->n_chunks, RT, 0, s>>>(x.c, ns->fixed, ns->v_n, ns->v, ns->alm);
    NCK(cudaGetLastError());
    return enq_residual(x, s, true);
}

// add a conditional WHILE node to the graph being captured on `s`; returns its body graph
static tlfe_status add_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    NCK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
    if (cs != cudaStreamCaptureStatusActive) return fail(TLFE_E_CUDA, "stream is not capturing");
    // cudaGraphNodeParams has no usable default constructor: zero a buffer
    alignas(cudaGraphNodeParams) unsigned char buf[sizeof(cudaGraphNodeParams)];
    memset(buf, 0, sizeof(buf));
    cudaGraphNodeParams *cp = reinterpret_cast<cudaGraphNodeParams *>(buf);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = h;
    cp->conditional.type = cudaGraphCondTypeWhile;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    NCK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, cp));
    NCK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = cp->conditional.phGraph_out[0];
    return TLFE_OK;
}

// Captures on the step's own streams (the caller's stream may be the legacy
// default stream, which cannot be captured); the graph is launched on the
// caller's stream afterwards.
static tlfe_status build_graph(StepCtx &x)
{
    NewtonState *ns = x.ns;
    cudaStream_t s = ns->s_main;
    if (ns->exec) {
        cudaGraphExecDestroy(ns->exec);
        ns->exec = nullptr;
    }
    if (ns->graph) {
        cudaGraphDestroy(ns->graph);
        ns->graph = nullptr;
    }
    NCK(cudaGraphCreate(&ns->graph, 0));
    NCK(cudaGraphConditionalHandleCreate(&ns->hN, ns->graph, 0, 0));
    x.use_handle = 1;
    // main graph: prologue, Newton WHILE
    NCK(cudaStreamBeginCaptureToGraph(s, ns->graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    tlfe_status st = enq_prologue(x, s);
    cudaGraph_t body_n = nullptr;
    if (st == TLFE_OK) st = add_while(s, ns->hN, &body_n);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != TLFE_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "end capture (main)");
    // Newton body: Jacobi + CG init, CG WHILE, update + residual
    NCK(cudaGraphConditionalHandleCreate(&ns->hC, body_n, 0, 0));
    NCK(cudaStreamBeginCaptureToGraph(ns->s_body, body_n, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    st = enq_cg_init(x, ns->s_body);
    cudaGraph_t body_c = nullptr;
    if (st == TLFE_OK) st = add_while(ns->s_body, ns->hC, &body_c);
    if (st == TLFE_OK) st = enq_newton_tail(x, ns->s_body);
    e = cudaStreamEndCapture(ns->s_body, &g);
    if (st != TLFE_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "end capture (newton body)");
    // CG body
    NCK(cudaStreamBeginCaptureToGraph(ns->s_cg, body_c, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    st = enq_cg_iter(x, ns->s_cg);
    e = cudaStreamEndCapture(ns->s_cg, &g);
    if (st != TLFE_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "end capture (cg body)");
    NCK(cudaGraphInstantiate(&ns->exec, ns->graph, 0));
    return TLFE_OK;
}

// warm the per-kernel occupancy caches outside any capture
static tlfe_status warm(StepCtx &x, cudaStream_t s)
{
    x.use_handle = 0;
    tlfe_status st = enq_prologue(x, s);
    if (st == TLFE_OK) st = enq_cg_init(x, s);
    if (st == TLFE_OK && x.ns->max_cg > 0) st = enq_cg_iter(x, s);
    if (st != TLFE_OK) return st;
    NCK(cudaStreamSynchronize(s));
    return TLFE_OK;
}

// partial of x.x per chunk
__global__ void k_sq_partials(ChunkArgs c, const double *x, double *partials)
{
    __shared__ double sh[32];
    const int ch = blockIdx.x;
    double acc = 0.0;
    for (int i = c.start[ch] + threadIdx.x; i < c.end[ch]; i += blockDim.x) acc += x[i] * x[i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[ch] = s;
}

__global__ void k_body_norms(int nb, const int32_t *boff, const double *partials, double *out)
{
    for (int b = threadIdx.x >> 5; b < nb; b += blockDim.x >> 5) {  // one warp per body
        const double s = warp_body_sum(partials, boff[b], boff[b + 1]);
        if ((threadIdx.x & 31) == 0) out[b] = sqrt(s);
    }
}

}  // namespace tlfe

using namespace tlfe;

namespace tlfe {
tlfe_mesh *newton_twin(tlfe_mesh *m) { return m->newton ? m->newton->twin : nullptr; }
}  // namespace tlfe

extern "C" tlfe_status tlfe_body_norms(tlfe_mesh *m, const double *x, double *out, void *stream)
{
    TLFE_TRACE("tlfe_body_norms");
    if (!m || !x || !out) return fail(TLFE_E_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    // per-body tables (a workspace built for a coupled, constrained step has one group)
    if (m->newton && m->newton->coupled) destroy_newton(m);
    if (!m->newton) {
        tlfe_status st = setup_newton(m, s, 0);
        if (st != TLFE_OK) {
            destroy_newton(m);
            return st;
        }
        NCK(cudaMemsetAsync(m->newton->alm, 0, 2 * sizeof(int), s));
    }
    NewtonState *ns = m->newton;
    ChunkArgs c{ns->chunk_start, ns->chunk_end, ns->chunk_body, ns->n_chunks};
    k_sq_partials<<<ns->n_chunks, RT, 0, s>>>(c, x, ns->partials);
    k_body_norms<<<1, 1024, 0, s>>>(ns->nb, ns->body_chunk_off, ns->partials, out);
    NCK(cudaGetLastError());
    return TLFE_OK;
}

// One Newton solve of the step (graph replay or host-driven loop) and its
// per-group residual report.
static tlfe_status newton_solve(StepCtx &x, const tlfe_step_params *prm, tlfe_step_report *rep, cudaStream_t s)
{
    NewtonState *ns = x.ns;
    tlfe_status st;
    if (ns->use_graph == 1 && prm->use_graph) {
        NCK(cudaGraphLaunch(ns->exec, s));
    } else {
        // host-driven loop over the same kernels
        x.use_handle = 0;
        st = enq_prologue(x, s);
        if (st != TLFE_OK) return st;
        int flags[I_COUNT];
        for (;;) {
            NCK(cudaMemcpyAsync(flags, ns->it, sizeof(flags), cudaMemcpyDeviceToHost, s));
            NCK(cudaStreamSynchronize(s));
            if (!flags[I_ANY_N]) break;
            st = enq_cg_init(x, s);
            if (st != TLFE_OK) return st;
            for (;;) {
                NCK(cudaMemcpyAsync(flags, ns->it, sizeof(flags), cudaMemcpyDeviceToHost, s));
                NCK(cudaStreamSynchronize(s));
                if (!flags[I_ANY_C]) break;
                st = enq_cg_iter(x, s);
                if (st != TLFE_OK) return st;
            }
            st = enq_newton_tail(x, s);
            if (st != TLFE_OK) return st;
        }
    }
    std::vector<double> sc((size_t)S_COUNT * ns->nb);
    int it[I_COUNT];
    NCK(cudaMemcpyAsync(sc.data(), ns->sc, 8 * sc.size(), cudaMemcpyDeviceToHost, s));
    NCK(cudaMemcpyAsync(it, ns->it, sizeof(it), cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    int conv = 0, nit = 0;
    double worst = 0.0;
    for (int b = 0; b < ns->nb; ++b) {
        const double g0 = sc[S_G0 * ns->nb + b], gn = sc[S_GN * ns->nb + b];
        if (!(g0 > 0.0)) {
            ++conv;  // nothing to solve for this group (or it owns no node)
            continue;
        }
        const double rel = gn / g0;
        worst = std::max(worst, rel);
        if (rel <= prm->newton_rtol) ++conv;
        nit = std::max(nit, (int)sc[S_NIT * ns->nb + b]);
    }
    rep->newton_iters += nit;
    rep->cg_iters += it[I_CG_TOTAL];
    rep->n_bodies_converged = conv;
    rep->rel_residual = worst;
    rep->status = conv == ns->nb ? TLFE_OK : TLFE_E_NOT_CONVERGED;
    return TLFE_OK;
}

// constraint workspace for n constraints (the graph captures its pointers)
static tlfe_status ensure_constraints(NewtonState *ns, int n)
{
    if (n <= ns->cap_cons) return TLFE_OK;
    tlfe_status st;
    tlfe_constraint *c = nullptr;
    cudaError_t e = cudaMalloc(&c, sizeof(tlfe_constraint) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (constraints)");
    ns->allocs.push_back(c);
    ns->cons = c;
    if ((st = nalloc(ns, &ns->con_sh, (size_t)n * 4 * CON_MAXN)) != TLFE_OK) return st;
    if ((st = nalloc(ns, &ns->con_nd, (size_t)n * 4 * CON_MAXN)) != TLFE_OK) return st;
    if ((st = nalloc(ns, &ns->con_gp, (size_t)n * 12)) != TLFE_OK) return st;
    if ((st = nalloc(ns, &ns->con_c, (size_t)n)) != TLFE_OK) return st;
    if ((st = nalloc(ns, &ns->con_w, (size_t)n)) != TLFE_OK) return st;
    if ((st = nalloc(ns, &ns->con_wrow, (size_t)n)) != TLFE_OK) return st;
    if ((st = nalloc(ns, &ns->lam, (size_t)n)) != TLFE_OK) return st;
    ns->cap_cons = n;
    ns->use_graph = -1;  // buffers moved: the graph is rebuilt
    return TLFE_OK;
}

extern "C" tlfe_status tlfe_newton_step(tlfe_mesh *m, const double *u_n, const double *v_n,
                                        const tlfe_step_params *prm, double *v_out, tlfe_step_report *rep,
                                        void *stream)
{
    TLFE_TRACE("tlfe_newton_step");
    if (!m || !u_n || !v_n || !prm || !v_out || !rep) return fail(TLFE_E_INVALID, "NULL argument");
    memset(rep, 0, sizeof(*rep));
    if (!(prm->h > 0.0) || !std::isfinite(prm->h) || !(prm->newton_rtol >= 0.0) || !(prm->cg_rtol >= 0.0) ||
        prm->max_newton < 0 || prm->max_cg < 0)
        return fail(TLFE_E_INVALID, "bad step parameters");
    const int n_cons = prm->n_cons;
    if (n_cons < 0 || (n_cons > 0 && (!prm->cons_dev || !prm->lambda_dev || !(prm->rho > 0.0) ||
                                      !std::isfinite(prm->rho) || !(prm->alm_tol >= 0.0) || prm->max_outer < 0)))
        return fail(TLFE_E_INVALID, "bad constraint parameters");
    for (auto &B : m->blocks)
        if (B.n_elem > 0 && !B.affine) return fail(TLFE_E_UNSUPPORTED, "newton step needs affine elements (consistent mass)");
    cudaStream_t s = (cudaStream_t)stream;
    tlfe_status st;
    const int coupled = n_cons > 0 ? 1 : 0;
    if (m->newton && m->newton->coupled != coupled) destroy_newton(m);
    if (!m->newton) {
        st = setup_newton(m, s, coupled);
        if (st != TLFE_OK) {
            destroy_newton(m);
            return st;
        }
        NCK(cudaMemsetAsync(m->newton->alm, 0, 2 * sizeof(int), s));
    }
    NewtonState *ns = m->newton;
    const size_t N = (size_t)m->n_nodes, N3 = 3 * N;
    if (n_cons > 0) {
        st = ensure_constraints(ns, n_cons);
        if (st != TLFE_OK) return st;
        const ConBlocks bt = con_blocks(m);
        if (bt.n < 0) return fail(TLFE_E_UNSUPPORTED, "constraints support at most 16 element blocks");
        int bad = 0;
        NCK(cudaMemcpyAsync(ns->cons, prm->cons_dev, sizeof(tlfe_constraint) * (size_t)n_cons,
                            cudaMemcpyDeviceToDevice, s));
        NCK(cudaMemsetAsync(ns->con_bad, 0, sizeof(int), s));
        NCK(con_prepare(bt, n_cons, ns->cons, ns->con_sh, ns->con_nd, ns->con_bad, s));
        // constant row weights from the reference configuration (Eq. row_weights):
        // the step works on the normalised rows w_k c_k (Eq. rev_normalized)
        NCK(con_row_weights(n_cons, ns->cons, ns->con_sh, ns->con_nd, m->d_X, ns->con_wrow, s));
        NCK(cudaMemcpyAsync(&bad, ns->con_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        if (bad) return fail(TLFE_E_INVALID, "constraint with a bad type or an element outside the mesh");
    }
    const bool same = ns->use_graph >= 0 && ns->h == prm->h && ns->grav[0] == prm->gravity[0] &&
                      ns->grav[1] == prm->gravity[1] && ns->grav[2] == prm->gravity[2] &&
                      ns->nrtol == prm->newton_rtol && ns->crtol == prm->cg_rtol && ns->max_newton == prm->max_newton &&
                      ns->max_cg == prm->max_cg && ns->fixed_user == (const void *)prm->fixed_dev &&
                      ns->n_cons == n_cons && (n_cons == 0 || ns->rho == prm->rho);
    StepCtx x{m, ns, {ns->chunk_start, ns->chunk_end, ns->chunk_body, ns->n_chunks}, 0};
    if (!same) {
        ns->h = prm->h;
        memcpy(ns->grav, prm->gravity, sizeof(ns->grav));
        ns->nrtol = prm->newton_rtol;
        ns->crtol = prm->cg_rtol;
        ns->max_newton = prm->max_newton;
        ns->max_cg = prm->max_cg;
        ns->fixed_user = prm->fixed_dev;
        ns->n_cons = n_cons;
        ns->rho = prm->rho;
        // clamped nodes: user's flags, plus nodes outside every element
        std::vector<uint8_t> fx(N, 0);
        if (prm->fixed_dev) NCK(cudaMemcpy(fx.data(), prm->fixed_dev, N, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < N; ++k)
            if (m->node_body[k] < 0) fx[k] = 1;
        NCK(cudaMemcpy(ns->fixed, fx.data(), N, cudaMemcpyHostToDevice));
        // f_ff = M b0 (Eq. virtual_work_force_field_uniform with sum_j s_j = 1)
        NCK(cudaMemcpyAsync(ns->u_n, u_n, 8 * N3, cudaMemcpyDeviceToDevice, s));
        k_fill_grav<<<(unsigned)((N + 255) / 256), 256, 0, s>>>((int64_t)N, prm->gravity[0], prm->gravity[1],
                                                                prm->gravity[2], ns->gv);
        NCK(cudaGetLastError());
        tlfe_mesh *m64 = ns->twin ? ns->twin : m;
        st = run_op<OP_MATVEC, double>(m64, ns->u_n, nullptr, ns->gv, ns->fgrav, nullptr, nullptr, 1.0, 0.0, 0.0, 0, s);
        if (st != TLFE_OK) return st;
        NCK(cudaMemcpyAsync(ns->fff, ns->fgrav, 8 * N3, cudaMemcpyDeviceToDevice, s));
        NCK(cudaMemcpyAsync(ns->v_n, v_n, 8 * N3, cudaMemcpyDeviceToDevice, s));
        if (n_cons > 0)
            NCK(cudaMemcpyAsync(ns->lam, prm->lambda_dev, sizeof(double) * (size_t)n_cons, cudaMemcpyDeviceToDevice, s));
        NCK(cudaMemsetAsync(ns->alm, 0, 2 * sizeof(int), s));
        st = warm(x, s);
        if (st != TLFE_OK) return st;
        ns->use_graph = prm->use_graph ? 1 : 0;
        if (prm->use_graph) {
            NCK(cudaStreamSynchronize(s));
            st = build_graph(x);
            if (st != TLFE_OK) {
                ns->use_graph = -1;
                return st;
            }
        }
    }
    // inputs into the workspace (the graph only ever sees workspace pointers)
    NCK(cudaMemcpyAsync(ns->u_n, u_n, 8 * N3, cudaMemcpyDeviceToDevice, s));
    NCK(cudaMemcpyAsync(ns->v_n, v_n, 8 * N3, cudaMemcpyDeviceToDevice, s));
    if (n_cons > 0)
        NCK(cudaMemcpyAsync(ns->lam, prm->lambda_dev, sizeof(double) * (size_t)n_cons, cudaMemcpyDeviceToDevice, s));
    // applied load of this step: f_ff + f_ext (Sec. 4), read by the residual
    if (prm->f_ext_dev) {
        k_add<<<(unsigned)((N3 + 255) / 256), 256, 0, s>>>((int64_t)N3, ns->fgrav, prm->f_ext_dev, ns->fff);
        NCK(cudaGetLastError());
    } else {
        NCK(cudaMemcpyAsync(ns->fff, ns->fgrav, 8 * N3, cudaMemcpyDeviceToDevice, s));
    }
    // the Newton solve; with constraints, the augmented-Lagrangian loop of
    // Sec. 7 around it (later solves warm-start and keep the first reference)
    static const int flags0[2] = {0, 0}, flags1[2] = {1, 1};
    NCK(cudaMemcpyAsync(ns->alm, flags0, sizeof(flags0), cudaMemcpyHostToDevice, s));
    std::vector<double> ch((size_t)std::max(0, n_cons));
    for (int outer = 0;; ++outer) {
        st = newton_solve(x, prm, rep, s);
        if (st != TLFE_OK) return st;
        if (n_cons == 0) break;
        // c at the solution (the last residual evaluated it at q(v))
        NCK(cudaMemcpyAsync(ch.data(), ns->con_c, sizeof(double) * (size_t)n_cons, cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        double cn = 0.0;
        for (double c : ch) cn += c * c;
        rep->c_norm = std::sqrt(cn);
        rep->outer_iters = outer;
        if (rep->c_norm <= prm->alm_tol || outer >= prm->max_outer) break;
        NCK(con_lam_update(n_cons, ns->lam, ns->con_c, ns->rho, s));  // Eq. alm_multiplier_update
        NCK(cudaMemcpyAsync(ns->alm, flags1, sizeof(flags1), cudaMemcpyHostToDevice, s));
    }
    if (n_cons > 0) {
        NCK(cudaMemcpyAsync(prm->lambda_dev, ns->lam, sizeof(double) * (size_t)n_cons, cudaMemcpyDeviceToDevice, s));
        NCK(cudaMemcpyAsync(ns->alm, flags0, sizeof(flags0), cudaMemcpyHostToDevice, s));
        if (rep->status == TLFE_OK && rep->c_norm > prm->alm_tol) rep->status = TLFE_E_NOT_CONVERGED;
    }
    NCK(cudaMemcpyAsync(v_out, ns->v, 8 * N3, cudaMemcpyDeviceToDevice, s));
    int64_t ninv = 0;
    st = tlfe_sync(m, stream, &ninv);
    if (st == TLFE_OK && ns->twin) st = tlfe_sync(ns->twin, stream, &ninv);
    if (st != TLFE_OK) return st;
    if (rep->status != TLFE_OK) return fail(TLFE_E_NOT_CONVERGED, "newton step did not reach the tolerance");
    return TLFE_OK;
}
