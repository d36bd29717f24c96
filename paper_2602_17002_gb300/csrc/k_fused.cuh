// One persistent launch per operation over every pass of a multi-block,
// multi-law mesh (FP32, affine tile path): the batch of uneven bodies of
// mixed element types and laws runs as one kernel instead of one launch per
// (block, law).
//
// Work items are contiguous tile runs of one pass, listed longest first (the
// heaviest element type and quadrature first, so that the light items fill
// the tail). Each warp takes the next item from an atomic counter, sets up
// fresh mbarrier phases, and runs the same per-warp tile loop (elem_tiles)
// as the per-pass kernels, with the pass's parameters read from the launch's
// own parameter table (kernel parameter space, indexed by the item's pass).
// The shared-memory region of a warp is the largest any covered pass needs.
#pragma once

#include "k_elem.cuh"
#include "tlfe_fused.h"

namespace tlfe {

// resident CTAs of 4 warps the register allocation aims at, as for the
// per-pass affine FP32 kernels of the same op (k_elem min_ctas)
template <int OP> constexpr int fused_min_ctas() { return OP == OP_FORCE ? 4 : (OP == OP_VJP ? 2 : 3); }

// one (element type, quadrature, material mode) body per function: kept out
// of line, so that each is compiled and register-allocated on its own (inlined
// into one switch, the bodies spilled heavily and compiled several times
// slower)
template <typename R, int OP, int CODE, int MAT>
__device__ __noinline__ bool fused_run(const KParams<R> *__restrict__ pp, unsigned char *wbase, uint64_t *bar, int t0,
                                       int n)
{
    // the parameters are read through a pointer no store of the body aliases
    const KParams<R> &p = *pp;
    if constexpr (CODE == FK_T4Q1) return elem_tiles<ET_T4, 1, R, OP, true, MAT>(p, wbase, bar, t0, 1, n);
    if constexpr (CODE == FK_T10Q4) return elem_tiles<ET_T10, 4, R, OP, true, MAT>(p, wbase, bar, t0, 1, n);
    if constexpr (CODE == FK_T10Q5) return elem_tiles<ET_T10, 5, R, OP, true, MAT>(p, wbase, bar, t0, 1, n);
    if constexpr (CODE == FK_H8Q8) return elem_tiles<ET_H8, 8, R, OP, true, MAT>(p, wbase, bar, t0, 1, n);
    return true;
}

template <typename R, int OP, int CODE>
__device__ __forceinline__ bool fused_mat(int mat, const KParams<R> *p, unsigned char *wbase, uint64_t *bar, int t0,
                                          int n)
{
    switch (mat) {
    case MAT_NH: return fused_run<R, OP, CODE, MAT_NH>(p, wbase, bar, t0, n);
    case MAT_NH_KV: return fused_run<R, OP, CODE, MAT_NH_KV>(p, wbase, bar, t0, n);
    case MAT_SVK: return fused_run<R, OP, CODE, MAT_SVK>(p, wbase, bar, t0, n);
    case MAT_SVK_KV: return fused_run<R, OP, CODE, MAT_SVK_KV>(p, wbase, bar, t0, n);
    default: return fused_run<R, OP, CODE, MAT_ANY>(p, wbase, bar, t0, n);
    }
}

// bytes of the per-warp copy of the current pass's parameters, ahead of the
// warp's region: the out-of-line bodies read the parameters through a
// pointer, which into shared memory is a short-latency load
template <typename R> __host__ __device__ constexpr size_t fused_param_bytes()
{
    return (sizeof(KParams<R>) + 127) / 128 * 128;
}

template <typename R, int OP>
__global__ void __launch_bounds__(128, fused_min_ctas<OP>()) k_fused(const __grid_constant__ FusedArgs<R> a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr size_t PB = fused_param_bytes<R>();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + wib * (NSLICE + 2);
    unsigned char *pbase = smem + 128 + (size_t)wib * (a.wreg + PB);
    unsigned char *wbase = pbase + PB;
    KParams<R> *ps = reinterpret_cast<KParams<R> *>(pbase);
    bool first = true;
    int cur = -1;  // pass whose parameters the copy holds
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(a.counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.n_items) break;
        const int4 w = a.items[it];
        // fresh phases for this item: every copy of the previous item has been
        // waited for, so its barriers hold no pending arrival
        if (lane == 0) {
            for (int b = 0; b < NSLICE + 2; ++b) {
                if (!first) mbar_inval(bar + b);
                mbar_init(bar + b, 1);
            }
            fence_mbar_init();
        }
        first = false;
        __syncwarp();
        if (w.x != cur) {  // warp-uniform
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&a.pass[w.x]);
            uint32_t *dst = reinterpret_cast<uint32_t *>(ps);
            for (int k = lane; k < (int)(sizeof(KParams<R>) / 4); k += 32) dst[k] = src[k];
            cur = w.x;
            __syncwarp();
        }
        const KParams<R> *p = ps;
        const int kind = a.kind[w.x];
        const int mat = kind % MAT_N;
        const int n = w.z - w.y;
        bool ok = true;
        switch (kind / MAT_N) {
        case FK_T4Q1: ok = fused_mat<R, OP, FK_T4Q1>(mat, p, wbase, bar, w.y, n); break;
        case FK_T10Q4: ok = fused_mat<R, OP, FK_T10Q4>(mat, p, wbase, bar, w.y, n); break;
        case FK_T10Q5: ok = fused_mat<R, OP, FK_T10Q5>(mat, p, wbase, bar, w.y, n); break;
        case FK_H8Q8: ok = fused_mat<R, OP, FK_H8Q8>(mat, p, wbase, bar, w.y, n); break;
        default: break;
        }
        if (!ok) break;  // a bounded wait ran out: recorded; this warp stops
        __syncwarp();
    }
}

// shared-memory region of one warp for a pass of code `code` (affine path)
template <typename R, int OP> size_t fused_warp_region(int code, int umax, int meta_bytes)
{
    switch (code) {
    case FK_T4Q1: return warp_region_bytes<ET_T4, R, OP, true>(umax, meta_bytes);
    case FK_T10Q4:
    case FK_T10Q5: return warp_region_bytes<ET_T10, R, OP, true>(umax, meta_bytes);
    case FK_H8Q8: return warp_region_bytes<ET_H8, R, OP, true>(umax, meta_bytes);
    default: return 0;
    }
}

// resident warps per SM of the fused kernel at warp regions of `wreg` bytes,
// best CTA size among 4, 2, 1 warps (or only *wpb_io when positive on entry)
template <int OP, typename R> int occupancy_fused(size_t wreg, int *wpb_io)
{
    const int only = *wpb_io;
    *wpb_io = 0;
    int best = 0;
    for (int wpb : {4, 2, 1}) {
        if (only > 0 && wpb != only) continue;
        const size_t smem = 128 + (size_t)wpb * (wreg + fused_param_bytes<R>());
        if (smem > 227 * 1024) continue;
        int nb = 0;
        cudaError_t e = cudaFuncSetAttribute(k_fused<R, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused<R, OP>, 32 * wpb, smem);
        if (e != cudaSuccess) return 0;
        if (nb * wpb > best) {
            best = nb * wpb;
            *wpb_io = wpb;
        }
    }
    return best;
}

template <int OP, typename R>
cudaError_t launch_fused(const FusedArgs<R> &a, int grid, int wpb, cudaStream_t s)
{
    const size_t smem = 128 + (size_t)wpb * (a.wreg + fused_param_bytes<R>());
    cudaError_t e = cudaFuncSetAttribute(k_fused<R, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fused<R, OP><<<grid, 32 * wpb, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tlfe
