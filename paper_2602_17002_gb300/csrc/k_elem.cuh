// Element kernels of the TL-FEA hot path (internal force, operator product,
// adjoint, Jacobi diagonal, and the force and operator product of one state
// in one pass), templated on element type, quadrature size, arithmetic type
// and operation.
//
// Work decomposition: one thread per element, one warp per tile of 32
// elements, warps independent of each other (persistent, grid-striding over
// tiles). Per warp:
//   - the tile's metadata (unique-node list, local indices, node-to-slot
//     lists) comes by cp.async.bulk one tile ahead into a double buffer, with
//     the per-element J^{-1} and det J record on the affine path;
//   - slab path only: the reference data of one quadrature point of one tile
//     (h_i rows and w_q J_p, a contiguous "slice" of the slab
//     [tile][q][3 npe + 1][32]) is streamed by cp.async.bulk into a ring of
//     NSLICE shared-memory slots, issued NSLICE slices ahead by lane 0 and
//     completed on one mbarrier per slot; the affine path instead forms
//     h_i = J^{-T} g_i from the parent gradients g_i at each point;
//   - the nodes of the next tile are prefetched into L2, after the first
//     quadrature point in the affine force, operator and diagonal kernels,
//     after the last one on the slab path (the affine adjoint runs faster
//     without);
//   - the nodal values of the tile's unique nodes (a list built at mesh
//     creation) are gathered into a shared-memory patch, one record per list
//     entry, with consecutive lanes on consecutive entries; each lane then
//     reads its element's nodes from the patch through precomputed local
//     indices. The list orders the nodes so that the 8 lanes of a quarter
//     warp, which read the same element-local node of their elements in one
//     16-byte load, hit distinct bank groups;
//   - each lane evaluates F = I + sum_i u_i h_i^T per quadrature point and the
//     stress, its directional derivative, its adjoint or the diagonal moduli,
//     accumulating its element vector sum_q w_q J_p (.) h_iq in registers;
//   - element vectors go to conflict-free shared slots [i * 32 + lane]; one
//     lane per unique node sums that node's slots (a node-to-slot list built
//     at mesh creation) and adds the sum to the global array with one atomic
//     per component (a plain read-add-write in colour passes, where no two
//     elements of a launch share a node).
// Every mbarrier wait is bounded; on timeout the kernel latches ST_TIMEOUT in
// the status word, waits (again bounded) for the copies it still has in
// flight, each by the parity of its barrier's one outstanding phase, and
// returns.
// Affine Q27 blocks do not come here: they run the warp-per-element kernels
// of k_wpe.cuh (kernel_for / smem_for below dispatch on wpe_path).
#pragma once

#include <string>

#include "tlfe_elem.cuh"
#include "tlfe_internal.h"

namespace tlfe {

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier, bulk async copy, cp.async
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bulk copy global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <int BYTES> __device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

constexpr long long MBAR_SPIN_LIMIT = 1ll << 20;  // try_wait rounds before giving up

// ---------------------------------------------------------------------------
// per-op sizes
// ---------------------------------------------------------------------------

template <int OP> struct OpFields {
    static constexpr int IN = op_in_fields(OP);   // input values per node (u, udot [, v])
    static constexpr int OUT = op_nf(OP) - IN;    // output values per node
    static constexpr int NFI = IN / 3;            // input vector fields per node
    static constexpr int NFO = OUT / 3;           // output vector fields per node
};

// Patch record of one node.
//   FP32 (12 floats, 48 B), laid out for paired arithmetic (FFMA2 on the x
//   and y components of a 3-vector, the z component alone):
//     [h0 h1 l0 l1 | h2 l2 ud2 v2 | ud0 ud1 v0 v1]
//   FP64: [u(3) | udot(3) | v(3)]  (6 or 10 doubles)
// The displacement arrives in FP64; FP32 kernels keep it as an unevaluated
// pair (h, l) with u = h + l to about 2^-46 |u|, so that element-relative
// differences u_i - u_0 are formed without the rounding of |u| (large rigid
// motions). The FP64 displacement is first copied into the record's bytes
// 0..23 (the h, l slots and the unused h2, l2 of slot 2's first half) and
// split there in place.
template <int OP, typename R> struct Rec {
    static constexpr bool PK = sizeof(R) == 4;
    // FP32 slots (float offsets)
    static constexpr int H01 = 0, L01 = 2, H2 = 4, L2 = 5, UD2 = 6, V2 = 7, UD01 = 8, V01 = 10;
    // FP64 offsets
    static constexpr int OFF_UD = 3;                            // udot
    static constexpr int OFF_V = 6;                             // direction / cotangent
    static constexpr int REC = PK ? 12 : (3 * OpFields<OP>::NFI + 1) / 2 * 2;
};

// packed FP32 pairs (sm_100 and later: one instruction for two lanes of work)
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float4 lds4(const float *r) { return *reinterpret_cast<const float4 *>(r); }
// shared-memory loads the compiler may not hoist out of the point loop and
// keep in registers (volatile): the force and adjoint kernels re-read each
// element's local node indices at every point, and the adjoint also its
// J^{-1} and node 0's displacement pair, instead of holding them across the
// loop, which frees registers for the point's arithmetic
__device__ __forceinline__ float lds_f32_volatile(const float *p)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ float4 lds4_volatile(const float *p)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ int lds_u16_volatile(const uint16_t *p)
{
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(smem_u32(p)));
    return (int)v;
}

constexpr int NSLICE = 2;  // ring depth per warp (quadrature-point slices)

template <int ET, typename R> struct Slice {
    static constexpr int NPE = Elem<ET>::NPE;
    static constexpr int ROWS = NPE * 3 + 1;
    static constexpr uint32_t BYTES = ROWS * 32 * sizeof(R);  // multiple of 128
};

// per-element affine record of a tile: J^{-1} (row-major, 9 rows) and det J, [10][32]
template <typename R> struct AffRec {
    static constexpr int ROWS = AFF_ROWS;
    static constexpr uint32_t BYTES = ROWS * 32 * sizeof(R);  // multiple of 16
};

// shared memory of one warp: slice ring (isoparametric path only), two
// metadata buffers (each followed, on the affine path, by the tile's affine
// record), and a work area holding first the node patch [umax][REC] and later
// the element-vector slots [npe * 32][3] of one output field; rounded up to
// 128 bytes so that every bulk-copy destination stays 16-byte aligned
template <int ET, typename R, int OP, bool AFF>
__host__ __device__ constexpr size_t warp_region_bytes(int umax, int meta_bytes)
{
    const size_t patch = (size_t)umax * Rec<OP, R>::REC * sizeof(R);
    const size_t slots = (size_t)Elem<ET>::NPE * 32 * 3 * sizeof(R);  // one output field at a time
    const size_t ring = AFF ? 0 : (size_t)NSLICE * Slice<ET, R>::BYTES;
    const size_t mrec = (size_t)meta_bytes + (AFF ? AffRec<R>::BYTES : 0);
    return (ring + 2 * mrec + (patch > slots ? patch : slots) + 127) / 128 * 128;
}

// dynamic shared memory of one CTA with `wpb` warps (mbarriers, then the warp regions)
template <int ET, typename R, int OP, bool AFF>
__host__ __device__ constexpr size_t elem_smem_bytes(int umax, int meta_bytes, int wpb)
{
    return 128 + (size_t)wpb * warp_region_bytes<ET, R, OP, AFF>(umax, meta_bytes);
}

// 3-vectors at compile-time offsets of a 16-byte-aligned shared record, with
// the widest aligned vector accesses the offset allows
template <int OFF> __device__ __forceinline__ void ld3c(const float *r, float &x, float &y, float &z)
{
    if constexpr (OFF % 4 == 0) {
        const float4 v = *reinterpret_cast<const float4 *>(r + OFF);
        x = v.x, y = v.y, z = v.z;
    } else if constexpr (OFF % 4 == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(r + OFF);
        x = v.x, y = v.y, z = r[OFF + 2];
    } else {
        const float2 v = *reinterpret_cast<const float2 *>(r + OFF + 1);
        x = r[OFF], y = v.x, z = v.y;
    }
}
template <int OFF> __device__ __forceinline__ void ld3c(const double *r, double &x, double &y, double &z)
{
    if constexpr (OFF % 2 == 0) {
        const double2 v = *reinterpret_cast<const double2 *>(r + OFF);
        x = v.x, y = v.y, z = r[OFF + 2];
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(r + OFF + 1);
        x = r[OFF], y = v.x, z = v.y;
    }
}
template <int OFF> __device__ __forceinline__ void st3c(float *r, float x, float y, float z)
{
    if constexpr (OFF % 4 == 0) {
        *reinterpret_cast<float4 *>(r + OFF) = make_float4(x, y, z, 0.f);
    } else if constexpr (OFF % 4 == 2) {
        *reinterpret_cast<float2 *>(r + OFF) = make_float2(x, y);
        r[OFF + 2] = z;
    } else {
        r[OFF] = x;
        *reinterpret_cast<float2 *>(r + OFF + 1) = make_float2(y, z);
    }
}
template <int OFF> __device__ __forceinline__ void st3c(double *r, double x, double y, double z)
{
    if constexpr (OFF % 2 == 0) {
        *reinterpret_cast<double2 *>(r + OFF) = make_double2(x, y);
        r[OFF + 2] = z;
    } else {
        r[OFF] = x;
        *reinterpret_cast<double2 *>(r + OFF + 1) = make_double2(y, z);
    }
}
// FP64 displacement of a record (the FP32 kernels read their (h, l) pairs
// from the paired slots directly)
__device__ __forceinline__ void ld_u(const double *r, double h[3], double l[3])
{
    ld3c<0>(r, h[0], h[1], h[2]);
    l[0] = l[1] = l[2] = 0.0;
}

// x = hi + lo to about 2^-46 |x| with hi, lo in FP32, by integer and FP32
// operations only (the FP64 pipe of this GPU runs at a small fraction of the
// FP32 rate): hi keeps the leading 24 significant bits of x (exact in FP32),
// lo the next 23 bits scaled by 2^(e - 46). |x| < 2^-126 gives (+-0, +-0);
// |x| >= 2^128, inf and NaN fall back to the plain FP32 rounding with lo = 0.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu) - 1023;  // unbiased binary exponent
    if (e < -126) {
        hi = __uint_as_float(sign);
        lo = __uint_as_float(sign);
    } else if (e <= 127) {
        const unsigned mhi = ((hw & 0xFFFFFu) << 3) | (lw >> 29);  // significand bits 51..29
        hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | mhi);
        const unsigned r = (lw >> 6) & 0x7FFFFFu;                   // significand bits 28..6
        const float rf = __uint_as_float(0x4B000000u | r) - 8388608.0f;  // = r exactly
        const float sc = e >= -80 ? __uint_as_float((unsigned)(e + 81) << 23) : 0.0f;  // 2^(e - 46)
        lo = __uint_as_float(sign | __float_as_uint(rf * sc));
    } else {
        hi = (float)x;
        lo = 0.0f;
    }
}

// bounded wait on an mbarrier phase; returns false when the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    long long spins = 0;
    while (!mbar_try_wait(bar, parity))
        if (++spins > MBAR_SPIN_LIMIT) return false;
    return true;
}

// Resident CTAs (of 4 warps) per SM the register allocation aims at, by
// measurement on the beam workload: the FP32 affine force kernel fits 16
// warps per SM in 128 registers; the adjoint, with two element vectors live,
// fits 12 warps in 168 registers (its local indices, J^{-1} and node 0's
// pair re-read from shared memory at every point) without spill or with a
// few bytes for the laws listed below, and runs 7 % faster there than at 8
// warps and 214 registers; with the generic law or the undamped
// neo-Hookean one it would spill 70-200 bytes and keeps 8 warps. FP64 kernels take all 255 registers,
// and so do Q27 kernels (81-entry element vectors; their shared-memory
// footprint limits the resident warps anyway).
template <int ET, typename R, int OP, bool AFF, int MAT> constexpr int min_ctas()
{
    if (sizeof(R) != 4 || ET == ET_Q27) return 1;
    if (OP == OP_VJP || OP == OP_FM) {
        const bool fits = ET == ET_T4 || MAT == MAT_NH_KV || MAT == MAT_SVK || (MAT == MAT_SVK_KV && AFF) ||
                          (ET == ET_H8 && MAT != MAT_ANY);
        return fits ? 3 : 2;
    }
    return (OP == OP_FORCE && AFF) ? 4 : 3;
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The work of one warp on the tiles t0, t0 + tstep, ... (n_my of them) of
// the pass described by p: wbase is the warp's shared-memory region (laid out
// by warp_region_bytes) and bar its NSLICE + 2 mbarriers, freshly initialised
// by the caller (every phase count starts at 0). Returns false when a bounded
// wait ran out (the status word has the timeout, and every copy the warp had
// in flight has been waited for).
template <int ET, int NQ, typename R, int OP, bool AFF, int MAT>
__device__ __forceinline__ bool elem_tiles(const KParams<R> &p, unsigned char *wbase, uint64_t *bar, int t0,
                                           int tstep, int n_my)
{
    constexpr int NPE = Elem<ET>::NPE;
    using RC = Rec<OP, R>;
    constexpr int REC = RC::REC;
    constexpr int OFF_UD = RC::OFF_UD;
    constexpr int OFF_V = RC::OFF_V;
    constexpr bool PK = RC::PK;                        // FP32: paired (x, y) arithmetic
    constexpr bool PKA = PK && OP != OP_DIAG;          // ... and paired element-vector accumulators
    constexpr int NFO = OpFields<OP>::NFO;
    constexpr bool HAS_V = OpFields<OP>::NFI == 3;
    constexpr bool DD_REG = OP == OP_FORCE || OP == OP_DIAG;
    using SL = Slice<ET, R>;
    constexpr int ROWS = SL::ROWS;
    using PG = ParentGrad<ET, NQ, R>;
    constexpr uint32_t AB = AFF ? AffRec<R>::BYTES : 0;
    constexpr bool PF_EARLY = AFF && OP != OP_VJP;  // where the next tile's L2 prefetch goes (see prefetch_next)
    constexpr bool PF_NONE = AFF && OP == OP_VJP;
    constexpr bool LI_REREAD = OP == OP_FORCE || OP == OP_VJP || OP == OP_FM;
    // two element vectors per element: the adjoint's (g_u, g_udot) and the
    // fused force + operator product's (f, y)
    constexpr bool TWO = OP == OP_VJP || OP == OP_FM;
    // the adjoint (and the fused force + operator product, which holds as
    // many accumulators) also re-reads J^{-1} (affine record) and node 0's
    // pair at every point: 168 registers without spill (12 warps per SM)
    constexpr bool DIET = OP == OP_VJP || OP == OP_FM;

    const int lane = threadIdx.x & 31;
    const int MB = p.meta_bytes;
    uint64_t *mbar = bar + NSLICE;
    const size_t MRB = (size_t)MB + AB;                        // metadata (+ affine) record bytes
    unsigned char *ring = wbase;
    unsigned char *mbuf = wbase + (AFF ? 0 : NSLICE * SL::BYTES);  // [2][MB + AB]
    R *work = reinterpret_cast<R *>(mbuf + 2 * MRB);           // patch [umax][REC], later slots

    const bool mass_only = OP == OP_MATVEC && p.mass_only != 0;
    const int n_slices = (mass_only || AFF) ? 0 : n_my * NQ;
    const bool need_ud = p.visc != 0;

    auto issue = [&](int j) {  // slab slice j of this warp into ring slot j % NSLICE
        const int t = t0 + (j / NQ) * tstep;
        const int q = j % NQ;
        const int b = j % NSLICE;
        mbar_arrive_expect_tx(bar + b, SL::BYTES);
        bulk_g2s(ring + (size_t)b * SL::BYTES, p.slab + ((size_t)t * NQ + q) * ROWS * 32, SL::BYTES, bar + b);
    };
    auto issue_meta = [&](int k) {  // metadata (+ affine record) of the warp's k-th tile into buffer k & 1
        const int t = t0 + k * tstep;
        unsigned char *dst = mbuf + (size_t)(k & 1) * MRB;
        mbar_arrive_expect_tx(mbar + (k & 1), (uint32_t)MRB);
        bulk_g2s(dst, p.meta + (size_t)t * MB, (uint32_t)MB, mbar + (k & 1));
        if constexpr (AFF) bulk_g2s(dst + MB, p.aff + (size_t)t * AffRec<R>::ROWS * 32, AB, mbar + (k & 1));
    };
    if (lane == 0) {
        if (n_my > 0) issue_meta(0);
        for (int j = 0; j < NSLICE && j < n_slices; ++j) issue(j);
    }
    // copies issued and waited for, counted alike in every lane (the issue
    // decisions are warp-uniform): slices j < sl_issued and metadata records
    // k < mt_issued were requested, those below sl_done / mt_done have landed.
    // A barrier never holds more than one outstanding phase (slot b is
    // re-armed only after its previous slice was consumed; record k + 1 is
    // requested only after record k - 1, the previous user of its barrier,
    // was waited for), so the timeout drain below can wait on each
    // outstanding phase by its parity without ambiguity.
    int sl_issued = n_slices < NSLICE ? n_slices : NSLICE, sl_done = 0;
    int mt_issued = n_my > 0 ? 1 : 0, mt_done = 0;

    bool timed_out = false;
    for (int k = 0; k < n_my; ++k) {
        const int t = t0 + k * tstep;
        // ---- metadata of this tile (prefetched one tile ahead)
        if (!mbar_wait_bounded(mbar + (k & 1), (uint32_t)((k >> 1) & 1))) timed_out = true;
        if (__any_sync(0xffffffffu, timed_out)) {
            timed_out = true;
            break;
        }
        mt_done = k + 1;
        if (k + 1 < n_my) {
            if (lane == 0) issue_meta(k + 1);
            mt_issued = k + 2;
        }
        const unsigned char *M = mbuf + (size_t)(k & 1) * MRB;
        const int U = (int)bounds_clamp(*reinterpret_cast<const int32_t *>(M), (int64_t)p.umax + 1, p.status);
        const int e = reinterpret_cast<const int32_t *>(M + 16)[lane];
        const int32_t *nodes = reinterpret_cast<const int32_t *>(M + 16 + 128);
        const uint16_t *mlidx = reinterpret_cast<const uint16_t *>(M + 16 + 128 + 4 * p.umaxp);
        const uint16_t *spos = mlidx + NPE * 32;  // slot (i, lane) -> node-sorted position
        const uint16_t *soff = spos + NPE * 32;   // positions of unique node kk: [soff[kk], soff[kk + 1])

        // ---- gather the tile's nodal inputs into the patch, one record per
        // unique node: every lane issues asynchronous copies (cp.async) for all
        // of its nodes before waiting once, so that the load latencies of the
        // whole tile overlap without holding registers; FP32 kernels then
        // split the FP64 displacement in place into its (hi, lo) pair (both
        // take the same 24 bytes of the record)
        for (int kk = lane; kk < U; kk += 32) {
            const int64_t n = bounds_clamp(nodes[kk], p.n_nodes, p.status);
            R *rec = work + (size_t)kk * REC;
#pragma unroll
            for (int a = 0; a < 3; ++a) cp_async<8>(reinterpret_cast<double *>(rec) + a, p.u + 3 * n + a);
            if constexpr (PK) {
                if (need_ud) {
                    cp_async<4>(rec + RC::UD01, p.ud + 3 * n);
                    cp_async<4>(rec + RC::UD01 + 1, p.ud + 3 * n + 1);
                    cp_async<4>(rec + RC::UD2, p.ud + 3 * n + 2);
                }
                if (HAS_V) {
                    cp_async<4>(rec + RC::V01, p.v + 3 * n);
                    cp_async<4>(rec + RC::V01 + 1, p.v + 3 * n + 1);
                    cp_async<4>(rec + RC::V2, p.v + 3 * n + 2);
                }
            } else {
                if (need_ud)
#pragma unroll
                    for (int a = 0; a < 3; ++a) cp_async<sizeof(R)>(rec + OFF_UD + a, p.ud + 3 * n + a);
                if (HAS_V)
#pragma unroll
                    for (int a = 0; a < 3; ++a) cp_async<sizeof(R)>(rec + OFF_V + a, p.v + 3 * n + a);
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
        if constexpr (PK) {
            for (int kk = lane; kk < U; kk += 32) {
                R *rec = work + (size_t)kk * REC;
                const double2 u01 = *reinterpret_cast<const double2 *>(rec);
                const double u2 = reinterpret_cast<const double *>(rec)[2];
                float h[3], l[3];
                split_f64(u01.x, h[0], l[0]);
                split_f64(u01.y, h[1], l[1]);
                split_f64(u2, h[2], l[2]);
                *reinterpret_cast<float4 *>(rec) = make_float4(h[0], h[1], l[0], l[1]);
                *reinterpret_cast<float2 *>(rec + RC::H2) = make_float2(h[2], l[2]);
            }
        }
        int li[NPE];
#pragma unroll
        for (int i = 0; i < NPE; ++i) li[i] = (int)bounds_clamp(mlidx[i * 32 + lane], U, p.status);
        const bool valid = e >= 0;
        Mat<R> m = p.mat0;
        if (p.mats) m = p.mats[bounds_clamp(p.emat[(size_t)t * 32 + lane], p.n_mats, p.status)];
        if (p.elam) {
            m.mu = p.elam[((size_t)t * 2 + 0) * 32 + lane];
            m.lam = p.elam[((size_t)t * 2 + 1) * 32 + lane];
        }
        // material: the law and the presence of the viscous term are
        // compile-time constants when the block allows (MAT != MAT_ANY)
        if constexpr (MAT == MAT_NH || MAT == MAT_NH_KV) m.model = MODEL_NH;
        if constexpr (MAT == MAT_SVK || MAT == MAT_SVK_KV) m.model = MODEL_SVK;
        const bool visc = MAT == MAT_ANY ? (need_ud && (m.mu_v != R(0) || m.lam_v != R(0)))
                                         : (MAT == MAT_NH_KV || MAT == MAT_SVK_KV);
        // affine path: J^{-1} and det J of this lane's element (Sec. 6, affine case)
        R Ji[9], detJ = R(0);
        if constexpr (AFF) {
            const R *A = reinterpret_cast<const R *>(M + MB) + lane;
#pragma unroll
            for (int r = 0; r < 9; ++r) Ji[r] = A[r * 32];
            detJ = A[9 * 32];
        }
        __syncwarp();

        // element-relative displacements d_i = u_i - u_0 (sum_i h_i = 0, so
        // G = sum_i u_i h_i^T = sum_{i>0} d_i h_i^T, with rigid translation
        // removed exactly). Kept in registers by the force and diagonal
        // kernels; the operator and adjoint kernels, which hold more
        // accumulators, re-form them from the patch at every point.
        R h0v[3], l0v[3];
        R dd[NPE][3];
        // FP32: node 0's pair, negated, with x and y paired; d_i = (h_i - h_0)
        // + (l_i - l_0) as (h_i + (-h_0)) + (l_i + (-l_0)), the same roundings
        float2 nh01 = make_float2(0.f, 0.f), nl01 = make_float2(0.f, 0.f), dp[NPE];
        float nh2 = 0.f, nl2 = 0.f;
        if constexpr (PK) {
            const float4 A = lds4(work + li[0] * REC), B = lds4(work + li[0] * REC + 4);
            nh01 = make_float2(-A.x, -A.y);
            nl01 = make_float2(-A.z, -A.w);
            nh2 = -B.x;
            nl2 = -B.y;
        } else {
            ld_u(work + li[0] * REC, h0v, l0v);
        }
        if constexpr (DD_REG) {
#pragma unroll
            for (int i = 1; i < NPE; ++i) {
                if constexpr (PK) {
                    const float4 A = lds4(work + li[i] * REC), B = lds4(work + li[i] * REC + 4);
                    dp[i] = add2(add2(make_float2(A.x, A.y), nh01), add2(make_float2(A.z, A.w), nl01));
                    dd[i][2] = (B.x + nh2) + (B.y + nl2);
                } else {
                    R hv[3], lv[3];
                    ld_u(work + li[i] * REC, hv, lv);
#pragma unroll
                    for (int a = 0; a < 3; ++a) dd[i][a] = (hv[a] - h0v[a]) + (lv[a] - l0v[a]);
                }
            }
        }
        // element vectors: FP32 keeps (x, y) of each node as a pair and z alone
        R acc0[NPE][3], acc1[NPE][3];
        float2 ap0[NPE], ap1[NPE];
#pragma unroll
        for (int i = 0; i < NPE; ++i) {
            if constexpr (PKA) {
                ap0[i] = make_float2(0.f, 0.f);
                acc0[i][2] = R(0);
                if (TWO) {
                    ap1[i] = make_float2(0.f, 0.f);
                    acc1[i][2] = R(0);
                }
            } else {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    acc0[i][d] = R(0);
                    if (TWO) acc1[i][d] = R(0);
                }
            }
        }
        R gmu_acc = R(0), glam_acc = R(0);
        int bad = 0;

        // ---- the next tile's nodal inputs towards L2 (its metadata was
        // requested at the start of this tile); false when that metadata never
        // landed. Issued after this tile's first point on the affine path
        // (force, operator, diagonal), after the last on the slab path, and
        // not at all by the affine adjoint: measured on the beam, the early
        // prefetch cut the affine K v kernel by 18 % and the force by 12 %,
        // and slowed the slab path; the affine adjoint runs 4-5 % faster
        // without it than with it early or late, also with the L2 flushed
        // before the launch. (The tile-start wait on the metadata barrier
        // stands without it.)
        auto prefetch_next = [&]() -> bool {
            if (k + 1 >= n_my) return true;
            const bool ok = mbar_wait_bounded(mbar + ((k + 1) & 1), (uint32_t)(((k + 1) >> 1) & 1));
            if (__any_sync(0xffffffffu, !ok)) return false;
            const unsigned char *Mn = mbuf + (size_t)((k + 1) & 1) * MRB;
            const int Un = *reinterpret_cast<const int32_t *>(Mn);
            const int32_t *nodes_n = reinterpret_cast<const int32_t *>(Mn + 16 + 128);
            for (int kk = lane; kk < Un; kk += 32) {
                const int64_t n = nodes_n[kk];
                prefetch_l2(p.u + 3 * n);
                if (need_ud) prefetch_l2(p.ud + 3 * n);
                if (HAS_V) prefetch_l2(p.v + 3 * n);
            }
            return true;
        };

#pragma unroll 1
        for (int q = 0; q < (mass_only ? 0 : NQ); ++q) {
            // reference gradients of this point: the slab slice (isoparametric
            // path), or the parent gradients g_i with h_i = J^{-T} g_i (affine path)
            const R *sl = nullptr;
            PG pg;
            R w;
            if constexpr (AFF) {
                pg.at(q);
                w = quad_weight<ET, NQ, R>(q) * detJ;
            } else {
                const int j = k * NQ + q;
                const int b = j % NSLICE;
                if (!mbar_wait_bounded(bar + b, (uint32_t)((j / NSLICE) & 1))) timed_out = true;
                if (__any_sync(0xffffffffu, timed_out)) {
                    timed_out = true;
                    break;
                }
                sl_done = j + 1;
                sl = reinterpret_cast<const R *>(ring + (size_t)b * SL::BYTES) + lane;
                w = sl[NPE * 3 * 32];
            }
            // gradient entry k of node i; nz(i, k) = false where it vanishes identically
            auto grad = [&](int i, int k2) -> R { return AFF ? pg.g(i, k2) : sl[(i * 3 + k2) * 32]; };
            auto nz = [&](int i, int k2) -> bool { return !AFF || PG::nz(i, k2); };

            // kinematics: G = sum d_i h_i^T, Fd = sum udot_i h_i^T, D = sum v_i h_i^T
            // (affine path: the same sums against g_i, then times J^{-1})
            QP<R> s1;
            R D[9];
            if constexpr (PK) {
                // rows 0 and 1 of G', Fd', D' paired per column k, row 2 alone
                if constexpr (DIET && !DD_REG) {  // node 0's negated pair, read again for this point
                    const int l0 = (int)bounds_clamp(lds_u16_volatile(mlidx + lane), U, p.status);
                    const float4 A0 = lds4_volatile(work + l0 * REC), B0 = lds4_volatile(work + l0 * REC + 4);
                    nh01 = make_float2(-A0.x, -A0.y);
                    nl01 = make_float2(-A0.z, -A0.w);
                    nh2 = -B0.x;
                    nl2 = -B0.y;
                }
                float2 Gp[3], Fp[3], Dp[3];
                float Gs[3], Fs[3], Ds[3];
#pragma unroll
                for (int k2 = 0; k2 < 3; ++k2) {
                    Gp[k2] = Fp[k2] = Dp[k2] = make_float2(0.f, 0.f);
                    Gs[k2] = Fs[k2] = Ds[k2] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < NPE; ++i) {
                    R hk[3];
#pragma unroll
                    for (int k2 = 0; k2 < 3; ++k2) hk[k2] = nz(i, k2) ? grad(i, k2) : R(0);
                    const int lii = LI_REREAD ? (int)bounds_clamp(lds_u16_volatile(mlidx + i * 32 + lane), U, p.status)
                                              : li[i];
                    const float *rec = work + lii * REC;
                    float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
                    if ((i > 0 && !DD_REG) || visc || HAS_V) B = lds4(rec + 4);
                    if (i > 0) {
                        float2 d01;
                        float d2;
                        if constexpr (DD_REG) {
                            d01 = dp[i];
                            d2 = dd[i][2];
                        } else {
                            const float4 A = lds4(rec);
                            d01 = add2(add2(make_float2(A.x, A.y), nh01), add2(make_float2(A.z, A.w), nl01));
                            d2 = (B.x + nh2) + (B.y + nl2);
                        }
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            if (nz(i, k2)) {
                                Gp[k2] = fma2(d01, bc2(hk[k2]), Gp[k2]);
                                Gs[k2] = fmaf(d2, hk[k2], Gs[k2]);
                            }
                    }
                    if (visc || HAS_V) {
                        const float4 C4 = lds4(rec + 8);
                        if (visc)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2)
                                if (nz(i, k2)) {
                                    Fp[k2] = fma2(make_float2(C4.x, C4.y), bc2(hk[k2]), Fp[k2]);
                                    Fs[k2] = fmaf(B.z, hk[k2], Fs[k2]);
                                }
                        if (HAS_V)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2)
                                if (nz(i, k2)) {
                                    Dp[k2] = fma2(make_float2(C4.z, C4.w), bc2(hk[k2]), Dp[k2]);
                                    Ds[k2] = fmaf(B.w, hk[k2], Ds[k2]);
                                }
                    }
                }
                // affine path: X = X' J^{-1}, rows 0 and 1 paired
                auto finish = [&](const float2 Xp[3], const float Xs[3], float *X) {
#pragma unroll
                    for (int b2 = 0; b2 < 3; ++b2) {
                        if constexpr (AFF) {
                            const float *Ajl = reinterpret_cast<const float *>(M + MB) + lane;
                            const float j0 = DIET ? lds_f32_volatile(Ajl + b2 * 32) : Ji[b2];
                            const float j3 = DIET ? lds_f32_volatile(Ajl + (3 + b2) * 32) : Ji[3 + b2];
                            const float j6 = DIET ? lds_f32_volatile(Ajl + (6 + b2) * 32) : Ji[6 + b2];
                            float2 q2 = mul2(Xp[0], bc2(j0));
                            q2 = fma2(Xp[1], bc2(j3), q2);
                            q2 = fma2(Xp[2], bc2(j6), q2);
                            X[b2] = q2.x;
                            X[3 + b2] = q2.y;
                            X[6 + b2] = fmaf(Xs[2], j6, fmaf(Xs[1], j3, Xs[0] * j0));
                        } else {
                            X[b2] = Xp[b2].x;
                            X[3 + b2] = Xp[b2].y;
                            X[6 + b2] = Xs[b2];
                        }
                    }
                };
                finish(Gp, Gs, s1.G);
                if (visc) finish(Fp, Fs, s1.Fd);
                else
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) s1.Fd[k2] = 0.f;
                if (HAS_V) finish(Dp, Ds, D);
                else
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) D[k2] = 0.f;
            } else {
#pragma unroll
            for (int k2 = 0; k2 < 9; ++k2) {
                s1.G[k2] = R(0);
                s1.Fd[k2] = R(0);
                D[k2] = R(0);
            }
#pragma unroll
            for (int i = 0; i < NPE; ++i) {
                R hk[3];
#pragma unroll
                for (int k2 = 0; k2 < 3; ++k2) hk[k2] = nz(i, k2) ? grad(i, k2) : R(0);
                const R *rec = work + li[i] * REC;
                R x[3];
                if (i > 0) {
                    if constexpr (!DD_REG) {
                        R hv[3], lv[3];
                        ld_u(rec, hv, lv);
#pragma unroll
                        for (int a = 0; a < 3; ++a) dd[i][a] = (hv[a] - h0v[a]) + (lv[a] - l0v[a]);
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            if (nz(i, k2)) s1.G[a * 3 + k2] += dd[i][a] * hk[k2];
                }
                if (visc) {
                    ld3c<OFF_UD>(rec, x[0], x[1], x[2]);
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            if (nz(i, k2)) s1.Fd[a * 3 + k2] += x[a] * hk[k2];
                }
                if (HAS_V) {
                    ld3c<OFF_V>(rec, x[0], x[1], x[2]);
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            if (nz(i, k2)) D[a * 3 + k2] += x[a] * hk[k2];
                }
            }
            if constexpr (AFF) {
                R T[9];
                mm3(s1.G, Ji, T);
#pragma unroll
                for (int k2 = 0; k2 < 9; ++k2) s1.G[k2] = T[k2];
                if (visc) {
                    mm3(s1.Fd, Ji, T);
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) s1.Fd[k2] = T[k2];
                }
                if (HAS_V) {
                    mm3(D, Ji, T);
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) D[k2] = T[k2];
                }
            }
            }
            R P[9];
            stress<R>(m, s1, visc, P);
            bad += (valid && !s1.ok) ? 1 : 0;

            if (OP == OP_DIAG) {
                // diagonal of a_K K^e + a_C C: A_d[c][b] = dP_{d b} / dF_{d c}
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    R A[9];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        R E[9], dP[9];
#pragma unroll
                        for (int k2 = 0; k2 < 9; ++k2) E[k2] = (k2 == d * 3 + c) ? R(1) : R(0);
                        dstress<R>(m, s1, visc, E, p.aK, p.aC, true, dP);
#pragma unroll
                        for (int b2 = 0; b2 < 3; ++b2) A[c * 3 + b2] = w * dP[d * 3 + b2];
                    }
#pragma unroll
                    for (int i = 0; i < NPE; ++i) {
                        R hh[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            if constexpr (AFF) {  // h_i = J^{-T} g_i
                                hh[c] = R(0);
#pragma unroll
                                for (int k2 = 0; k2 < 3; ++k2)
                                    if (nz(i, k2)) hh[c] += grad(i, k2) * Ji[k2 * 3 + c];
                            } else {
                                hh[c] = grad(i, c);
                            }
                        }
                        const R h0 = hh[0], h1 = hh[1], h2 = hh[2];
                        acc0[i][d] += h0 * (A[0] * h0 + A[1] * h1 + A[2] * h2) +
                                      h1 * (A[3] * h0 + A[4] * h1 + A[5] * h2) +
                                      h2 * (A[6] * h0 + A[7] * h1 + A[8] * h2);
                    }
                }
            } else {
                R T0[9], T1[9];  // element-vector operators of this point (scaled by w below)
                if (OP == OP_FORCE) {
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) T0[k2] = P[k2];
                } else if (OP == OP_MATVEC) {
                    dstress<R>(m, s1, visc, D, p.aK, p.aC, p.sym_only != 0, T0);
                } else if (OP == OP_FM) {
                    // FP32 only: the force's and the operator product's
                    // element vectors are accumulated one after the other below
                } else {
                    R gmu, glam;
                    astress<R>(m, s1, visc, D, T0, T1, gmu, glam);
                    gmu_acc += w * gmu;
                    glam_acc += w * glam;
                }
                if constexpr (PKA) {
                    // w T h_i = w (T J^{-T}) g_i: rows 0 and 1 of the point's
                    // operator paired per column, then accumulated into the
                    // paired element vectors
                    auto pack = [&](const float *T, float2 Tp[3], float Ts[3]) {
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2) {
                            if constexpr (AFF) {
                                const float *Ajl = reinterpret_cast<const float *>(M + MB) + lane;
                                const float j0 = DIET ? lds_f32_volatile(Ajl + (k2 * 3) * 32) : Ji[k2 * 3];
                                const float j1 = DIET ? lds_f32_volatile(Ajl + (k2 * 3 + 1) * 32) : Ji[k2 * 3 + 1];
                                const float j2 = DIET ? lds_f32_volatile(Ajl + (k2 * 3 + 2) * 32) : Ji[k2 * 3 + 2];
                                float2 q2 = mul2(make_float2(T[0], T[3]), bc2(j0));
                                q2 = fma2(make_float2(T[1], T[4]), bc2(j1), q2);
                                q2 = fma2(make_float2(T[2], T[5]), bc2(j2), q2);
                                Tp[k2] = mul2(q2, bc2(w));
                                Ts[k2] = w * fmaf(T[8], j2, fmaf(T[7], j1, T[6] * j0));
                            } else {
                                Tp[k2] = mul2(make_float2(T[k2], T[3 + k2]), bc2(w));
                                Ts[k2] = w * T[6 + k2];
                            }
                        }
                    };
                    if constexpr (OP == OP_FM) {
                        // force first (P packed and accumulated, then dead),
                        // then the stress derivative along the direction, so
                        // that the two point operators are never live together
                        float2 Tp[3];
                        float Ts[3];
                        pack(P, Tp, Ts);
#pragma unroll
                        for (int i = 0; i < NPE; ++i)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2)
                                if (nz(i, k2)) {
                                    const float hk = grad(i, k2);
                                    ap0[i] = fma2(Tp[k2], bc2(hk), ap0[i]);
                                    acc0[i][2] = fmaf(Ts[k2], hk, acc0[i][2]);
                                }
                        dstress<R>(m, s1, visc, D, p.aK, p.aC, p.sym_only != 0, T1);
                        pack(T1, Tp, Ts);
#pragma unroll
                        for (int i = 0; i < NPE; ++i)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2)
                                if (nz(i, k2)) {
                                    const float hk = grad(i, k2);
                                    ap1[i] = fma2(Tp[k2], bc2(hk), ap1[i]);
                                    acc1[i][2] = fmaf(Ts[k2], hk, acc1[i][2]);
                                }
                    } else {
                    float2 Tp0[3], Tp1[3];
                    float Ts0[3], Ts1[3];
                    pack(T0, Tp0, Ts0);
                    if (TWO) pack(T1, Tp1, Ts1);
#pragma unroll
                    for (int i = 0; i < NPE; ++i) {
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            if (nz(i, k2)) {
                                const float hk = grad(i, k2);
                                ap0[i] = fma2(Tp0[k2], bc2(hk), ap0[i]);
                                acc0[i][2] = fmaf(Ts0[k2], hk, acc0[i][2]);
                                if (TWO) {
                                    ap1[i] = fma2(Tp1[k2], bc2(hk), ap1[i]);
                                    acc1[i][2] = fmaf(Ts1[k2], hk, acc1[i][2]);
                                }
                            }
                    }
                    }
                } else {
#pragma unroll
                for (int k2 = 0; k2 < 9; ++k2) {
                    T0[k2] *= w;
                    if (TWO) T1[k2] *= w;
                }
                if constexpr (AFF) {
                    // T h_i = (T J^{-T}) g_i
                    R T[9];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            T[a * 3 + k2] = T0[a * 3] * Ji[k2 * 3] + T0[a * 3 + 1] * Ji[k2 * 3 + 1] +
                                            T0[a * 3 + 2] * Ji[k2 * 3 + 2];
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) T0[k2] = T[k2];
                    if (TWO) {
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int k2 = 0; k2 < 3; ++k2)
                                T[a * 3 + k2] = T1[a * 3] * Ji[k2 * 3] + T1[a * 3 + 1] * Ji[k2 * 3 + 1] +
                                                T1[a * 3 + 2] * Ji[k2 * 3 + 2];
#pragma unroll
                        for (int k2 = 0; k2 < 9; ++k2) T1[k2] = T[k2];
                    }
                }
#pragma unroll
                for (int i = 0; i < NPE; ++i) {
                    R hk[3];
#pragma unroll
                    for (int k2 = 0; k2 < 3; ++k2) hk[k2] = nz(i, k2) ? grad(i, k2) : R(0);
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            if (nz(i, k2)) {
                                acc0[i][a] += T0[a * 3 + k2] * hk[k2];
                                if (TWO) acc1[i][a] += T1[a * 3 + k2] * hk[k2];
                            }
                }
                }
            }
            if (PF_EARLY && q == 0 && !prefetch_next()) {
                timed_out = true;
                break;
            }
            if constexpr (!AFF) {
                // slot b is no longer read: hand it to the slice NSLICE ahead
                const int j = k * NQ + q;
                __syncwarp();
                if (j + NSLICE < n_slices) {
                    if (lane == 0) {
                        fence_proxy_async();
                        issue(j + NSLICE);
                    }
                    sl_issued = j + NSLICE + 1;
                }
            }
        }
        if (timed_out) break;

        if (!PF_NONE && !(PF_EARLY && !mass_only) && !prefetch_next()) {
            timed_out = true;
            break;
        }

        // consistent mass of affine elements: m_ij = rho V Mhat_ij (Sec. 4.1),
        // into the operator product (the second element vector of OP_FM)
        if ((OP == OP_MATVEC || OP == OP_DIAG || OP == OP_FM) && p.aM != R(0)) {
            const R c = p.aM * m.rho * p.evol[(size_t)t * 32 + lane];
            if (OP == OP_MATVEC || OP == OP_FM) {
                float2 *apy = OP == OP_FM ? ap1 : ap0;
                R(*accy)[3] = OP == OP_FM ? acc1 : acc0;
#pragma unroll
                for (int jn = 0; jn < NPE; ++jn) {
                    const int lj = LI_REREAD ? (int)bounds_clamp(lds_u16_volatile(mlidx + jn * 32 + lane), U, p.status)
                                             : li[jn];
                    if constexpr (PKA) {
                        const float *rec = work + lj * REC;
                        const float2 v01 = *reinterpret_cast<const float2 *>(rec + RC::V01);
                        const float v2 = rec[RC::V2];
#pragma unroll
                        for (int i = 0; i < NPE; ++i) {
                            const float mh = c * float(mass_hat(ET, i, jn));
                            apy[i] = fma2(v01, bc2(mh), apy[i]);
                            accy[i][2] += mh * v2;
                        }
                    } else {
                        R x[3];
                        ld3c<OFF_V>(work + lj * REC, x[0], x[1], x[2]);
#pragma unroll
                        for (int i = 0; i < NPE; ++i) {
                            const R mh = c * R(mass_hat(ET, i, jn));
                            accy[i][0] += mh * x[0];
                            accy[i][1] += mh * x[1];
                            accy[i][2] += mh * x[2];
                        }
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < NPE; ++i) {
                    const R mh = c * R(mass_hat(ET, i, i));
                    acc0[i][0] += mh;
                    acc0[i][1] += mh;
                    acc0[i][2] += mh;
                }
            }
        }
        if (OP == OP_VJP && valid && p.gth && bounds_ok(e, p.n_elem_total, p.status)) {
            p.gth[(size_t)e * 2 + 0] = double(gmu_acc);
            p.gth[(size_t)e * 2 + 1] = double(glam_acc);
        }
        const int nbad = __reduce_add_sync(0xffffffffu, bad);
        if (lane == 0 && nbad) atomicAdd(p.status + ST_INVERTED, nbad);

        // ---- per output field: each lane writes its element vector into the
        // node-sorted position array (the patch is dead now), then one lane per
        // unique node sums that node's contiguous positions and adds the sum
        // to the global array. The sorted scatter stores the sum as the tile's
        // partial instead (word 1 of the record: the tile's first partial
        // position); it runs as its own copy of the loop, so that the adding
        // path compiles as it does without it.
        auto slots_in = [&](int fo) {
            __syncwarp();
            if (valid) {
#pragma unroll
                for (int i = 0; i < NPE; ++i) {
                    const int ps = (int)bounds_clamp(spos[i * 32 + lane], NPE * 32, p.status);
                    if constexpr (PKA) {
                        const float2 a01 = fo == 0 ? ap0[i] : ap1[i];
                        work[ps * 3] = a01.x;
                        work[ps * 3 + 1] = a01.y;
                        work[ps * 3 + 2] = fo == 0 ? acc0[i][2] : acc1[i][2];
                    } else {
#pragma unroll
                        for (int d = 0; d < 3; ++d) work[ps * 3 + d] = fo == 0 ? acc0[i][d] : acc1[i][d];
                    }
                }
            }
            __syncwarp();
        };
        auto node_sum = [&](int kk, R &a0, R &a1, R &a2) {
            const int s0 = (int)bounds_clamp(soff[kk], NPE * 32 + 1, p.status);
            const int s1e = (int)bounds_clamp(soff[kk + 1], NPE * 32 + 1, p.status);
            a0 = a1 = a2 = R(0);
            for (int sb = s0; sb < s1e; sb += 4) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (sb + j < s1e) {
                        a0 += work[(sb + j) * 3 + 0];
                        a1 += work[(sb + j) * 3 + 1];
                        a2 += work[(sb + j) * 3 + 2];
                    }
            }
        };
        if (p.part0) {
#pragma unroll
            for (int fo = 0; fo < NFO; ++fo) {
                slots_in(fo);
                const int64_t P0 = reinterpret_cast<const int32_t *>(M)[1];
                R *dst = (fo == 0 ? p.part0 : p.part1) + P0 * 3;
                for (int kk = lane; kk < U; kk += 32) {
                    if (!bounds_ok(P0 + kk, p.n_part, p.status)) continue;
                    R a0, a1, a2;
                    node_sum(kk, a0, a1, a2);
                    dst[kk * 3] = a0;
                    dst[kk * 3 + 1] = a1;
                    dst[kk * 3 + 2] = a2;
                }
            }
        } else {
#pragma unroll
            for (int fo = 0; fo < NFO; ++fo) {
                R *out = fo == 0 ? p.out0 : p.out1;
                slots_in(fo);
                for (int kk = lane; kk < U; kk += 32) {
                    const int64_t n = bounds_clamp(nodes[kk], p.n_nodes, p.status);
                    R a0, a1, a2;
                    node_sum(kk, a0, a1, a2);
                    if (p.rmw_scatter) {
                        out[3 * n] += a0;
                        out[3 * n + 1] += a1;
                        out[3 * n + 2] += a2;
                    } else {
                        atomicAdd(out + 3 * n, a0);
                        atomicAdd(out + 3 * n + 1, a1);
                        atomicAdd(out + 3 * n + 2, a2);
                    }
                }
            }
        }
        __syncwarp();
    }
    if (timed_out) {
        // a copy never landed: record it, then wait (bounded) for every copy
        // this warp still has in flight, by the parity of the one phase its
        // barrier has outstanding, so that no bulk copy is still writing into
        // shared memory when the CTA exits
        if (lane == 0) atomicAdd(p.status + ST_TIMEOUT, 1);
        for (int j = sl_done; j < sl_issued; ++j) mbar_wait_bounded(bar + j % NSLICE, (uint32_t)((j / NSLICE) & 1));
        for (int k = mt_done; k < mt_issued; ++k) mbar_wait_bounded(mbar + (k & 1), (uint32_t)((k >> 1) & 1));
        return false;
    }
    return true;
}

// One element kernel per (type, quadrature, precision, op, path, material
// mode): one launch per pass, warps persistent over the pass's tiles.
template <int ET, int NQ, typename R, int OP, bool AFF, int MAT>
__global__ void __launch_bounds__(128, min_ctas<ET, R, OP, AFF, MAT>()) k_elem(const KParams<R> p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem) + wib * (NSLICE + 2);  // [wpb][NSLICE + 2] (<= 128 B)
    unsigned char *wbase = smem + 128 + (size_t)wib * warp_region_bytes<ET, R, OP, AFF>(p.umax, p.meta_bytes);

    const int gw = blockIdx.x * wpb + wib;
    const int W = gridDim.x * wpb;
    // tiles of this warp: interleaved (t0 + k W) or, with tile_chunk, one
    // contiguous run of neighbouring tiles (which share nodes through L2)
    const int n_tiles = p.tile_end - p.tile_begin;
    const int per = (n_tiles + W - 1) / W;
    const int t0 = p.tile_chunk ? p.tile_begin + gw * per : p.tile_begin + gw;
    const int tstep = p.tile_chunk ? 1 : W;
    const int n_my = p.tile_chunk ? max(0, min(per, n_tiles - gw * per))
                                  : (t0 < p.tile_end ? (p.tile_end - t0 + W - 1) / W : 0);
    if (lane == 0) {
        for (int b = 0; b < NSLICE + 2; ++b) mbar_init(bar + b, 1);
        fence_mbar_init();
    }
    __syncwarp();
    elem_tiles<ET, NQ, R, OP, AFF, MAT>(p, wbase, bar, t0, tstep, n_my);
}

}  // namespace tlfe

#include "k_wpe.cuh"

namespace tlfe {

template <int OP, typename R, bool AFF, int MAT> static void (*kernel_for_(int et, int nq))(const KParams<R>)
{
    if constexpr (OP == OP_FM) {  // the fused force + operator product: FP32 T4, T10 and H8 blocks
        if (sizeof(R) != 4 || et == ET_Q27) return nullptr;
    }
    if (et == ET_T4 && nq == 1) return k_elem<ET_T4, 1, R, OP, AFF, MAT>;
    if (et == ET_T10 && nq == 4) return k_elem<ET_T10, 4, R, OP, AFF, MAT>;
    if (et == ET_T10 && nq == 5) return k_elem<ET_T10, 5, R, OP, AFF, MAT>;
    if (et == ET_H8 && nq == 8) return k_elem<ET_H8, 8, R, OP, AFF, MAT>;
    if constexpr (OP != OP_FM)
        if (et == ET_Q27 && nq == 27) return k_elem<ET_Q27, 27, R, OP, AFF, MAT>;
    return nullptr;
}
// FP32 kernels are specialised on the material mode; FP64 kernels (the plain
// reference path, FP64-pipe bound) use the generic mode only
template <int OP, typename R, bool AFF> static void (*kernel_for_m(int et, int nq, int mat))(const KParams<R>)
{
    if constexpr (sizeof(R) == 4) {
        switch (mat) {
        case MAT_NH: return kernel_for_<OP, R, AFF, MAT_NH>(et, nq);
        case MAT_NH_KV: return kernel_for_<OP, R, AFF, MAT_NH_KV>(et, nq);
        case MAT_SVK: return kernel_for_<OP, R, AFF, MAT_SVK>(et, nq);
        case MAT_SVK_KV: return kernel_for_<OP, R, AFF, MAT_SVK_KV>(et, nq);
        default: break;
        }
    }
    return kernel_for_<OP, R, AFF, MAT_ANY>(et, nq);
}
template <int OP, typename R> static void (*kernel_for(int et, int nq, bool aff, int mat))(const KParams<R>)
{
    if constexpr (OP == OP_FM) {
        if (wpe_path(et, aff)) return nullptr;
    } else {
        if (wpe_path(et, aff)) return wpe_kernel_for<OP, R>(mat);
    }
    return aff ? kernel_for_m<OP, R, true>(et, nq, mat) : kernel_for_m<OP, R, false>(et, nq, mat);
}

template <int OP, typename R, bool AFF> size_t smem_for_(int et, int umax, int meta_bytes, int wpb)
{
    if (et == ET_T4) return elem_smem_bytes<ET_T4, R, OP, AFF>(umax, meta_bytes, wpb);
    if (et == ET_T10) return elem_smem_bytes<ET_T10, R, OP, AFF>(umax, meta_bytes, wpb);
    if (et == ET_H8) return elem_smem_bytes<ET_H8, R, OP, AFF>(umax, meta_bytes, wpb);
    if (et == ET_Q27 && OP != OP_FM) return elem_smem_bytes<ET_Q27, R, OP, AFF>(umax, meta_bytes, wpb);
    return 0;
}
template <int OP, typename R> size_t smem_for(int et, int umax, int meta_bytes, int wpb, bool aff)
{
    if (wpe_path(et, aff)) return OP == OP_FM ? 0 : wpe_smem_bytes<R>(wpb);
    return aff ? smem_for_<OP, R, true>(et, umax, meta_bytes, wpb) : smem_for_<OP, R, false>(et, umax, meta_bytes, wpb);
}

// resident warps per SM for the best CTA size among 4, 2 and 1 warps, or for
// the CTA size *wpb_io when it is positive on entry
template <int OP, typename R>
int occupancy_op(int et, int nq, bool aff, int mat, int umax, int meta_bytes, int *wpb_io, std::string *why)
{
    void (*kern)(const KParams<R>) = kernel_for<OP, R>(et, nq, aff, mat);
    const int only = *wpb_io;
    *wpb_io = 0;
    if (!kern) {
        *why = "no kernel for this element type and quadrature size";
        return 0;
    }
    int best = 0;
    for (int wpb : {4, 2, 1}) {
        if (only > 0 && wpb != only) continue;
        const size_t smem = smem_for<OP, R>(et, umax, meta_bytes, wpb, aff);
        if (smem > 227 * 1024) continue;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * wpb, smem);
        if (e != cudaSuccess) {
            *why = std::string("occupancy query failed: ") + cudaGetErrorString(e);
            return 0;
        }
        if (nb * wpb > best) {
            best = nb * wpb;
            *wpb_io = wpb;
        }
    }
    if (best == 0)
        *why = "shared memory per warp too large (patch of " + std::to_string(umax) + " nodes, metadata " +
               std::to_string(meta_bytes) + " B)";
    return best;
}

// launch on the affine path when p.aff is set, else on the isoparametric
// (slab) path; material mode p.mat_mode
template <int OP, typename R>
cudaError_t launch_op(int et, int nq, const KParams<R> &p, int grid, int wpb, cudaStream_t s)
{
    const bool aff = p.aff != nullptr;
    void (*kern)(const KParams<R>) = kernel_for<OP, R>(et, nq, aff, p.mat_mode);
    if (!kern) return cudaErrorInvalidValue;
    const size_t smem = smem_for<OP, R>(et, p.umax, p.meta_bytes, wpb, aff);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<grid, 32 * wpb, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace tlfe
