// Element kernels of the TL-FEA hot path (force, operator product, adjoint,
// Jacobi diagonal), templated on element type, quadrature size, arithmetic
// type and operation.
//
// Work decomposition: one warp owns a tile of 32 elements (one element per
// lane) at a time, grid-striding over tiles. Per tile:
//   1. the warp gathers the nodal values of the tile's unique nodes (a sorted
//      list built at mesh creation) into a shared-memory patch: consecutive
//      lanes read consecutive node ids, so the gather is close to coalesced;
//   2. each lane reads its element's node values from the patch through the
//      precomputed local indices, streams its H and wJ slices (AoSoA layout,
//      one 128-byte line per warp load, evict-first), and evaluates
//      F = I + sum u_i h_i^T, the stress (or its directional derivative /
//      adjoint) and the element vector sum_q wJ_q (.) h_i per quadrature point
//      in registers;
//   3. element vectors are summed into the patch with shared-memory atomics
//      and the patch is added to the global array with one atomic per unique
//      node and component (or a plain read-add-write in colour passes, where no
//      two elements of a launch share a node).
#pragma once

#include "tlfe_elem.cuh"
#include "tlfe_internal.h"

namespace tlfe {

template <typename R> __device__ __forceinline__ R ld_stream(const R *p) { return __ldcs(p); }

template <typename R> __device__ __forceinline__ void atomic_add_global(R *p, R v) { atomicAdd(p, v); }

template <int OP> struct OpFields {
    static constexpr int IN = op_in_fields(OP);
    static constexpr int NF = op_nf(OP);
};

template <int ET, int NQ, typename R, int OP>
__global__ void __launch_bounds__(128) k_elem(const KParams<R> p)
{
    constexpr int NPE = Elem<ET>::NPE;
    constexpr int NF = OpFields<OP>::NF;
    constexpr int IN = OpFields<OP>::IN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int umax = p.umax;
    R *sw = reinterpret_cast<R *>(smem_raw) + (size_t)wib * umax * NF;
    R *sU = sw;
    R *sUd = sw + 3 * umax;
    R *sV = sw + 6 * umax;
    R *sO0 = sw + IN * umax;
    R *sO1 = sO0 + 3 * umax;
    const bool need_ud = p.visc != 0;

    for (int t = p.tile_begin + blockIdx.x * wpb + wib; t < p.tile_end; t += gridDim.x * wpb) {
        const int nb = p.tnode_off[t];
        const int U = p.tnode_off[t + 1] - nb;
        // ---- 1. gather the tile's nodal values into the patch
        for (int k = lane; k < U; k += 32) {
            const int64_t n = p.tnodes[nb + k];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                sU[3 * k + d] = __ldg(p.u + 3 * n + d);
                if (need_ud) sUd[3 * k + d] = __ldg(p.ud + 3 * n + d);
                if (OP == OP_MATVEC || OP == OP_VJP) sV[3 * k + d] = __ldg(p.v + 3 * n + d);
                sO0[3 * k + d] = R(0);
                if (OP == OP_VJP) sO1[3 * k + d] = R(0);
            }
        }
        __syncwarp();

        // ---- 2. element computation, one element per lane
        const int e = p.eid[t * 32 + lane];
        const bool valid = e >= 0;
        int li[NPE];
#pragma unroll
        for (int i = 0; i < NPE; ++i) li[i] = p.lidx[((size_t)t * NPE + i) * 32 + lane];
        Mat<R> m = p.mat0;
        if (p.mats) m = p.mats[p.emat[t * 32 + lane]];
        if (p.elam) {
            m.mu = p.elam[(size_t)(t * 2 + 0) * 32 + lane];
            m.lam = p.elam[(size_t)(t * 2 + 1) * 32 + lane];
        }
        const bool visc = need_ud && (m.mu_v != R(0) || m.lam_v != R(0));

        R ue[NPE][3], ve[NPE][3], acc0[NPE][3], acc1[NPE][3];
#pragma unroll
        for (int i = 0; i < NPE; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ue[i][d] = sU[3 * li[i] + d];
                if (OP == OP_MATVEC || OP == OP_VJP) ve[i][d] = sV[3 * li[i] + d];
                acc0[i][d] = R(0);
                if (OP == OP_VJP) acc1[i][d] = R(0);
            }
        R gmu_acc = R(0), glam_acc = R(0), vol = R(0);
        int bad = 0;

#pragma unroll 1
        for (int q = 0; q < NQ; ++q) {
            R h[NPE][3];
            const R *Hq = p.H + ((size_t)t * NQ + q) * NPE * 3 * 32 + lane;
#pragma unroll
            for (int i = 0; i < NPE; ++i)
#pragma unroll
                for (int d = 0; d < 3; ++d) h[i][d] = ld_stream(Hq + (i * 3 + d) * 32);
            const R w = ld_stream(p.wJ + ((size_t)t * NQ + q) * 32 + lane);
            vol += w;

            QP<R> s;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    R g = R(0);
#pragma unroll
                    for (int i = 0; i < NPE; ++i) g += ue[i][a] * h[i][c];
                    s.G[a * 3 + c] = g;
                }
            if (visc) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        R g = R(0);
#pragma unroll
                        for (int i = 0; i < NPE; ++i) g += sUd[3 * li[i] + a] * h[i][c];
                        s.Fd[a * 3 + c] = g;
                    }
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k) s.Fd[k] = R(0);
            }
            R P[9];
            stress<R>(m, s, visc, P);
            bad += s.ok ? 0 : 1;

            if (OP == OP_FORCE) {
#pragma unroll
                for (int k = 0; k < 9; ++k) P[k] *= w;
#pragma unroll
                for (int i = 0; i < NPE; ++i)
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        acc0[i][a] += P[a * 3] * h[i][0] + P[a * 3 + 1] * h[i][1] + P[a * 3 + 2] * h[i][2];
            } else if (OP == OP_MATVEC || OP == OP_VJP) {
                R D[9];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        R g = R(0);
#pragma unroll
                        for (int i = 0; i < NPE; ++i) g += ve[i][a] * h[i][c];
                        D[a * 3 + c] = g;
                    }
                if (OP == OP_MATVEC) {
                    R dP[9];
                    dstress<R>(m, s, visc, D, p.aK, p.aC, p.sym_only != 0, dP);
#pragma unroll
                    for (int k = 0; k < 9; ++k) dP[k] *= w;
#pragma unroll
                    for (int i = 0; i < NPE; ++i)
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            acc0[i][a] += dP[a * 3] * h[i][0] + dP[a * 3 + 1] * h[i][1] + dP[a * 3 + 2] * h[i][2];
                } else {
                    R gF[9], gFd[9], gmu, glam;
                    astress<R>(m, s, visc, D, gF, gFd, gmu, glam);
                    gmu_acc += w * gmu;
                    glam_acc += w * glam;
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        gF[k] *= w;
                        gFd[k] *= w;
                    }
#pragma unroll
                    for (int i = 0; i < NPE; ++i)
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            acc0[i][a] += gF[a * 3] * h[i][0] + gF[a * 3 + 1] * h[i][1] + gF[a * 3 + 2] * h[i][2];
                            acc1[i][a] += gFd[a * 3] * h[i][0] + gFd[a * 3 + 1] * h[i][1] + gFd[a * 3 + 2] * h[i][2];
                        }
                }
            } else {  // OP_DIAG: diagonal of the symmetric operator a_K K^e + a_C C
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    R A[3][3];  // A[c][b] = dP_{d b} / dF_{d c}
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        R E[9], dP[9];
#pragma unroll
                        for (int k = 0; k < 9; ++k) E[k] = (k == d * 3 + c) ? R(1) : R(0);
                        dstress<R>(m, s, visc, E, p.aK, p.aC, true, dP);
#pragma unroll
                        for (int b = 0; b < 3; ++b) A[c][b] = dP[d * 3 + b];
                    }
#pragma unroll
                    for (int i = 0; i < NPE; ++i) {
                        R t2 = R(0);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            t2 += h[i][c] * (A[c][0] * h[i][0] + A[c][1] * h[i][1] + A[c][2] * h[i][2]);
                        acc0[i][d] += w * t2;
                    }
                }
            }
        }

        // consistent mass of affine elements: m_ij = rho V Mhat_ij (Sec. 4.1)
        if ((OP == OP_MATVEC || OP == OP_DIAG) && p.aM != R(0)) {
            const R c = p.aM * m.rho * p.evol[t * 32 + lane];
#pragma unroll
            for (int i = 0; i < NPE; ++i) {
                if (OP == OP_MATVEC) {
                    R sx = R(0), sy = R(0), sz = R(0);
#pragma unroll
                    for (int j = 0; j < NPE; ++j) {
                        const R mh = R(mass_hat(ET, i, j));
                        sx += mh * ve[j][0];
                        sy += mh * ve[j][1];
                        sz += mh * ve[j][2];
                    }
                    acc0[i][0] += c * sx;
                    acc0[i][1] += c * sy;
                    acc0[i][2] += c * sz;
                } else {
                    const R mh = R(mass_hat(ET, i, i));
                    acc0[i][0] += c * mh;
                    acc0[i][1] += c * mh;
                    acc0[i][2] += c * mh;
                }
            }
        }
        (void)vol;

        if (valid) {
#pragma unroll
            for (int i = 0; i < NPE; ++i)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    atomicAdd(sO0 + 3 * li[i] + d, acc0[i][d]);
                    if (OP == OP_VJP) atomicAdd(sO1 + 3 * li[i] + d, acc1[i][d]);
                }
            if (OP == OP_VJP && p.gth) {
                p.gth[(size_t)e * 2 + 0] = double(gmu_acc);
                p.gth[(size_t)e * 2 + 1] = double(glam_acc);
            }
        }
        if (!valid) bad = 0;
        const int nbad = __reduce_add_sync(0xffffffffu, bad);
        if (lane == 0 && nbad) atomicAdd(p.status + ST_INVERTED, nbad);
        __syncwarp();

        // ---- 3. add the patch into the global arrays
        for (int k = lane; k < U; k += 32) {
            const int64_t n = p.tnodes[nb + k];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (p.rmw_scatter) {
                    p.out0[3 * n + d] += sO0[3 * k + d];
                    if (OP == OP_VJP && p.out1) p.out1[3 * n + d] += sO1[3 * k + d];
                } else {
                    atomic_add_global(p.out0 + 3 * n + d, sO0[3 * k + d]);
                    if (OP == OP_VJP && p.out1) atomic_add_global(p.out1 + 3 * n + d, sO1[3 * k + d]);
                }
            }
        }
        __syncwarp();
    }
}

template <int OP, typename R> static void (*kernel_for(int et, int nq))(const KParams<R>)
{
    if (et == ET_T4 && nq == 1) return k_elem<ET_T4, 1, R, OP>;
    if (et == ET_T10 && nq == 4) return k_elem<ET_T10, 4, R, OP>;
    if (et == ET_T10 && nq == 5) return k_elem<ET_T10, 5, R, OP>;
    if (et == ET_H8 && nq == 8) return k_elem<ET_H8, 8, R, OP>;
    return nullptr;
}

template <int OP, typename R> size_t smem_bytes(const KParams<R> &p)
{
    return (size_t)4 * p.umax * OpFields<OP>::NF * sizeof(R);
}

template <int OP, typename R> int occupancy_op(int et, int nq, size_t smem)
{
    void (*kern)(const KParams<R>) = kernel_for<OP, R>(et, nq);
    if (!kern) return 0;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 128, smem) != cudaSuccess) return 0;
    return nb;
}

template <int OP, typename R>
cudaError_t launch_op(int et, int nq, const KParams<R> &p, int grid, cudaStream_t s)
{
    void (*kern)(const KParams<R>) = kernel_for<OP, R>(et, nq);
    if (!kern) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes<OP, R>(p);
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    kern<<<grid, 128, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace tlfe
