// Warp-per-element kernels for affine Q27 bricks (internal force, operator
// product, adjoint, Jacobi diagonal).
//
// A Q27 element vector holds 81 values: one thread per element cannot keep it
// (and the 78 nodal differences) in registers. Here one warp takes one element
// at a time, in two phases separated by __syncwarp:
//   A. lane q < 27 owns Gauss point q: it forms G = sum_n d_n g_n(q)^T (and
//      the rate and direction gradients) against the parent gradients g_n(q)
//      of a per-CTA shared table, applies J^{-1}, evaluates the stress (or its
//      derivative, adjoint, or the diagonal moduli) and writes the point's
//      weighted operator, already multiplied by J^{-T}, to a shared row;
//   B. lane n < 27 owns node n: it sums T_q g_n(q) over the 27 rows and adds
//      the result to the global array (one atomic per component, or a plain
//      read-add-write in colour passes).
// The element's nodal values come straight from global memory (one lane per
// node; the node arrays of a mesh this size stay in L2). The displacement
// differences d_n = u_n - u_0 are formed from the FP64 state as in the tile
// kernels (an FP32 (hi, lo) pair per value) and shared by all lanes through a
// small per-warp buffer. Warps take the block's element slots (the tile order
// of the mesh) interleaved or in contiguous runs, as the launch schedule says.
// No waits on other warps or on asynchronous copies: nothing to time out.
#pragma once

namespace tlfe {

template <typename R> struct Wpe {
    static constexpr int NODE = 12;                     // per-node row: d (3) | udot (3) | v (3), 16-byte padded
    static constexpr int TS = sizeof(R) == 4 ? 28 : 30;  // per-point row: T0 | T1, or the 27 diagonal moduli
    static constexpr int TAB = 27 * 27 * 4;             // parent gradients [q][n][4]
    static constexpr int WARP = 27 * NODE + 27 * TS;    // values per warp
};

template <typename R> __host__ __device__ constexpr size_t wpe_smem_bytes(int wpb)
{
    return (size_t)(Wpe<R>::TAB + wpb * Wpe<R>::WARP) * sizeof(R);
}

// entry (i, j) of the 1D quadratic mass on [-1, 1] times 30/L: [[4, 2, -1], [2, 16, 2], [-1, 2, 4]]
__device__ __forceinline__ int q27_m1(int i, int j) { return i == j ? (i == 1 ? 16 : 4) : ((i == 1 || j == 1) ? 2 : -1); }

template <typename R, int OP, int MAT>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 2) k_wpe_q27(const KParams<R> p)
{
    constexpr bool HAS_V = OpFields<OP>::NFI == 3;
    constexpr int NODE = Wpe<R>::NODE, TS = Wpe<R>::TS;
    extern __shared__ __align__(128) unsigned char smem[];
    R *tab = reinterpret_cast<R *>(smem);  // [27][27][4]
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    R *nb = tab + Wpe<R>::TAB + (size_t)wib * Wpe<R>::WARP;  // [27][NODE]
    R *tb = nb + 27 * NODE;                                 // [27][TS]

    // parent gradients of the 3x3x3 Gauss points from the constant table
    for (int k = threadIdx.x; k < 27 * 27; k += blockDim.x) {
        const R *src;
        if constexpr (sizeof(R) == 4) src = kQ27F.g[k / 27] + (k % 27) * 3;
        else src = kQ27D.g[k / 27] + (k % 27) * 3;
        tab[k * 4 + 0] = src[0];
        tab[k * 4 + 1] = src[1];
        tab[k * 4 + 2] = src[2];
        tab[k * 4 + 3] = R(0);
    }
    __syncthreads();

    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    const int W = gridDim.x * (blockDim.x >> 5);
    const int s_begin = p.tile_begin * TILE, s_end = p.tile_end * TILE;
    const int n_slots = s_end - s_begin;
    const int per = (n_slots + W - 1) / W;
    const int s0 = p.tile_chunk ? s_begin + gw * per : s_begin + gw;
    const int s1 = p.tile_chunk ? min(s_end, s0 + per) : s_end;
    const int sstep = p.tile_chunk ? 1 : W;
    const bool mass_only = OP == OP_MATVEC && p.mass_only != 0;
    const bool need_ud = p.visc != 0;
    const bool q_lane = lane < 27;  // phase A: point `lane`; phase B: node `lane`
    int bad = 0;

    for (int s = s0; s < s1; s += sstep) {
        const int e = p.eid[s];
        if (e < 0) continue;  // warp-uniform
        const int t = s >> 5, l = s & 31;
        Mat<R> m = p.mat0;
        if (p.mats) m = p.mats[p.emat[s]];
        if (p.elam) {
            m.mu = p.elam[((size_t)t * 2 + 0) * 32 + l];
            m.lam = p.elam[((size_t)t * 2 + 1) * 32 + l];
        }
        if constexpr (MAT == MAT_NH || MAT == MAT_NH_KV) m.model = MODEL_NH;
        if constexpr (MAT == MAT_SVK || MAT == MAT_SVK_KV) m.model = MODEL_SVK;
        const bool visc = MAT == MAT_ANY ? (need_ud && (m.mu_v != R(0) || m.lam_v != R(0)))
                                         : (MAT == MAT_NH_KV || MAT == MAT_SVK_KV);
        R Ji[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) Ji[r] = p.aff[((size_t)t * AFF_ROWS + r) * 32 + l];
        const R detJ = p.aff[((size_t)t * AFF_ROWS + 9) * 32 + l];

        // ---- nodal values of the element: lane n loads node n
        const int nl = q_lane ? lane : 0;
        const int64_t node = bounds_clamp(p.conn[bounds_clamp((int64_t)e - p.elem_base, p.n_elem_block, p.status) * 27 + nl],
                                          p.n_nodes, p.status);
        {
            double u3[3];
            R d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) u3[a] = p.u[3 * node + a];
            if constexpr (sizeof(R) == 4) {
                float h[3], lo[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) split_f64(u3[a], h[a], lo[a]);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float h0 = __shfl_sync(0xffffffffu, h[a], 0), l0 = __shfl_sync(0xffffffffu, lo[a], 0);
                    d[a] = (h[a] - h0) + (lo[a] - l0);
                }
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) d[a] = R(u3[a] - __shfl_sync(0xffffffffu, u3[a], 0));
            }
            if (q_lane) {
                R *row = nb + lane * NODE;
                row[0] = d[0], row[1] = d[1], row[2] = d[2], row[3] = R(0);
                if (visc) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) row[4 + a] = p.ud[3 * node + a];
                }
                if (HAS_V) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) row[8 + a] = p.v[3 * node + a];
                }
            }
        }
        __syncwarp();

        // ---- phase A: point q = lane
        R gmu = R(0), glam = R(0);
        if (q_lane && !mass_only) {
            const int q = lane;
            const R w = quad_weight<ET_Q27, 27, R>(q) * detJ;
            QP<R> s1;
            R D[9];
#pragma unroll
            for (int k2 = 0; k2 < 9; ++k2) {
                s1.G[k2] = R(0);
                s1.Fd[k2] = R(0);
                D[k2] = R(0);
            }
#pragma unroll
            for (int n = 0; n < 27; ++n) {
                const R *g = tab + (q * 27 + n) * 4;
                const R g0 = g[0], g1 = g[1], g2 = g[2];
                const R *row = nb + n * NODE;
                if (n > 0) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R x = row[a];
                        s1.G[a * 3 + 0] += x * g0;
                        s1.G[a * 3 + 1] += x * g1;
                        s1.G[a * 3 + 2] += x * g2;
                    }
                }
                if (visc) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R x = row[4 + a];
                        s1.Fd[a * 3 + 0] += x * g0;
                        s1.Fd[a * 3 + 1] += x * g1;
                        s1.Fd[a * 3 + 2] += x * g2;
                    }
                }
                if (HAS_V) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R x = row[8 + a];
                        D[a * 3 + 0] += x * g0;
                        D[a * 3 + 1] += x * g1;
                        D[a * 3 + 2] += x * g2;
                    }
                }
            }
            {
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
            R P[9];
            stress<R>(m, s1, visc, P);
            bad += s1.ok ? 0 : 1;
            R *trow = tb + q * TS;
            if (OP == OP_DIAG) {
                // diagonal moduli A_d[c][b] = w dP_{d b} / dF_{d c}, d = 0..2
#pragma unroll
                for (int dd = 0; dd < 3; ++dd)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        R E[9], dP[9];
#pragma unroll
                        for (int k2 = 0; k2 < 9; ++k2) E[k2] = (k2 == dd * 3 + c) ? R(1) : R(0);
                        dstress<R>(m, s1, visc, E, p.aK, p.aC, true, dP);
#pragma unroll
                        for (int b2 = 0; b2 < 3; ++b2) trow[dd * 9 + c * 3 + b2] = w * dP[dd * 3 + b2];
                    }
            } else {
                R T0[9], T1[9];
                if (OP == OP_FORCE) {
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) T0[k2] = w * P[k2];
                } else if (OP == OP_MATVEC) {
                    dstress<R>(m, s1, visc, D, p.aK, p.aC, p.sym_only != 0, T0);
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) T0[k2] *= w;
                } else {
                    astress<R>(m, s1, visc, D, T0, T1, gmu, glam);
                    gmu *= w;
                    glam *= w;
#pragma unroll
                    for (int k2 = 0; k2 < 9; ++k2) {
                        T0[k2] *= w;
                        T1[k2] *= w;
                    }
                }
                // rows hold T J^{-T}, so that phase B contracts with the parent gradients
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int k2 = 0; k2 < 3; ++k2)
                        trow[a * 3 + k2] =
                            T0[a * 3] * Ji[k2 * 3] + T0[a * 3 + 1] * Ji[k2 * 3 + 1] + T0[a * 3 + 2] * Ji[k2 * 3 + 2];
                if (OP == OP_VJP) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int k2 = 0; k2 < 3; ++k2)
                            trow[12 + a * 3 + k2] = T1[a * 3] * Ji[k2 * 3] + T1[a * 3 + 1] * Ji[k2 * 3 + 1] +
                                                    T1[a * 3 + 2] * Ji[k2 * 3 + 2];
                }
            }
        }
        __syncwarp();

        // ---- phase B: node n = lane
        if (q_lane) {
            const int n = lane;
            R acc0[3] = {R(0), R(0), R(0)}, acc1[3] = {R(0), R(0), R(0)};
            if (!mass_only) {
#pragma unroll 3
                for (int q = 0; q < 27; ++q) {
                    const R *g = tab + (q * 27 + n) * 4;
                    const R g0 = g[0], g1 = g[1], g2 = g[2];
                    const R *trow = tb + q * TS;
                    if (OP == OP_DIAG) {
                        R hh[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) hh[c] = g0 * Ji[c] + g1 * Ji[3 + c] + g2 * Ji[6 + c];
#pragma unroll
                        for (int dd = 0; dd < 3; ++dd) {
                            const R *A = trow + dd * 9;
                            acc0[dd] += hh[0] * (A[0] * hh[0] + A[1] * hh[1] + A[2] * hh[2]) +
                                        hh[1] * (A[3] * hh[0] + A[4] * hh[1] + A[5] * hh[2]) +
                                        hh[2] * (A[6] * hh[0] + A[7] * hh[1] + A[8] * hh[2]);
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            acc0[a] += trow[a * 3] * g0 + trow[a * 3 + 1] * g1 + trow[a * 3 + 2] * g2;
                            if (OP == OP_VJP)
                                acc1[a] += trow[12 + a * 3] * g0 + trow[12 + a * 3 + 1] * g1 + trow[12 + a * 3 + 2] * g2;
                        }
                    }
                }
            }
            // consistent mass of the parallelepiped: m_nj = rho V Mhat_nj with
            // Mhat the product of the normalised 1D quadratic masses
            if ((OP == OP_MATVEC || OP == OP_DIAG) && p.aM != R(0)) {
                const R c = p.aM * m.rho * p.evol[s] * R(1.0 / 27000.0);
                const int ni = n % 3, nj = (n / 3) % 3, nk = n / 9;
                if (OP == OP_MATVEC) {
#pragma unroll
                    for (int j = 0; j < 27; ++j) {
                        const R mh = c * R(q27_m1(ni, j % 3) * q27_m1(nj, (j / 3) % 3) * q27_m1(nk, j / 9));
                        const R *row = nb + j * NODE;
                        acc0[0] += mh * row[8];
                        acc0[1] += mh * row[9];
                        acc0[2] += mh * row[10];
                    }
                } else {
                    const R mh = c * R(q27_m1(ni, ni) * q27_m1(nj, nj) * q27_m1(nk, nk));
                    acc0[0] += mh;
                    acc0[1] += mh;
                    acc0[2] += mh;
                }
            }
#pragma unroll
            for (int fo = 0; fo < OpFields<OP>::NFO; ++fo) {
                R *out = fo == 0 ? p.out0 : p.out1;
                R *part = fo == 0 ? p.part0 : p.part1;
                const R *a3 = fo == 0 ? acc0 : acc1;
                if (part) {  // sorted scatter: this element's partial for node n
                    const int64_t pos = (int64_t)((int)p.part_base + s * 27 + n);  // positions < 2^31
                    R *dst = part + bounds_clamp(pos, p.n_part, p.status) * 3;
                    dst[0] = a3[0];
                    dst[1] = a3[1];
                    dst[2] = a3[2];
                } else if (p.rmw_scatter) {
                    out[3 * node] += a3[0];
                    out[3 * node + 1] += a3[1];
                    out[3 * node + 2] += a3[2];
                } else {
                    atomicAdd(out + 3 * node, a3[0]);
                    atomicAdd(out + 3 * node + 1, a3[1]);
                    atomicAdd(out + 3 * node + 2, a3[2]);
                }
            }
        }
        if (OP == OP_VJP && p.gth && bounds_ok(e, p.n_elem_total, p.status)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                gmu += __shfl_xor_sync(0xffffffffu, gmu, o);
                glam += __shfl_xor_sync(0xffffffffu, glam, o);
            }
            if (lane == 0) {
                p.gth[(size_t)e * 2 + 0] = double(gmu);
                p.gth[(size_t)e * 2 + 1] = double(glam);
            }
        }
        __syncwarp();  // nb and tb are rewritten by the next element
    }
    const int nbad = __reduce_add_sync(0xffffffffu, bad);
    if (lane == 0 && nbad) atomicAdd(p.status + ST_INVERTED, nbad);
}

template <int OP, typename R> static void (*wpe_kernel_for(int mat))(const KParams<R>)
{
    if constexpr (sizeof(R) == 4) {
        switch (mat) {
        case MAT_NH: return k_wpe_q27<R, OP, MAT_NH>;
        case MAT_NH_KV: return k_wpe_q27<R, OP, MAT_NH_KV>;
        case MAT_SVK: return k_wpe_q27<R, OP, MAT_SVK>;
        case MAT_SVK_KV: return k_wpe_q27<R, OP, MAT_SVK_KV>;
        default: break;
        }
    }
    return k_wpe_q27<R, OP, MAT_ANY>;
}

}  // namespace tlfe
