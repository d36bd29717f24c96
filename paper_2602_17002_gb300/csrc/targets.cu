// tlfe_get_scatter_targets: the global node that the element kernels' device
// tables route each (element, local node) to, read back from those tables, so
// that the gather and scatter indices can be compared with the connectivity
// bit for bit (the scatter target of component d of local node i of element e
// is 3 conn[e][i] + d in the [n_nodes][3] node arrays).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "tlfe_mesh.h"

namespace tlfe {

// Inverse of the sorted-scatter transpose: inv[pos[k]] = n for every position
// k of node n (positions of no node keep -1).
__global__ void k_part_inverse(int n_nodes, const int64_t *__restrict__ ptr, const int32_t *__restrict__ pos,
                               int32_t *__restrict__ inv)
{
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_nodes; n += gridDim.x * blockDim.x)
        for (int64_t k = ptr[n]; k < ptr[n + 1]; ++k) inv[pos[k]] = n;
}

// Tile path: one thread per element slot. Walks the slot's metadata record as
// the element kernel does: the gather reads node ids[lidx[i][lane]]; the
// scatter writes slot (i, lane) to node-sorted position spos[i][lane], which
// belongs to the list entry kk with soff[kk] <= position < soff[kk + 1];
// that node's sum goes to node ids[kk] (atomic and colour modes) or to
// partial position P + kk, whose node the transpose names (sorted mode).
__global__ void k_tile_targets(int n_slots, int npe, const unsigned char *__restrict__ meta, int meta_bytes,
                               int umaxp, int elem_base, const int32_t *__restrict__ part_node,
                               int32_t *__restrict__ gather, int32_t *__restrict__ scatter)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots) return;
    const int t = slot >> 5, lane = slot & 31;
    const unsigned char *M = meta + (size_t)t * meta_bytes;
    const int U = reinterpret_cast<const int32_t *>(M)[0];
    const int P = reinterpret_cast<const int32_t *>(M)[1];
    const int e = reinterpret_cast<const int32_t *>(M + 16)[lane];
    if (e < 0) return;
    const int32_t *nodes = reinterpret_cast<const int32_t *>(M + 16 + 128);
    const uint16_t *lidx = reinterpret_cast<const uint16_t *>(M + 16 + 128 + 4 * umaxp);
    const uint16_t *spos = lidx + npe * 32;
    const uint16_t *soff = spos + npe * 32;
    const int64_t o = (int64_t)(e - elem_base) * npe;
    for (int i = 0; i < npe; ++i) {
        gather[o + i] = nodes[lidx[i * 32 + lane]];
        const int ps = spos[i * 32 + lane];
        int lo = 0, hi = U;  // largest kk in [0, U) with soff[kk] <= ps
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (soff[mid] <= ps) lo = mid;
            else hi = mid;
        }
        const bool inside = U > 0 && soff[lo] <= ps && ps < soff[lo + 1];
        scatter[o + i] = !inside ? -1 : (part_node ? part_node[(int64_t)P + lo] : nodes[lo]);
    }
}

// Warp-per-element path (affine Q27): lane n of the element's warp gathers and
// scatters node conn[e][n]; in sorted mode it stores to position
// part_base + slot * 27 + n.
__global__ void k_wpe_targets(int n_slots, const int32_t *__restrict__ eid, const int32_t *__restrict__ conn,
                              int elem_base, int64_t part_base, const int32_t *__restrict__ part_node,
                              int32_t *__restrict__ gather, int32_t *__restrict__ scatter)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots) return;
    const int e = eid[slot];
    if (e < 0) return;
    const int64_t o = (int64_t)(e - elem_base) * 27;
    for (int n = 0; n < 27; ++n) {
        gather[o + n] = conn[o + n];
        scatter[o + n] = part_node ? part_node[part_base + (int64_t)slot * 27 + n] : conn[o + n];
    }
}

}  // namespace tlfe

using namespace tlfe;

extern "C" tlfe_status tlfe_get_scatter_targets(const tlfe_mesh *m, int32_t *gather_host, int32_t *scatter_host)
{
    TLFE_TRACE("tlfe_get_scatter_targets");
    if (!m || (!gather_host && !scatter_host)) return fail(TLFE_E_INVALID, "NULL argument");
    int64_t total = 0;
    for (auto &B : m->blocks) total += (int64_t)B.n_elem * B.npe;
    if (total == 0) return TLFE_OK;
    const bool sorted = m->scatter == TLFE_SCATTER_SORTED;
    int32_t *d_g = nullptr, *d_s = nullptr, *d_inv = nullptr;
    cudaError_t e = cudaMalloc(&d_g, sizeof(int32_t) * total);
    if (e == cudaSuccess) e = cudaMalloc(&d_s, sizeof(int32_t) * total);
    if (e == cudaSuccess && sorted) e = cudaMalloc(&d_inv, sizeof(int32_t) * std::max<int64_t>(1, m->n_part));
    if (e == cudaSuccess) e = cudaMemset(d_g, 0xff, sizeof(int32_t) * total);
    if (e == cudaSuccess) e = cudaMemset(d_s, 0xff, sizeof(int32_t) * total);
    if (e == cudaSuccess && sorted) {
        e = cudaMemset(d_inv, 0xff, sizeof(int32_t) * std::max<int64_t>(1, m->n_part));
        if (e == cudaSuccess) {
            k_part_inverse<<<std::max(1, std::min((m->n_nodes + 255) / 256, 4096)), 256>>>(m->n_nodes, m->d_part_ptr,
                                                                                         m->d_part_pos, d_inv);
            e = cudaGetLastError();
        }
    }
    int64_t off = 0;
    for (size_t bi = 0; bi < m->blocks.size() && e == cudaSuccess; ++bi) {
        const BlockStore &B = m->blocks[bi];
        if (B.n_elem > 0) {
            const int n_slots = B.n_tiles * TILE;
            const int grid = (n_slots + 127) / 128;
            if (wpe_path(B.et, B.use_affine))
                k_wpe_targets<<<grid, 128>>>(n_slots, B.d_eid, B.d_conn, B.elem_base, B.part_base, d_inv, d_g + off,
                                             d_s + off);
            else
                k_tile_targets<<<grid, 128>>>(n_slots, B.npe, B.d_meta, B.meta_bytes, B.meta_umaxp, B.elem_base, d_inv,
                                              d_g + off, d_s + off);
            e = cudaGetLastError();
        }
        off += (int64_t)B.n_elem * B.npe;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && gather_host) e = cudaMemcpy(gather_host, d_g, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && scatter_host)
        e = cudaMemcpy(scatter_host, d_s, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
    cudaFree(d_g);
    cudaFree(d_s);
    cudaFree(d_inv);
    if (e != cudaSuccess) return cuda_fail(e, "tlfe_get_scatter_targets");
    return TLFE_OK;
}
