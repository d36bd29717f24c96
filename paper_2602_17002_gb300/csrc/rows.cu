// tlfe_gather_nodes / tlfe_scatter_nodes: rows of a [n][3] node array packed
// into, or written back from, a compact buffer (the interface exchange of a
// body split across GPUs: duplicated interface nodes are summed over the
// ranks through one compact buffer per operator application).
#include <cuda_runtime.h>

#include <string>

#include "tlfe_mesh.h"

namespace tlfe {

// dst[(dmap ? dmap[k] : k)][c] = src[(smap ? smap[k] : k)][c], k < n, c < 3
template <typename R>
__global__ void k_move_rows(const R *__restrict__ src, const int32_t *__restrict__ smap, const int32_t *__restrict__ dmap,
                            int n, R *__restrict__ dst)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) {
        const int k = i / 3, c = i - 3 * k;
        const int64_t sr = smap ? smap[k] : k, dr = dmap ? dmap[k] : k;
        dst[3 * dr + c] = src[3 * sr + c];
    }
}

template <typename R> __global__ void k_zero_rows(int n, R *__restrict__ x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) x[i] = R(0);
}

static int grid_for(int n) { return (3 * n + 255) / 256 < 4096 ? (3 * n + 255) / 256 : 4096; }

template <typename R>
static cudaError_t move_rows(const void *src, const int32_t *smap, const int32_t *dmap, int n, void *dst, int clear,
                             cudaStream_t s)
{
    if (clear > 0) k_zero_rows<R><<<grid_for(clear), 256, 0, s>>>(clear, (R *)dst);
    if (n > 0) k_move_rows<R><<<grid_for(n), 256, 0, s>>>((const R *)src, smap, dmap, n, (R *)dst);
    return cudaGetLastError();
}

static tlfe_status rows(const char *what, int32_t precision, const void *src, const int32_t *smap,
                        const int32_t *dmap, int32_t n, void *dst, int32_t clear, void *stream)
{
    if ((precision != TLFE_FP32 && precision != TLFE_FP64) || n < 0 || clear < 0 || (n > 0 && !src) ||
        ((n > 0 || clear > 0) && !dst))
        return fail(TLFE_E_INVALID, std::string(what) + ": bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = precision == TLFE_FP32 ? move_rows<float>(src, smap, dmap, n, dst, clear, s)
                                           : move_rows<double>(src, smap, dmap, n, dst, clear, s);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return TLFE_OK;
}

}  // namespace tlfe

extern "C" tlfe_status tlfe_gather_nodes(int32_t precision, const void *x_dev, const int32_t *idx_dev, int32_t n,
                                         void *out_dev, const int32_t *out_idx_dev, int32_t n_out_clear,
                                         void *stream)
{
    TLFE_TRACE("tlfe_gather_nodes");
    if (n > 0 && !idx_dev) return tlfe::fail(TLFE_E_INVALID, "tlfe_gather_nodes: idx is NULL");
    return tlfe::rows("tlfe_gather_nodes", precision, x_dev, idx_dev, out_idx_dev, n, out_dev, n_out_clear, stream);
}

extern "C" tlfe_status tlfe_scatter_nodes(int32_t precision, const void *in_dev, const int32_t *in_idx_dev,
                                          const int32_t *idx_dev, int32_t n, void *x_dev, void *stream)
{
    TLFE_TRACE("tlfe_scatter_nodes");
    if (n > 0 && !idx_dev) return tlfe::fail(TLFE_E_INVALID, "tlfe_scatter_nodes: idx is NULL");
    return tlfe::rows("tlfe_scatter_nodes", precision, in_dev, in_idx_dev, idx_dev, n, x_dev, 0, stream);
}
