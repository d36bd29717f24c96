// tlfe_norm_noalloc: a variant of the deterministic chunked FP64 norm that the
// Newton step and tlfe_body_norms use, for callers that cannot allocate device
// memory. Its partial sums live in a file-scope device array instead of a
// workspace allocated by the mesh handle.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "tlfe_mesh.h"

namespace tlfe {

constexpr int NA_CHUNK = 4096;              // values per partial (one CTA each)
constexpr int NA_MAX_PARTIALS = 4096;       // size of the scratch array (32 KiB)
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

// Scratch of every call on a device: one partial sum per chunk. Each device
// holds its own copy; all calls on one device share it (each call overwrites
// the partials it reads), so calls that overlap on the same device race.
static __device__ __align__(256) double g_norm_scratch[NA_MAX_PARTIALS];

// Device addresses of g_norm_scratch, looked up once per device. In host code
// the symbol itself is only a host-side stand-in and must not reach a kernel.
// An address stays valid for the life of the device's context; a
// cudaDeviceReset would reload the module elsewhere, so the header asks for a
// process restart after one.
static double *g_scratch_addr[NA_MAX_DEVICES] = {};
static std::mutex g_scratch_mutex;

__global__ void k_na_partials(const double *__restrict__ x, int64_t n, double *__restrict__ partials)
{
    __shared__ double sh[NA_THREADS / 32];
    const int64_t b0 = (int64_t)blockIdx.x * NA_CHUNK;
    const int64_t b1 = b0 + NA_CHUNK < n ? b0 + NA_CHUNK : n;
    double acc = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc += x[i] * x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < NA_THREADS / 32; ++k) s += sh[k];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_na_finish(const double *__restrict__ partials, int n_partials, double *out)
{
    double s = 0.0;
    for (int k = 0; k < n_partials; ++k) s += partials[k];  // fixed order: deterministic
    out[0] = sqrt(s);
}

}  // namespace tlfe

using namespace tlfe;

extern "C" tlfe_status tlfe_norm_noalloc(const double *x_dev, int64_t n, double *out_dev, void *stream)
{
    if (!out_dev || (n > 0 && !x_dev) || n < 0) return fail(TLFE_E_INVALID, "tlfe_norm_noalloc: bad arguments");
    if (n > (int64_t)NA_CHUNK * NA_MAX_PARTIALS)
        return fail(TLFE_E_INVALID, "tlfe_norm_noalloc: n = " + std::to_string(n) + " exceeds the maximum of " +
                                        std::to_string((int64_t)NA_CHUNK * NA_MAX_PARTIALS) +
                                        " values (fixed scratch of " + std::to_string(NA_MAX_PARTIALS) +
                                        " partial sums)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "tlfe_norm_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(TLFE_E_UNSUPPORTED, "tlfe_norm_noalloc: device index too large");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            // once per device, with that device current
            e = cudaGetSymbolAddress((void **)&scratch, g_norm_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "tlfe_norm_noalloc: cudaGetSymbolAddress");
            g_scratch_addr[dev] = scratch;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nc = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    if (nc > 0) k_na_partials<<<nc, NA_THREADS, 0, s>>>(x_dev, n, scratch);
    k_na_finish<<<1, 1, 0, s>>>(scratch, nc, out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tlfe_norm_noalloc: launch");
    return TLFE_OK;
}
