// tlfe_peak_probe: independent fused multiply-add chains on every lane, the
// measured denominator of the element kernels' ALU roofline (FP32) and of the
// plain FP64 path. Each thread runs PROBE_CHAINS independent chains
// x <- x * b + c (b just below 1, c small, so values stay normal) for `iters`
// rounds; one FMA counts as 2 FLOP. The sum of the chains goes to out_dev so
// that nothing is optimised away.
#include <cuda_runtime.h>

#include "tlfe_mesh.h"

namespace tlfe {

constexpr int PROBE_CHAINS = 16;
constexpr int PROBE_THREADS = 256;

template <typename R> __global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(int64_t iters, R *out)
{
    R x[PROBE_CHAINS];
    const R b = R(0.9999999), c = R(1e-7);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = R(threadIdx.x + k);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], b, c);
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == R(-1)) out[0] = s;  // never true for these inputs; keeps the chains alive
    if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

}  // namespace tlfe

using namespace tlfe;

extern "C" tlfe_status tlfe_peak_probe(int32_t precision, int32_t ctas_per_sm, int64_t iters, void *out_dev,
                                       double *flop_host, void *stream)
{
    TLFE_TRACE("tlfe_peak_probe");
    if ((precision != TLFE_FP32 && precision != TLFE_FP64) || ctas_per_sm < 1 || ctas_per_sm > 32 || iters < 1 ||
        iters > ((int64_t)1 << 32) || !out_dev || !flop_host)
        return fail(TLFE_E_INVALID, "tlfe_peak_probe: bad arguments");
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "tlfe_peak_probe: device query");
    const int grid = n_sm * ctas_per_sm;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == TLFE_FP32) k_fma_probe<float><<<grid, PROBE_THREADS, 0, s>>>(iters, (float *)out_dev);
    else k_fma_probe<double><<<grid, PROBE_THREADS, 0, s>>>(iters, (double *)out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tlfe_peak_probe: launch");
    *flop_host = 2.0 * PROBE_CHAINS * (double)PROBE_THREADS * grid * (double)iters;
    return TLFE_OK;
}
