// Diagnostic for the failure path of bounded device-side waits.
//
// The element kernels wait on mbarriers for their bulk copies with a bounded
// number of try_wait rounds; when a copy never lands they latch ST_TIMEOUT in
// the mesh's status word and return, so that the host sees TLFE_E_TIMEOUT at
// the next tlfe_sync and the context stays usable. Nothing in a correct run
// makes such a wait run out, so this entry point provokes exactly that path
// without any fault: one warp arms an mbarrier for 16 bytes that no copy will
// deliver and waits on it with the same bounded try_wait loop.
#include "k_elem.cuh"
#include "tlfe_mesh.h"

namespace tlfe {

__global__ void k_wait_timeout(int *status, long long spin_limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);  // the arrival; its 16 bytes never come
    __syncthreads();
    long long spins = 0;
    bool done = false;
    while (!(done = mbar_try_wait(&bar, 0)) && ++spins < spin_limit) {
    }
    if (!done && threadIdx.x == 0) atomicAdd(status + ST_TIMEOUT, 1);
}

}  // namespace tlfe

using namespace tlfe;

extern "C" tlfe_status tlfe_selftest_wait_timeout(tlfe_mesh *m, int64_t spin_limit, void *stream)
{
    TLFE_TRACE("tlfe_selftest_wait_timeout");
    if (!m) return fail(TLFE_E_INVALID, "mesh is NULL");
    if (spin_limit < 1 || spin_limit > (int64_t)MBAR_SPIN_LIMIT)
        return fail(TLFE_E_INVALID, "spin_limit must be in [1, " + std::to_string(MBAR_SPIN_LIMIT) + "]");
    k_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(m->d_status, (long long)spin_limit);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tlfe_selftest_wait_timeout");
    return TLFE_OK;
}
