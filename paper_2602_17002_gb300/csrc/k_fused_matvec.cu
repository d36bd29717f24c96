// Fused (one launch over every pass) FP32 matvec kernel, compiled in its own
// translation unit so that the build runs the units in parallel.
#include "k_fused.cuh"

namespace tlfe {
template size_t fused_warp_region<float, OP_MATVEC>(int, int, int);
template int occupancy_fused<OP_MATVEC, float>(size_t, int *);
template cudaError_t launch_fused<OP_MATVEC, float>(const FusedArgs<float> &, int, int, cudaStream_t);
}  // namespace tlfe
