// Instantiations of the element kernel for OP_FM (internal force and operator
// product in one pass; FP32 T4, T10 and H8 blocks).
#include "k_elem.cuh"

namespace tlfe {
template cudaError_t launch_op<OP_FM, float>(int, int, const KParams<float> &, int, int, cudaStream_t);
template int occupancy_op<OP_FM, float>(int, int, bool, int, int, int, int *, std::string *);
}  // namespace tlfe
