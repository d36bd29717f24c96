// Instantiations of the element kernel for OP_VJP.
#include "k_elem.cuh"

namespace tlfe {
template cudaError_t launch_op<OP_VJP, float>(int, int, const KParams<float> &, int, cudaStream_t);
template cudaError_t launch_op<OP_VJP, double>(int, int, const KParams<double> &, int, cudaStream_t);
template int occupancy_op<OP_VJP, float>(int, int, size_t);
template int occupancy_op<OP_VJP, double>(int, int, size_t);
}  // namespace tlfe
