// Instantiations of the element kernel for OP_VJP.
#include "k_elem.cuh"

namespace tlfe {
template cudaError_t launch_op<OP_VJP, float>(int, int, const KParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_op<OP_VJP, double>(int, int, const KParams<double> &, int, int, cudaStream_t);
template int occupancy_op<OP_VJP, float>(int, int, bool, int, int, int, int *, std::string *);
template int occupancy_op<OP_VJP, double>(int, int, bool, int, int, int, int *, std::string *);
}  // namespace tlfe
