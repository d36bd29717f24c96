// Instantiations of the element kernel for OP_FORCE.
#include "k_elem.cuh"

namespace tlfe {
template cudaError_t launch_op<OP_FORCE, float>(int, int, const KParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_op<OP_FORCE, double>(int, int, const KParams<double> &, int, int, cudaStream_t);
template int occupancy_op<OP_FORCE, float>(int, int, bool, int, int, int, int *, std::string *);
template int occupancy_op<OP_FORCE, double>(int, int, bool, int, int, int, int *, std::string *);
}  // namespace tlfe
