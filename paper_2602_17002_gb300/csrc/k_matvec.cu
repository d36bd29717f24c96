// Instantiations of the element kernel for OP_MATVEC.
#include "k_elem.cuh"

namespace tlfe {
template cudaError_t launch_op<OP_MATVEC, float>(int, int, const KParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_op<OP_MATVEC, double>(int, int, const KParams<double> &, int, int, cudaStream_t);
template int occupancy_op<OP_MATVEC, float>(int, int, bool, int, int, int, int *, std::string *);
template int occupancy_op<OP_MATVEC, double>(int, int, bool, int, int, int, int *, std::string *);
}  // namespace tlfe
