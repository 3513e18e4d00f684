// Forward projector kernel, 3 j-blur strip(s) per thread.
#include "plane_kernels.cuh"

namespace spect {
template cudaError_t forward_launch_ipt<3>(const ForwardArgs&, int, cudaStream_t);
template int forward_occupancy_ipt<3>(int, size_t);
}  // namespace spect
