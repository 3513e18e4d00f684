// Forward projector kernel, 2 j-blur strip(s) per thread.
#include "plane_kernels.cuh"

namespace spect {
template cudaError_t forward_launch_ipt<2>(const ForwardArgs&, int, cudaStream_t);
template int forward_occupancy_ipt<2>(int, size_t);
}  // namespace spect
