// Back-projection plane blur kernel, 4 j-blur strip(s) per thread.
#include "plane_kernels.cuh"

namespace spect {
template cudaError_t blur_back_launch_ipt<4>(const BlurBackArgs&, int, cudaStream_t);
}  // namespace spect
