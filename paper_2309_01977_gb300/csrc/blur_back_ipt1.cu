// Back-projection plane blur kernel, 1 j-blur strip(s) per thread.
#include "plane_kernels.cuh"

namespace spect {
template cudaError_t blur_back_launch_ipt<1>(const BlurBackArgs&, int, cudaStream_t);
}  // namespace spect
