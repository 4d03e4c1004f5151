// 3D pass kernels, FP32 instances (inner solve of the mixed-precision path).
#include "pass3d.cuh"
namespace rve {
template cudaError_t launch_pass_a_3d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_pass_b_3d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_pass_c_3d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_pass_d_3d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_pass_e_3d<float>(const PassArgs<float>&, cudaStream_t);
}  // namespace rve
