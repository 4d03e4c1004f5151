// 3D pass kernels, FP64 instances.
#include "pass3d.cuh"
namespace rve {
template cudaError_t launch_pass_a_3d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_b_3d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_c_3d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_d_3d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_e_3d<double>(const PassArgs<double>&, cudaStream_t);
}  // namespace rve
