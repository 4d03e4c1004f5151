// 2D pass kernels, FP64 instances.
#include "factored.cuh"
namespace rve {
template cudaError_t launch_pass_a_2d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_c_2d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_e_2d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_cg_finish_x<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_force_stencil<double>(const PassArgs<double>&, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_strain_update<double>(const PassArgs<double>&, const double*, cudaStream_t);
}  // namespace rve
