// 2D pass kernels, FP32 instances (inner solve of the mixed-precision path).
#include "nodal.cuh"
namespace rve {
template cudaError_t launch_pass_a_2d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_pass_c_2d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_pass_e_2d<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_cg_finish_x<float>(const PassArgs<float>&, cudaStream_t);
template cudaError_t launch_force_stencil<float>(const PassArgs<float>&, const float*, float*, float*, cudaStream_t);
template cudaError_t launch_strain_update<float>(const PassArgs<float>&, const float*, cudaStream_t);
template cudaError_t launch_nodal_force<float>(const PassArgs<float>&, const float*, const float*, float*, float*, float*,
                                             cudaStream_t);
template cudaError_t launch_nodal_update<float>(const PassArgs<float>&, const float*, const float*, float*, float*, int,
                                              cudaStream_t);
template cudaError_t launch_nodal_finish<float>(const PassArgs<float>&, const float*, const float*, const float*, cudaStream_t);
}  // namespace rve
