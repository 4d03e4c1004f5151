// 2D pass kernels, FP64 instances.
#include "nodal.cuh"
namespace rve {
template cudaError_t launch_pass_a_2d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_c_2d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_pass_e_2d<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_cg_finish_x<double>(const PassArgs<double>&, cudaStream_t);
template cudaError_t launch_force_stencil<double>(const PassArgs<double>&, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_strain_update<double>(const PassArgs<double>&, const double*, cudaStream_t);
template cudaError_t launch_nodal_force<double>(const PassArgs<double>&, const double*, const double*, double*, double*, double*,
                                             cudaStream_t);
template cudaError_t launch_nodal_update<double>(const PassArgs<double>&, const double*, const double*, double*, double*, int,
                                              cudaStream_t);
template cudaError_t launch_nodal_finish<double>(const PassArgs<double>&, const double*, const double*, const double*, cudaStream_t);
}  // namespace rve
