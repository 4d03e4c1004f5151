// Launchers of the FP64 real-space kernels (residual, homogenisation,
// strain field, adjoint gradient), dispatched on the dimension.
#include "pass2d_fp64.cuh"
#include "pass3d_fp64.cuh"

namespace rve {

constexpr int kNT = 256;

cudaError_t launch_residual(const Fp64Args& a, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + kNT - 1) / kNT), a.L);
  if (a.dim == 2) residual_2d<kNT><<<grid, kNT, 0, s>>>(a);
  else return launch_residual_3d(a, s);
  return cudaGetLastError();
}

int homogenise_blocks(const Fp64Args& a) { return (int)((a.N + kNT - 1) / kNT); }

cudaError_t launch_homogenise(const Fp64Args& a, double* part, int* nblk_out, cudaStream_t s) {
  const int nblk = homogenise_blocks(a);
  *nblk_out = nblk;
  dim3 grid(nblk, a.L);
  if (a.dim == 2) homogenise_2d<kNT><<<grid, kNT, 0, s>>>(a, part, nblk);
  else homogenise_3d<kNT><<<grid, kNT, 0, s>>>(a, part, nblk);
  return cudaGetLastError();
}

cudaError_t launch_energy(const Fp64Args& a, double* part, int* nblk_out, cudaStream_t s) {
  const int nblk = homogenise_blocks(a);
  *nblk_out = nblk;
  if (a.dim == 2) energy_2d<kNT><<<nblk, kNT, 0, s>>>(a, part, nblk);
  else energy_3d<kNT><<<nblk, kNT, 0, s>>>(a, part, nblk);
  return cudaGetLastError();
}

cudaError_t launch_strain_field(const Fp64Args& a, int l, double* out, cudaStream_t s) {
  const unsigned nb = (unsigned)((a.N + kNT - 1) / kNT);
  if (a.dim == 2) strain_field_2d<<<nb, kNT, 0, s>>>(a, l, out);
  else strain_field_3d<<<nb, kNT, 0, s>>>(a, l, out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_grad(const Fp64Args& a, const double* uadj, const double* W, const int* has_adj,
                                double scale, double* grad, cudaStream_t s) {
  const unsigned nb = (unsigned)((a.N + 127) / 128);
  if (a.dim == 2) adjoint_grad_2d<<<nb, 128, 0, s>>>(a, uadj, W, has_adj, scale, grad);
  else adjoint_grad_3d<<<nb, 128, 0, s>>>(a, uadj, W, has_adj, scale, grad);
  return cudaGetLastError();
}

}  // namespace rve
