// Launchers of the FP64 real-space kernels (residual, homogenisation,
// strain field, adjoint gradient), dispatched on the dimension.
#include "pass2d_fp64.cuh"
#include "pass3d_fp64.cuh"

namespace rve {

constexpr int kNT = 256;

cudaError_t launch_residual(const Fp64Args& a, cudaStream_t s) {
  return a.dim == 2 ? launch_residual_2d(a, s) : launch_residual_3d(a, s);
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

// ---- strain-state solve (derivatives without a finite-element stencil) ----
// x: [L][m][N] FP64 strain fluctuation of the projected CG, m = nq * ns.

// Block partial sums of the mean stress of C (E + x) over all elements.
template <int NT>
__global__ void __launch_bounds__(NT) homogenise_strain(Fp64Args a, const double* __restrict__ x, double* part,
                                                        int nblk) {
  __shared__ double red[NT / 32];
  const int l = blockIdx.y;
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int ns = a.ns, D = a.dim, m = a.nq * a.ns;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (v < a.N) {
    const double e = a.E[(int64_t)(l / a.lcs) * a.N + v];
    for (int q = 0; q < a.nq; ++q) {
      double eps[6];
      for (int s2 = 0; s2 < ns; ++s2) eps[s2] = a.emac[l * ns + s2] + x[((int64_t)l * m + q * ns + s2) * a.N + v];
      double tr = 0.0;
      for (int s2 = 0; s2 < D; ++s2) tr += eps[s2];
      for (int s2 = 0; s2 < ns; ++s2) acc[s2] += (s2 < D) ? e * (a.lam * tr + a.mu2 * eps[s2]) : e * a.mu2 * eps[s2];
    }
  }
  for (int s2 = 0; s2 < ns; ++s2) {
    const double t = block_sum<NT>(acc[s2], red);
    if (threadIdx.x == 0) part[((int64_t)l * ns + s2) * nblk + blockIdx.x] = t;
  }
}

// out[c][v] = E_c + x[l][c][v] (total strain of load case l).
__global__ void strain_total(Fp64Args a, const double* __restrict__ x, int l, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = a.nq * a.ns;
  if (i >= (int64_t)m * a.N) return;
  const int c = (int)(i / a.N);
  out[i] = a.emac[l * a.ns + c % a.ns] + x[(int64_t)l * m * a.N + i];
}

cudaError_t launch_homogenise_strain(const Fp64Args& a, const double* x, double* part, int* nblk_out,
                                     cudaStream_t s) {
  const int nblk = homogenise_blocks(a);
  *nblk_out = nblk;
  homogenise_strain<kNT><<<dim3(nblk, a.L), kNT, 0, s>>>(a, x, part, nblk);
  return cudaGetLastError();
}

cudaError_t launch_strain_total(const Fp64Args& a, const double* x, int l, double* out, cudaStream_t s) {
  const int64_t tot = (int64_t)a.nq * a.ns * a.N;
  strain_total<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a, x, l, out);
  return cudaGetLastError();
}

}  // namespace rve
