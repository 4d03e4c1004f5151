// Host-side declarations shared by the C-ABI translation unit and the kernel
// translation units (one per dimension and precision).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rve_device.cuh"

namespace rve {

// Modes of the first pass (material + forward x-FFT)
enum PassAMode {
  A_CG = 0,      // p <- r + beta p ; sigma = C p ; <p, sigma> -> alpha
  A_MACRO = 1,   // sigma = C E_macro (broadcast)      (start: r0 = -G C E)
  A_FIELD = 2,   // sigma = C in  (in = strain field)  (operator application)
  A_BARE = 3,    // sigma = in (no material)           (bare projection / eps -> u)
  A_NODAL = 4    // transform the D nodal components of in (FP64 residual -> rhs)
};
// Modes of the last pass (inverse x-FFT + update)
enum PassEMode {
  E_CG = 0,      // r -= alpha q ; <r, r> -> beta, convergence
  E_INIT = 1,    // r = -q ; x = 0 ; <r, r> -> rr0
  E_OUT = 2,     // out = q (m components)
  E_NODAL = 3,   // u64 += q (D nodal components, accumulated in FP64)
  E_NOUT = 4     // out = q (D nodal components, inner precision)
};
// Modes of the projection pass
enum ProjMode {
  P_G = 0,       // eps^ = B (B^H B)^-1 B^H sigma^  (m -> m)
  P_NODAL_IN = 1,  // eps^ = B (B^H B)^-1 f^          (D -> m)
  P_NODAL_OUT = 2, // u^ = (B^H B)^-1 B^H eps^        (m -> D)
  P_SOLVE = 3,     // w^ = (B^H B)^-1 f^              (D -> D, factored form)
  P_FINITE = 4     // H^ = G H^ on deformation gradients (finite strain, n_q D^2 components)
};

// Everything a pass kernel needs; all pointers are device pointers.
// discrete derivative (B(k)) of the projection: the linear finite elements or
// one of the other stencils of Secs. 2.3-2.5 and Appendix C
enum Deriv { D_FE = 0, D_FOURIER = 1, D_CENTRAL = 2, D_FORWARD = 3, D_LSQ = 4, D_FOURIER2 = 5 };

template <typename T> struct PassArgs {
  int n[3];          // grid sizes (x, y, z); z = 1 in 2D
  int dim, L, m, ns, nq;
  int64_t N;         // voxels
  int kx;            // n_x/2 + 1
  const T* E;        // [L / lcs][N] Young's modulus (one field per material)
  int lcs;           // load-case slots per material: slot l uses field l / lcs
  T* x; T* r; T* p;  // [L][m][N] CG vectors
  T* p2;             // second direction buffer of the factored form (p alternates p, p2), else null
  const T* in;       // [L][m or D][N] input field (A_FIELD / A_BARE / A_NODAL)
  T* out;            // [L][m][N] output field (E_OUT)
  double* u64;       // [L][D][N] FP64 nodal displacement (E_NODAL)
  cplx<T>* spec;     // first spectrum buffer
  cplx<T>* spec2;    // second spectrum buffer (3D)
  const double* emac;  // [L][ns] macroscopic strains
  const cplx<T>* ph[3];  // exp(2 pi i j / n_a), j < n_a
  const cplx<T>* tw[3];  // exp(-2 pi i t / n_a), t < n_a
  T lam, mu2;        // unit-modulus Lame lambda and 2 mu
  T ih[3];           // inverse voxel sizes
  T inv_n;           // 1 / N
  T emac_scale;      // sign/scale for A_MACRO
  CgState* cg;       // [L]
  double* part;      // [L][part_stride] block partial sums
  int part_stride;
  int amode, emode, pmode;
  int cgphase;       // 1 inside the CG loop: passes skip load cases whose CG stopped
  int var_a, var_e;  // tile variants of passes A (0..6) and E (0..4): see the launchers
  int var_c, var_y;  // FFT split variants (FftSplit<N, V>) of pass C's axis and of passes B / D (3D)
  int comp_in;       // number of components in the spectrum for this pass (m or D)
  const void* tm_spec;  // host copy of the TMA tensor map of the first spectrum (3D FP32), or null
  int stall_copies;     // test hook: the pipelined passes issue no copies, so their bounded waits run out
  int pf_ahead;      // 3D passes A and E: blocks ahead in launch order whose rows each block asks the TMA
                     // unit to prefetch into L2 (tile variants A 6 and E 4), 0 = none
  int deriv;         // Deriv
};

// Arguments of the FP64 real-space kernels (residual, homogenisation, adjoint).
struct Fp64Args {
  int n[3];
  int dim, L, ns, nq;
  int64_t N;
  const double* E;      // [L / lcs][N]
  int lcs;              // load-case slots per material (slot l uses field l / lcs)
  const double* u;      // [L][D][N] nodal fluctuation displacement
  const double* emac;   // [L][ns]
  double ih[3], lam, mu2;
  CgState* cg;          // [L]
  double* part;         // [L][part_stride]
  int part_stride;
  void* fout;           // [L][D][N] residual in the inner precision
  int fout_f32;
};

// Launchers (return cudaError_t of the launch).  Defined per dimension and
// precision; they pick the template instance for the grid sizes.
template <typename T> cudaError_t launch_pass_a_2d(const PassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_pass_c_2d(const PassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_pass_e_2d(const PassArgs<T>& a, cudaStream_t s);

template <typename T> cudaError_t launch_cg_finish_x(const PassArgs<T>& a, cudaStream_t s);
// factored nodal form of the operator
template <typename T>
cudaError_t launch_force_stencil(const PassArgs<T>& a, const T* pold, T* pnew, T* f, cudaStream_t s);
template <typename T> cudaError_t launch_strain_update(const PassArgs<T>& a, const T* w, cudaStream_t s);
// nodal-state form
template <typename T>
cudaError_t launch_nodal_force(const PassArgs<T>& a, const T* rho, const T* pold, T* pnew, T* xi, T* f,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_nodal_update(const PassArgs<T>& a, const T* rho_old, const T* w, T* rho_new, T* xi, int init,
                                cudaStream_t s);
template <typename T>
cudaError_t launch_nodal_finish(const PassArgs<T>& a, const T* pi_even, const T* pi_odd, const T* xi,
                                cudaStream_t s);

template <typename T> cudaError_t launch_pass_a_3d(const PassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_pass_b_3d(const PassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_pass_c_3d(const PassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_pass_d_3d(const PassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_pass_e_3d(const PassArgs<T>& a, cudaStream_t s);

cudaError_t launch_residual(const Fp64Args& a, cudaStream_t s);
// part[(l*ns + s)*nblk + blk]; returns nblk through *nblk_out
cudaError_t launch_homogenise(const Fp64Args& a, double* part, int* nblk_out, cudaStream_t s);
int homogenise_blocks(const Fp64Args& a);
// part[p * nblk + blk] for the pairs p of (a <= b), a, b < L; returns nblk
cudaError_t launch_energy(const Fp64Args& a, double* part, int* nblk_out, cudaStream_t s);
cudaError_t launch_strain_field(const Fp64Args& a, int l, double* out, cudaStream_t s);
// finite strain (FP64): F, P, t are [L][m][N] deformation-gradient fields
cudaError_t launch_fs_init(const PassArgs<double>& a, double* F, const double* Fmac, cudaStream_t s);
cudaError_t launch_fs_stress(const PassArgs<double>& a, const double* F, double* P, cudaStream_t s);
cudaError_t launch_fs_dir_tangent(const PassArgs<double>& a, const double* F, double* t, cudaStream_t s);
cudaError_t launch_fs_add(const PassArgs<double>& a, double* F, cudaStream_t s);
int fs_mean_blocks(const PassArgs<double>& a);
cudaError_t launch_fs_mean(const PassArgs<double>& a, const double* F, double* part, cudaStream_t s);
// strain-state solve (FP64 CG vector x [L][m][N] holds the strain fluctuation)
cudaError_t launch_homogenise_strain(const Fp64Args& a, const double* x, double* part, int* nblk_out,
                                     cudaStream_t s);
cudaError_t launch_strain_total(const Fp64Args& a, const double* x, int l, double* out, cudaStream_t s);
cudaError_t launch_adjoint_grad(const Fp64Args& a, const double* uadj, const double* W, const int* has_adj,
                                double scale, double* grad, cudaStream_t s);

// Largest number of blocks per load case any reducing pass uses.
int max_reduce_blocks(const int* n, int dim, bool fp64);

bool size_supported(const int* n, int dim);

}  // namespace rve
