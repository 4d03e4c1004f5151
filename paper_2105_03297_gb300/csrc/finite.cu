// Finite strain (St. Venant-Kirchhoff), FP64: the elementwise kernels of the
// Newton-projected-CG solve.  The FFT passes (A in bare mode, B, C with the
// gradient projection, D, E) apply G; these kernels supply the law.
//
// Fields: [L][m][N] with m = n_q D^2 (+1 zero padding in 2D); component
// Theta D^2 + i D + a holds F_{ia} = d chi_i / d r_a of element Theta.
// Law (per voxel modulus E_v, unit-modulus lambda and 2 mu in a.lam, a.mu2):
//   E = (F^T F - I)/2,  S = E_v (lambda tr(E) I + 2 mu E),  P = F S,
//   dP = dF S + F dS,   dS = E_v (lambda tr(dE) I + 2 mu dE),  dE = sym(F^T dF).
#include "rve_device.cuh"
#include "rve_internal.h"

namespace rve {

namespace {

constexpr int kFT = 128;

__device__ __forceinline__ int n_elem(int dim) { return dim == 2 ? 2 : 6; }

template <int D>
__device__ __forceinline__ void pk2(const double F[3][3], double e, double lam, double mu2, double S[3][3]) {
  double E[3][3], tr = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double c = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) c += F[k][i] * F[k][j];
      E[i][j] = 0.5 * (c - (i == j ? 1.0 : 0.0));
    }
#pragma unroll
  for (int i = 0; i < D; ++i) tr += E[i][i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) S[i][j] = e * (mu2 * E[i][j] + (i == j ? lam * tr : 0.0));
}

template <int D>
__device__ __forceinline__ void load_mat(const double* src, int64_t stride, double M[3][3]) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int a = 0; a < D; ++a) M[i][a] = src[(i * D + a) * stride];
}

// F = F_macro on every element (padding 0).  grid (ceil(N/kFT), L).
template <int D>
__global__ void __launch_bounds__(kFT) fs_init(PassArgs<double> a, double* __restrict__ F,
                                               const double* __restrict__ Fmac) {
  const int l = blockIdx.y;
  const int64_t v = (int64_t)blockIdx.x * kFT + threadIdx.x;
  if (v >= a.N || !a.cg[l].active) return;
  const int nd = n_elem(D) * D * D;
  for (int c = 0; c < a.m; ++c)
    F[((int64_t)l * a.m + c) * a.N + v] = (c < nd) ? Fmac[l * D * D + c % (D * D)] : 0.0;
}

// P = F S(F) into P (padding 0) and |P|^2 of the slot into cg->fa2.
template <int D>
__global__ void __launch_bounds__(kFT) fs_stress(PassArgs<double> a, const double* __restrict__ F,
                                                 double* __restrict__ P) {
  __shared__ double red[kFT / 32];
  __shared__ int flag;
  const int l = blockIdx.y;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  const int64_t v = (int64_t)blockIdx.x * kFT + threadIdx.x;
  const int64_t N = a.N;
  double acc = 0.0;
  if (v < N) {
    const double e = a.E[(int64_t)(l / a.lcs) * N + v];
    const int64_t base = (int64_t)l * a.m * N + v;
    for (int q = 0; q < n_elem(D); ++q) {
      double Fm[3][3], S[3][3];
      load_mat<D>(F + base + (int64_t)q * D * D * N, N, Fm);
      pk2<D>(Fm, e, a.lam, a.mu2, S);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) s += Fm[i][k] * S[k][j];
          P[base + (int64_t)(q * D * D + i * D + j) * N] = s;
          acc += s * s;
        }
    }
    for (int c = n_elem(D) * D * D; c < a.m; ++c) P[base + (int64_t)c * N] = 0.0;
  }
  const double s = block_sum<kFT>(acc, red);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_r, blockIdx.x, gridDim.x, &flag)) {
    const double t = sum_partials<kFT>(part, gridDim.x, red);
    if (threadIdx.x == 0) { cg->fa2 = t; cg->cnt_r = 0; }
  }
}

// One CG step before the FFT passes: p = r + beta p_old, x += alpha_prev p_old
// (deferred update), t = K(F) : p, <p, t> -> alpha.
template <int D>
__global__ void __launch_bounds__(kFT) fs_dir_tangent(PassArgs<double> a, const double* __restrict__ F,
                                                      double* __restrict__ t) {
  __shared__ double red[kFT / 32];
  __shared__ int flag;
  const int l = blockIdx.y;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t v = (int64_t)blockIdx.x * kFT + threadIdx.x;
  const int64_t N = a.N;
  const double beta = cg->beta, alpha_prev = cg->alpha;
  const bool use_old = cg->it > 0;
  double acc = 0.0;
  if (v < N) {
    const double e = a.E[(int64_t)(l / a.lcs) * N + v];
    const int64_t base = (int64_t)l * a.m * N + v;
    for (int q = 0; q < n_elem(D); ++q) {
      const int64_t eb = base + (int64_t)q * D * D * N;
      double Fm[3][3], pm[3][3];
      load_mat<D>(F + eb, N, Fm);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const int64_t idx = eb + (int64_t)(i * D + j) * N;
          double pv = a.r[idx];
          if (use_old) {
            const double po = a.p[idx];
            pv += beta * po;
            a.x[idx] += alpha_prev * po;
          }
          a.p[idx] = pv;
          pm[i][j] = pv;
        }
      double S[3][3], dE[3][3], trd = 0.0;
      pk2<D>(Fm, e, a.lam, a.mu2, S);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double c1 = 0.0, c2 = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) { c1 += Fm[k][i] * pm[k][j]; c2 += Fm[k][j] * pm[k][i]; }
          dE[i][j] = 0.5 * (c1 + c2);
        }
#pragma unroll
      for (int i = 0; i < D; ++i) trd += dE[i][i];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double tv = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const double dS = e * (a.mu2 * dE[k][j] + (k == j ? a.lam * trd : 0.0));
            tv += pm[i][k] * S[k][j] + Fm[i][k] * dS;
          }
          t[eb + (int64_t)(i * D + j) * N] = tv;
          acc += pm[i][j] * tv;
        }
    }
    for (int c = n_elem(D) * D * D; c < a.m; ++c) t[base + (int64_t)c * N] = 0.0;
  }
  const double s = block_sum<kFT>(acc, red);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_a, blockIdx.x, gridDim.x, &flag)) {
    const double pq = sum_partials<kFT>(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      cg->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) { cg->status = ST_BAD; cg->alpha = 0.0; }
      else cg->alpha = cg->rr / pq;
      cg->cnt_a = 0;
    }
  }
}

// F += x for every slot still active.
__global__ void __launch_bounds__(kFT) fs_add(PassArgs<double> a, double* __restrict__ F) {
  const int l = blockIdx.y;
  if (!a.cg[l].active) return;
  const int64_t i = (int64_t)blockIdx.x * kFT + threadIdx.x;
  if (i >= (int64_t)a.m * a.N) return;
  const int64_t idx = (int64_t)l * a.m * a.N + i;
  F[idx] += a.x[idx];
}

// Block partial sums of P over all elements: part[(l D^2 + c) nblk + blk].
template <int D>
__global__ void __launch_bounds__(kFT) fs_mean(PassArgs<double> a, const double* __restrict__ F, double* part,
                                               int nblk) {
  __shared__ double red[kFT / 32];
  const int l = blockIdx.y;
  const int64_t v = (int64_t)blockIdx.x * kFT + threadIdx.x;
  const int64_t N = a.N;
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  if (v < N) {
    const double e = a.E[(int64_t)(l / a.lcs) * N + v];
    const int64_t base = (int64_t)l * a.m * N + v;
    for (int q = 0; q < n_elem(D); ++q) {
      double Fm[3][3], S[3][3];
      load_mat<D>(F + base + (int64_t)q * D * D * N, N, Fm);
      pk2<D>(Fm, e, a.lam, a.mu2, S);
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) s += Fm[i][k] * S[k][j];
          acc[i * D + j] += s;
        }
    }
  }
#pragma unroll
  for (int c = 0; c < D * D; ++c) {
    const double s = block_sum<kFT>(acc[c], red);
    if (threadIdx.x == 0) part[((int64_t)l * D * D + c) * nblk + blockIdx.x] = s;
  }
}

}  // namespace

cudaError_t launch_fs_init(const PassArgs<double>& a, double* F, const double* Fmac, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + kFT - 1) / kFT), a.L);
  if (a.dim == 2) fs_init<2><<<grid, kFT, 0, s>>>(a, F, Fmac);
  else fs_init<3><<<grid, kFT, 0, s>>>(a, F, Fmac);
  return cudaGetLastError();
}

cudaError_t launch_fs_stress(const PassArgs<double>& a, const double* F, double* P, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + kFT - 1) / kFT), a.L);
  if (a.dim == 2) fs_stress<2><<<grid, kFT, 0, s>>>(a, F, P);
  else fs_stress<3><<<grid, kFT, 0, s>>>(a, F, P);
  return cudaGetLastError();
}

cudaError_t launch_fs_dir_tangent(const PassArgs<double>& a, const double* F, double* t, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + kFT - 1) / kFT), a.L);
  if (a.dim == 2) fs_dir_tangent<2><<<grid, kFT, 0, s>>>(a, F, t);
  else fs_dir_tangent<3><<<grid, kFT, 0, s>>>(a, F, t);
  return cudaGetLastError();
}

cudaError_t launch_fs_add(const PassArgs<double>& a, double* F, cudaStream_t s) {
  dim3 grid((unsigned)(((int64_t)a.m * a.N + kFT - 1) / kFT), a.L);
  fs_add<<<grid, kFT, 0, s>>>(a, F);
  return cudaGetLastError();
}

int fs_mean_blocks(const PassArgs<double>& a) { return (int)((a.N + kFT - 1) / kFT); }

cudaError_t launch_fs_mean(const PassArgs<double>& a, const double* F, double* part, cudaStream_t s) {
  const int nblk = fs_mean_blocks(a);
  dim3 grid(nblk, a.L);
  if (a.dim == 2) fs_mean<2><<<grid, kFT, 0, s>>>(a, F, part, nblk);
  else fs_mean<3><<<grid, kFT, 0, s>>>(a, F, part, nblk);
  return cudaGetLastError();
}

}  // namespace rve
