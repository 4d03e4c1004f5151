// 3D FP64 real-space kernels (no FFT): nodal residual f = B^T C (E + B u),
// homogenisation, strain field and adjoint gradient, on the six Kuhn
// tetrahedra {0, e_a, e_a+e_b, e_a+e_b+e_c} of every voxel.
#pragma once
#include "pass3d.cuh"

namespace rve {

// Mandel strains of the six tetrahedra of voxel (vx, vy, vz) for the nodal
// displacement u ([3][N]) and macroscopic strain em.
__device__ __forceinline__ void strain_3d(const double* u, int64_t N, const int* n, int vx, int vy, int vz,
                                          const double* em, const double* ih, double eps[6][6]) {
  double uc[8][3];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int x = (vx + (c & 1)) & (n[0] - 1);
    const int y = (vy + ((c >> 1) & 1)) & (n[1] - 1);
    const int z = (vz + ((c >> 2) & 1)) & (n[2] - 1);
    const int64_t i = ((int64_t)z * n[1] + y) * n[0] + x;
#pragma unroll
    for (int j = 0; j < 3; ++j) uc[c][j] = u[j * N + i];
  }
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
    const int v1 = 1 << pa, v2 = v1 | (1 << pb);
    double H[3][3];  // H[i][j] = d u_j / d x_i
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      H[pa][j] = (uc[v1][j] - uc[0][j]) * ih[pa];
      H[pb][j] = (uc[v2][j] - uc[v1][j]) * ih[pb];
      H[pc][j] = (uc[7][j] - uc[v2][j]) * ih[pc];
    }
    eps[t][0] = em[0] + H[0][0];
    eps[t][1] = em[1] + H[1][1];
    eps[t][2] = em[2] + H[2][2];
    eps[t][3] = em[3] + kInvSqrt2 * (H[1][2] + H[2][1]);
    eps[t][4] = em[4] + kInvSqrt2 * (H[0][2] + H[2][0]);
    eps[t][5] = em[5] + kInvSqrt2 * (H[0][1] + H[1][0]);
  }
}

__device__ __forceinline__ void stress_3d(const double* eps, double e, double lam, double mu2, double* sig) {
  const double tr = lam * (eps[0] + eps[1] + eps[2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) sig[j] = e * (tr + mu2 * eps[j]);
#pragma unroll
  for (int j = 3; j < 6; ++j) sig[j] = e * mu2 * eps[j];
}

constexpr int kRTX = 16, kRTY = 4, kRTZ = 4;
constexpr int kRVox = (kRTX + 1) * (kRTY + 1) * (kRTZ + 1);

// Tiled gather: each block computes the corner forces of the voxels of its
// node tile plus a one-voxel halo on the low side (shared memory), then every
// node sums the contributions of the 8 voxels it is a corner of.
// grid (n_x/16, n_y/4, (n_z/4) * L), 256 threads.
__global__ void __launch_bounds__(256) residual_3d(Fp64Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* contrib = reinterpret_cast<double*>(smem_raw);  // [kRVox][8][3]
  double* cabs = contrib + kRVox * 24;                    // [kRVox][8][3] magnitudes
  __shared__ double red[8];
  __shared__ int flag;
  const int nzt = a.n[2] / kRTZ;
  const int l = blockIdx.z / nzt, tz = blockIdx.z % nzt;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  const int x0 = blockIdx.x * kRTX, y0 = blockIdx.y * kRTY, z0 = tz * kRTZ;
  const double* u = a.u + (int64_t)l * 3 * a.N;
  const double* em = a.emac + l * 6;
  for (int i = threadIdx.x; i < kRVox; i += blockDim.x) {
    const int ex = i % (kRTX + 1), ey = (i / (kRTX + 1)) % (kRTY + 1), ez = i / ((kRTX + 1) * (kRTY + 1));
    const int vx = (x0 - 1 + ex) & (a.n[0] - 1);
    const int vy = (y0 - 1 + ey) & (a.n[1] - 1);
    const int vz = (z0 - 1 + ez) & (a.n[2] - 1);
    double eps[6][6];
    strain_3d(u, a.N, a.n, vx, vy, vz, em, a.ih, eps);
    const double e = a.E[(int64_t)(l / a.lcs) * a.N + ((int64_t)vz * a.n[1] + vy) * a.n[0] + vx];
    double f[8][3], fa[8][3];
#pragma unroll
    for (int c = 0; c < 8; ++c) f[c][0] = f[c][1] = f[c][2] = fa[c][0] = fa[c][1] = fa[c][2] = 0.0;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      double s[6];
      stress_3d(eps[t], e, a.lam, a.mu2, s);
      double S[3][3];
      S[0][0] = s[0]; S[1][1] = s[1]; S[2][2] = s[2];
      S[1][2] = S[2][1] = kInvSqrt2 * s[3];
      S[0][2] = S[2][0] = kInvSqrt2 * s[4];
      S[0][1] = S[1][0] = kInvSqrt2 * s[5];
      const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
      const int v1 = 1 << pa, v2 = v1 | (1 << pb);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double Pa = a.ih[pa] * S[pa][j], Pb = a.ih[pb] * S[pb][j], Pc = a.ih[pc] * S[pc][j];
        f[0][j] -= Pa;
        f[v1][j] += Pa - Pb;
        f[v2][j] += Pb - Pc;
        f[7][j] += Pc;
        fa[0][j] += fabs(Pa);
        fa[v1][j] += fabs(Pa) + fabs(Pb);
        fa[v2][j] += fabs(Pb) + fabs(Pc);
        fa[7][j] += fabs(Pc);
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        contrib[(i * 8 + c) * 3 + j] = f[c][j];
        cabs[(i * 8 + c) * 3 + j] = fa[c][j];
      }
  }
  __syncthreads();
  const int lx = threadIdx.x % kRTX, ly = (threadIdx.x / kRTX) % kRTY, lz = threadIdx.x / (kRTX * kRTY);
  double fn[3] = {0, 0, 0}, fna[3] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    const int ex = lx + 1 - dx, ey = ly + 1 - dy, ez = lz + 1 - dz;
    const int i = (ez * (kRTY + 1) + ey) * (kRTX + 1) + ex;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      fn[j] += contrib[(i * 8 + c) * 3 + j];
      fna[j] += cabs[(i * 8 + c) * 3 + j];
    }
  }
  const int64_t node = ((int64_t)(z0 + lz) * a.n[1] + (y0 + ly)) * a.n[0] + x0 + lx;
  if (a.fout_f32) {
    float* fo = (float*)a.fout + (int64_t)l * 3 * a.N;
#pragma unroll
    for (int j = 0; j < 3; ++j) fo[j * a.N + node] = (float)fn[j];
  } else {
    double* fo = (double*)a.fout + (int64_t)l * 3 * a.N;
#pragma unroll
    for (int j = 0; j < 3; ++j) fo[j * a.N + node] = fn[j];
  }
  const double acc = fn[0] * fn[0] + fn[1] * fn[1] + fn[2] * fn[2];
  const double acca = fna[0] * fna[0] + fna[1] * fna[1] + fna[2] * fna[2];
  const double s = block_sum<256>(acc, red);
  const double sa = block_sum<256>(acca, red);
  const int nblk = gridDim.x * gridDim.y * nzt;
  const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * tz);
  double* part = a.part + (int64_t)l * a.part_stride;
  double* parta = part + a.part_stride / 2;
  if (threadIdx.x == 0) parta[blk] = sa;
  if (publish_partial(s, part, &cg->cnt_r, blk, nblk, &flag)) {
    const double t = sum_partials<256>(part, nblk, red);
    const double ta = sum_partials<256>(parta, nblk, red);
    if (threadIdx.x == 0) { cg->fn2 = t; cg->fa2 = ta; cg->cnt_r = 0; }
  }
}

inline cudaError_t launch_residual_3d(const Fp64Args& a, cudaStream_t s) {
  const size_t sm = sizeof(double) * kRVox * 48;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(residual_3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.n[0] / kRTX, a.n[1] / kRTY, (a.n[2] / kRTZ) * a.L);
  residual_3d<<<grid, 256, sm, s>>>(a);
  return cudaGetLastError();
}

template <int NT>
__global__ void __launch_bounds__(NT) homogenise_3d(Fp64Args a, double* part, int nblk) {
  __shared__ double red[NT / 32];
  const int l = blockIdx.y;
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (v < a.N) {
    const int x = (int)(v % a.n[0]), y = (int)((v / a.n[0]) % a.n[1]), z = (int)(v / ((int64_t)a.n[0] * a.n[1]));
    double eps[6][6], sig[6];
    strain_3d(a.u + (int64_t)l * 3 * a.N, a.N, a.n, x, y, z, a.emac + l * 6, a.ih, eps);
    const double e = a.E[(int64_t)(l / a.lcs) * a.N + v];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      stress_3d(eps[t], e, a.lam, a.mu2, sig);
#pragma unroll
      for (int s = 0; s < 6; ++s) acc[s] += sig[s];
    }
  }
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const double t = block_sum<NT>(acc[s], red);
    if (threadIdx.x == 0) part[((int64_t)l * 6 + s) * nblk + blockIdx.x] = t;
  }
}

// Block partial sums of eps_a : C : eps_b (pairs a <= b): part[p * nblk + blk].
template <int NT>
__global__ void __launch_bounds__(NT) energy_3d(Fp64Args a, double* part, int nblk) {
  __shared__ double red[NT / 32];
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  const bool ok = v < a.N;
  const int x = ok ? (int)(v % a.n[0]) : 0, y = ok ? (int)((v / a.n[0]) % a.n[1]) : 0;
  const int z = ok ? (int)(v / ((int64_t)a.n[0] * a.n[1])) : 0;
  int p = 0;
  for (int lb = 0; lb < a.L; ++lb) {
    const double e = ok ? a.E[(int64_t)(lb / a.lcs) * a.N + v] : 0.0;
    double sb[6][6];
    if (ok) {
      double eb[6][6];
      strain_3d(a.u + (int64_t)lb * 3 * a.N, a.N, a.n, x, y, z, a.emac + lb * 6, a.ih, eb);
      for (int t = 0; t < 6; ++t) stress_3d(eb[t], e, a.lam, a.mu2, sb[t]);
    }
    for (int la = 0; la <= lb; ++la, ++p) {
      double acc = 0.0;
      if (ok) {
        double ea[6][6];
        strain_3d(a.u + (int64_t)la * 3 * a.N, a.N, a.n, x, y, z, a.emac + la * 6, a.ih, ea);
        for (int t = 0; t < 6; ++t)
          for (int s = 0; s < 6; ++s) acc += ea[t][s] * sb[t][s];
      }
      const double bs = block_sum<NT>(acc, red);
      if (threadIdx.x == 0) part[(int64_t)p * nblk + blockIdx.x] = bs;
    }
  }
}

__global__ void strain_field_3d(Fp64Args a, int l, double* out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.N) return;
  const int x = (int)(v % a.n[0]), y = (int)((v / a.n[0]) % a.n[1]), z = (int)(v / ((int64_t)a.n[0] * a.n[1]));
  double eps[6][6];
  strain_3d(a.u + (int64_t)l * 3 * a.N, a.N, a.n, x, y, z, a.emac + l * 6, a.ih, eps);
#pragma unroll
  for (int t = 0; t < 6; ++t)
#pragma unroll
    for (int s = 0; s < 6; ++s) out[(t * 6 + s) * a.N + v] = eps[t][s];
}

// grad[v] = scale * sum_a sum_t (e_a + B lam_a)_t : Cbar : (sum_l W[a][l] (E_l + B u_l))_t
__global__ void adjoint_grad_3d(Fp64Args a, const double* uadj, const double* W, const int* has_adj,
                                double scale, double* grad) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.N) return;
  const int x = (int)(v % a.n[0]), y = (int)((v / a.n[0]) % a.n[1]), z = (int)(v / ((int64_t)a.n[0] * a.n[1]));
  double g = 0.0;
  for (int ai = 0; ai < 6; ++ai) {
    if (!has_adj[ai]) continue;
    double wsum[6][6];
    for (int t = 0; t < 6; ++t)
      for (int s = 0; s < 6; ++s) wsum[t][s] = 0.0;
    for (int l = 0; l < a.L; ++l) {
      const double w = W[ai * a.L + l];
      if (w == 0.0) continue;
      double eps[6][6];
      strain_3d(a.u + (int64_t)l * 3 * a.N, a.N, a.n, x, y, z, a.emac + l * 6, a.ih, eps);
      for (int t = 0; t < 6; ++t)
        for (int s = 0; s < 6; ++s) wsum[t][s] += w * eps[t][s];
    }
    double ea[6] = {0, 0, 0, 0, 0, 0};
    ea[ai] = 1.0;
    double le[6][6];
    strain_3d(uadj + (int64_t)ai * 3 * a.N, a.N, a.n, x, y, z, ea, a.ih, le);
    for (int t = 0; t < 6; ++t) {
      double cs[6];
      stress_3d(wsum[t], 1.0, a.lam, a.mu2, cs);
      for (int s = 0; s < 6; ++s) g += le[t][s] * cs[s];
    }
  }
  grad[v] = g * scale;
}

}  // namespace rve
