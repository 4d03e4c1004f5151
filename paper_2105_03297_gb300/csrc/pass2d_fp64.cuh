// 2D FP64 real-space kernels (no FFT): nodal residual f = B^T C (E + B u),
// homogenisation, strain field and adjoint gradient on the two triangles of
// every pixel.
#pragma once
#include "pass2d.cuh"

// ====================================================================
// FP64 real-space kernels (no FFT): nodal residual, homogenisation, adjoint.
// ====================================================================
namespace rve {



// Mandel strains E + sym(grad u) of the two triangles of voxel (vx, vy).
__device__ __forceinline__ void strain_2d(const double* u, int64_t N, int nx, int ny, int vx, int vy,
                                          const double* em, double ihx, double ihy, double eps[2][3]) {
  const int x1 = (vx + 1) & (nx - 1), y1 = (vy + 1) & (ny - 1);
  const int64_t i00 = (int64_t)vy * nx + vx, i10 = (int64_t)vy * nx + x1;
  const int64_t i01 = (int64_t)y1 * nx + vx, i11 = (int64_t)y1 * nx + x1;
  double u00[2], u10[2], u01[2], u11[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    u00[j] = u[j * N + i00]; u10[j] = u[j * N + i10];
    u01[j] = u[j * N + i01]; u11[j] = u[j * N + i11];
  }
  double hx[2][2], hy[2][2];  // [element][component]: d u_j / dx, d u_j / dy
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    hx[0][j] = (u10[j] - u00[j]) * ihx; hy[0][j] = (u01[j] - u00[j]) * ihy;
    hx[1][j] = (u11[j] - u01[j]) * ihx; hy[1][j] = (u11[j] - u10[j]) * ihy;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    eps[q][0] = em[0] + hx[q][0];
    eps[q][1] = em[1] + hy[q][1];
    eps[q][2] = em[2] + kInvSqrt2 * (hy[q][0] + hx[q][1]);   // Mandel: sqrt2 * (du_x/dy + du_y/dx)/2
  }
}

// sigma (Mandel) = e * Cbar eps
__device__ __forceinline__ void stress_2d(const double* eps, double e, double lam, double mu2, double* sig) {
  const double tr = lam * (eps[0] + eps[1]);
  sig[0] = e * (tr + mu2 * eps[0]);
  sig[1] = e * (tr + mu2 * eps[1]);
  sig[2] = e * mu2 * eps[2];
}

// f = B^T C (E + B u) per node (D = 2 components), its squared norm, and the
// copy of f in the inner precision.  grid (ceil(N/NT), L).
template <int NT>
__global__ void __launch_bounds__(NT) residual_2d(Fp64Args a) {
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int l = blockIdx.y;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  const int64_t n = (int64_t)blockIdx.x * NT + threadIdx.x;
  double acc = 0.0, acca = 0.0;
  if (n < a.N) {
    const int x = (int)(n % a.n[0]), y = (int)(n / a.n[0]);
    const double* u = a.u + (int64_t)l * 2 * a.N;
    const double* em = a.emac + l * 3;
    double fx = 0.0, fy = 0.0, ax = 0.0, ay = 0.0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int vx = (x - dx) & (a.n[0] - 1), vy = (y - dy) & (a.n[1] - 1);
        double eps[2][3], sig[3];
        strain_2d(u, a.N, a.n[0], a.n[1], vx, vy, em, a.ih[0], a.ih[1], eps);
        const double e = a.E[(int64_t)(l / a.lcs) * a.N + (int64_t)vy * a.n[0] + vx];
        // shape-function gradients of this node in element 0 / element 1
        double g0x = 0, g0y = 0, g1x = 0, g1y = 0;
        bool in0 = false, in1 = false;
        if (dx == 0 && dy == 0) { in0 = true; g0x = -a.ih[0]; g0y = -a.ih[1]; }
        if (dx == 1 && dy == 0) { in0 = true; g0x = a.ih[0]; in1 = true; g1y = -a.ih[1]; }
        if (dx == 0 && dy == 1) { in0 = true; g0y = a.ih[1]; in1 = true; g1x = -a.ih[0]; }
        if (dx == 1 && dy == 1) { in1 = true; g1x = a.ih[0]; g1y = a.ih[1]; }
        if (in0) {
          stress_2d(eps[0], e, a.lam, a.mu2, sig);
          const double sxy = kInvSqrt2 * sig[2];
          fx += g0x * sig[0] + g0y * sxy;
          fy += g0x * sxy + g0y * sig[1];
          ax += fabs(g0x * sig[0]) + fabs(g0y * sxy);
          ay += fabs(g0x * sxy) + fabs(g0y * sig[1]);
        }
        if (in1) {
          stress_2d(eps[1], e, a.lam, a.mu2, sig);
          const double sxy = kInvSqrt2 * sig[2];
          fx += g1x * sig[0] + g1y * sxy;
          fy += g1x * sxy + g1y * sig[1];
          ax += fabs(g1x * sig[0]) + fabs(g1y * sxy);
          ay += fabs(g1x * sxy) + fabs(g1y * sig[1]);
        }
      }
    acc = fx * fx + fy * fy;
    acca = ax * ax + ay * ay;
    if (a.fout_f32) {
      float* f = (float*)a.fout + (int64_t)l * 2 * a.N;
      f[n] = (float)fx; f[a.N + n] = (float)fy;
    } else {
      double* f = (double*)a.fout + (int64_t)l * 2 * a.N;
      f[n] = fx; f[a.N + n] = fy;
    }
  }
  const double s = block_sum<NT>(acc, red);
  const double sa = block_sum<NT>(acca, red);
  double* part = a.part + (int64_t)l * a.part_stride;
  double* parta = part + a.part_stride / 2;
  if (threadIdx.x == 0) parta[blockIdx.x] = sa;
  if (publish_partial(s, part, &cg->cnt_r, blockIdx.x, gridDim.x, &flag)) {
    const double t = sum_partials<NT>(part, gridDim.x, red);
    const double ta = sum_partials<NT>(parta, gridDim.x, red);
    if (threadIdx.x == 0) { cg->fn2 = t; cg->fa2 = ta; cg->cnt_r = 0; }
  }
}

// Block partial sums of the element stresses: part[(l*3 + s) * nblk + blk].
// grid (ceil(N/NT), L).
template <int NT>
__global__ void __launch_bounds__(NT) homogenise_2d(Fp64Args a, double* part, int nblk) {
  __shared__ double red[NT / 32];
  const int l = blockIdx.y;
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  double acc[3] = {0, 0, 0};
  if (v < a.N) {
    const int x = (int)(v % a.n[0]), y = (int)(v / a.n[0]);
    double eps[2][3], sig[3];
    strain_2d(a.u + (int64_t)l * 2 * a.N, a.N, a.n[0], a.n[1], x, y, a.emac + l * 3, a.ih[0], a.ih[1], eps);
    const double e = a.E[(int64_t)(l / a.lcs) * a.N + v];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      stress_2d(eps[q], e, a.lam, a.mu2, sig);
      acc[0] += sig[0]; acc[1] += sig[1]; acc[2] += sig[2];
    }
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const double t = block_sum<NT>(acc[s], red);
    if (threadIdx.x == 0) part[((int64_t)l * 3 + s) * nblk + blockIdx.x] = t;
  }
}

// Block partial sums of eps_a : C : eps_b over the elements, for the pairs
// a <= b of the L solved load cases: part[p * nblk + blk].
template <int NT>
__global__ void __launch_bounds__(NT) energy_2d(Fp64Args a, double* part, int nblk) {
  __shared__ double red[NT / 32];
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  const bool ok = v < a.N;
  const int x = ok ? (int)(v % a.n[0]) : 0, y = ok ? (int)(v / a.n[0]) : 0;
  int p = 0;
  for (int lb = 0; lb < a.L; ++lb) {
    const double e = ok ? a.E[(int64_t)(lb / a.lcs) * a.N + v] : 0.0;
    double sb[2][3] = {{0, 0, 0}, {0, 0, 0}};
    if (ok) {
      double eb[2][3];
      strain_2d(a.u + (int64_t)lb * 2 * a.N, a.N, a.n[0], a.n[1], x, y, a.emac + lb * 3, a.ih[0], a.ih[1], eb);
      for (int q = 0; q < 2; ++q) stress_2d(eb[q], e, a.lam, a.mu2, sb[q]);
    }
    for (int la = 0; la <= lb; ++la, ++p) {
      double t = 0.0;
      if (ok) {
        double ea[2][3];
        strain_2d(a.u + (int64_t)la * 2 * a.N, a.N, a.n[0], a.n[1], x, y, a.emac + la * 3, a.ih[0], a.ih[1], ea);
        for (int q = 0; q < 2; ++q)
          for (int s = 0; s < 3; ++s) t += ea[q][s] * sb[q][s];
      }
      const double bs = block_sum<NT>(t, red);
      if (threadIdx.x == 0) part[(int64_t)p * nblk + blockIdx.x] = bs;
    }
  }
}

// Total strain field eps[m][N] (FP64) of load case l.
__global__ void strain_field_2d(Fp64Args a, int l, double* out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.N) return;
  const int x = (int)(v % a.n[0]), y = (int)(v / a.n[0]);
  double eps[2][3];
  strain_2d(a.u + (int64_t)l * 2 * a.N, a.N, a.n[0], a.n[1], x, y, a.emac + l * 3, a.ih[0], a.ih[1], eps);
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int s = 0; s < 3; ++s) out[(q * 3 + s) * a.N + v] = eps[q][s];
}

// grad[v] = scale * sum_q sum_{a,l} W[a][l] (e_a + B lam_a)_q : Cbar : (E_l + B u_l)_q
// uadj: [3][2][N] adjoint displacements for unit strains (rows with has_adj[a]).
__global__ void adjoint_grad_2d(Fp64Args a, const double* uadj, const double* W /*[3][L]*/,
                                const int* has_adj, double scale, double* grad) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.N) return;
  const int x = (int)(v % a.n[0]), y = (int)(v / a.n[0]);
  double csig[6][2][3];  // Cbar eps_l per element (unit modulus)
  for (int l = 0; l < a.L; ++l) {
    double eps[2][3];
    strain_2d(a.u + (int64_t)l * 2 * a.N, a.N, a.n[0], a.n[1], x, y, a.emac + l * 3, a.ih[0], a.ih[1], eps);
    for (int q = 0; q < 2; ++q) stress_2d(eps[q], 1.0, a.lam, a.mu2, csig[l][q]);
  }
  double g = 0.0;
  for (int ai = 0; ai < 3; ++ai) {
    if (!has_adj[ai]) continue;
    double ea[3] = {0, 0, 0};
    ea[ai] = 1.0;
    double lam_eps[2][3];
    strain_2d(uadj + (int64_t)ai * 2 * a.N, a.N, a.n[0], a.n[1], x, y, ea, a.ih[0], a.ih[1], lam_eps);
    for (int l = 0; l < a.L; ++l) {
      const double w = W[ai * a.L + l];
      if (w == 0.0) continue;
      double t = 0.0;
      for (int q = 0; q < 2; ++q)
        for (int s = 0; s < 3; ++s) t += lam_eps[q][s] * csig[l][q][s];
      g += w * t;
    }
  }
  grad[v] = g * scale;
}

}  // namespace rve
