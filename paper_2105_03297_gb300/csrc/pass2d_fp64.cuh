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

// f = B^T C (E + B u) per node (D = 2 components), its squared norm, the
// squared norm of the summed term magnitudes (round-off scale), and the copy
// of f in the inner precision.  A block sweeps a node tile of tx (<= 256)
// nodes over ty (<= 16) rows: per pixel row it loads the displacements of the
// next node row into shared memory, computes every pixel's corner forces
// B_e^T C (E + B_e u) and their term magnitudes once (plus a one-pixel halo on
// the low side), and each node sums the four pixels it is a corner of.
// grid (n_x/tx, (n_y/ty) L), kRNT threads, residual_2d_smem() bytes.
constexpr int kRX = 256, kRY = 16, kRXE = kRX + 2, kRVX = kRX + 1, kRNT = 288;
constexpr size_t residual_2d_smem() { return sizeof(double) * (2 * 2 * kRXE + 2 * 3 * 4 * kRVX); }

__global__ void __launch_bounds__(kRNT) residual_2d(Fp64Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* un = reinterpret_cast<double*>(smem_raw);   // [2][2][kRXE]: u of two node rows
  double* lo = un + 2 * 2 * kRXE;                     // [4][kRVX]: corners dy = 0 of the current pixel row
  double* hi = lo + 4 * kRVX;                         // [2][4][kRVX]: corners dy = 1 of the current / previous row
  double* loa = hi + 2 * 4 * kRVX;                    // magnitudes, same layout
  double* hia = loa + 4 * kRVX;
  __shared__ double red[kRNT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1];
  const int tx = nx < kRX ? nx : kRX, ty = ny < kRY ? ny : kRY;
  const int nyc = ny / ty;
  const int l = blockIdx.y / nyc, yc = blockIdx.y % nyc;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  const int64_t N = a.N;
  const int x0 = blockIdx.x * tx, y0 = yc * ty;
  const int tid = threadIdx.x;
  const double* u = a.u + (int64_t)l * 2 * N;
  const double* em = a.emac + l * 3;
  const double* Eb = a.E + (int64_t)(l / a.lcs) * N;
  const double ihx = a.ih[0], ihy = a.ih[1];
  const int gx = (x0 - 1 + tid) & (nx - 1);

  auto load_row = [&](int py, double* dst) {
    if (tid < tx + 2) {
      const int64_t node = (int64_t)((y0 + py) & (ny - 1)) * nx + gx;
      dst[tid] = u[node];
      dst[kRXE + tid] = u[N + node];
    }
  };
  load_row(-1, un);
  double acc = 0.0, acca = 0.0;
  int cur = 0;
  for (int yy = -1; yy < ty; ++yy) {
    load_row(yy + 1, un + ((yy + 2) & 1) * 2 * kRXE);
    __syncthreads();
    if (tid <= tx) {
      const double* r0 = un + ((yy + 1) & 1) * 2 * kRXE;   // node row yy
      const double* r1 = un + ((yy + 2) & 1) * 2 * kRXE;   // node row yy + 1
      double u00[2], u10[2], u01[2], u11[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        u00[j] = r0[j * kRXE + tid]; u10[j] = r0[j * kRXE + tid + 1];
        u01[j] = r1[j * kRXE + tid]; u11[j] = r1[j * kRXE + tid + 1];
      }
      double hx[2][2], hy[2][2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        hx[0][j] = (u10[j] - u00[j]) * ihx; hy[0][j] = (u01[j] - u00[j]) * ihy;
        hx[1][j] = (u11[j] - u01[j]) * ihx; hy[1][j] = (u11[j] - u10[j]) * ihy;
      }
      const double e = Eb[(int64_t)((y0 + yy) & (ny - 1)) * nx + gx];
      double S[2][3];   // per element: xx, yy, xy (tensor)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        double eps[3], sig[3];
        eps[0] = em[0] + hx[q][0];
        eps[1] = em[1] + hy[q][1];
        eps[2] = em[2] + kInvSqrt2 * (hy[q][0] + hx[q][1]);
        stress_2d(eps, e, a.lam, a.mu2, sig);
        S[q][0] = sig[0]; S[q][1] = sig[1]; S[q][2] = kInvSqrt2 * sig[2];
      }
      // corner c = dx + 2 dy; element 0 on {00, 10, 01}, element 1 on {11, 01, 10}
      const double t[8][2] = {
          {-ihx * S[0][0], -ihy * S[0][2]}, {-ihx * S[0][2], -ihy * S[0][1]},   // corner 0, x / y
          {ihx * S[0][0], -ihy * S[1][2]},  {ihx * S[0][2], -ihy * S[1][1]},    // corner 1
          {ihy * S[0][2], -ihx * S[1][0]},  {ihy * S[0][1], -ihx * S[1][2]},    // corner 2
          {ihx * S[1][0], ihy * S[1][2]},   {ihx * S[1][2], ihy * S[1][1]}};    // corner 3
      double* hc = hi + cur * 4 * kRVX;
      double* hca = hia + cur * 4 * kRVX;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const double f = t[2 * c + j][0] + t[2 * c + j][1];
          const double fa = fabs(t[2 * c + j][0]) + fabs(t[2 * c + j][1]);
          if (c < 2) { lo[(2 * c + j) * kRVX + tid] = f; loa[(2 * c + j) * kRVX + tid] = fa; }
          else { hc[(2 * (c - 2) + j) * kRVX + tid] = f; hca[(2 * (c - 2) + j) * kRVX + tid] = fa; }
        }
    }
    __syncthreads();
    if (yy >= 0 && tid < tx) {
      // node (x0 + tid, y0 + yy): corner (dx, 0) of pixel (x - dx, y), corner (dx, 1) of pixel (x - dx, y - 1)
      const double* hp = hi + (cur ^ 1) * 4 * kRVX;
      const double* hpa = hia + (cur ^ 1) * 4 * kRVX;
      double fn[2] = {0, 0}, fna[2] = {0, 0};
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int i = tid + 1 - dx;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          fn[j] += lo[(2 * dx + j) * kRVX + i] + hp[(2 * dx + j) * kRVX + i];
          fna[j] += loa[(2 * dx + j) * kRVX + i] + hpa[(2 * dx + j) * kRVX + i];
        }
      }
      const int64_t node = (int64_t)(y0 + yy) * nx + x0 + tid;
      if (a.fout_f32) {
        float* fo = (float*)a.fout + (int64_t)l * 2 * N;
        fo[node] = (float)fn[0]; fo[N + node] = (float)fn[1];
      } else {
        double* fo = (double*)a.fout + (int64_t)l * 2 * N;
        fo[node] = fn[0]; fo[N + node] = fn[1];
      }
      acc += fn[0] * fn[0] + fn[1] * fn[1];
      acca += fna[0] * fna[0] + fna[1] * fna[1];
    }
    cur ^= 1;
    __syncthreads();
  }
  const double s = block_sum<kRNT>(acc, red);
  const double sa = block_sum<kRNT>(acca, red);
  const int nblk = gridDim.x * nyc;
  const int blk = blockIdx.x + gridDim.x * yc;
  double* part = a.part + (int64_t)l * a.part_stride;
  double* parta = part + a.part_stride / 2;
  if (threadIdx.x == 0) parta[blk] = sa;
  if (publish_partial(s, part, &cg->cnt_r, blk, nblk, &flag)) {
    const double tt = sum_partials<kRNT>(part, nblk, red);
    const double ta = sum_partials<kRNT>(parta, nblk, red);
    if (threadIdx.x == 0) { cg->fn2 = tt; cg->fa2 = ta; cg->cnt_r = 0; }
  }
}

inline cudaError_t launch_residual_2d(const Fp64Args& a, cudaStream_t s) {
  const int tx = a.n[0] < kRX ? a.n[0] : kRX, ty = a.n[1] < kRY ? a.n[1] : kRY;
  const size_t sm = residual_2d_smem();
  static DeviceOnce attr;
  attr.run(current_device(), [&] { cudaFuncSetAttribute(residual_2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); });
  dim3 grid(a.n[0] / tx, (a.n[1] / ty) * a.L);
  residual_2d<<<grid, kRNT, sm, s>>>(a);
  return cudaGetLastError();
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
