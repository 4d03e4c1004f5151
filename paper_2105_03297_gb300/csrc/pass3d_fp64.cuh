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

// f = B^T C (E + B u) per node, its squared norm, the squared norm of the
// summed term magnitudes (round-off scale) and the copy of f in the inner
// precision.  A block sweeps a node tile of (at most) 32 x 8 nodes through a
// z-chunk of (at most) 16 planes: per voxel plane it loads the displacements
// of the next node plane into shared memory, computes every voxel's corner
// forces and term magnitudes once (plus a one-voxel halo on the low side), and
// each node sums the 8 voxels it is a corner of.  grid (n_x/tx, n_y/ty,
// (n_z/tz) L), kR3NT threads, residual_3d_smem() bytes.
constexpr int kR3X = 32, kR3Y = 8, kR3Z = 16;
constexpr int kR3NES = (kR3X + 2) * (kR3Y + 2);   // 340 nodes (both halos in x and y)
constexpr int kR3VS = (kR3X + 1) * (kR3Y + 1);    // 297 voxels (low halo)
constexpr int kR3NT = 352;
static_assert(kR3NT >= kR3NES && kR3NT >= kR3VS, "one thread per node and per voxel of the tile");
constexpr size_t residual_3d_smem() { return sizeof(double) * (2 * 3 * kR3NES + 2 * 3 * 12 * kR3VS); }

__global__ void __launch_bounds__(kR3NT, 1) residual_3d(Fp64Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* un = reinterpret_cast<double*>(smem_raw);   // [2][3][kR3NES]: u of two node planes
  double* lo = un + 2 * 3 * kR3NES;                   // [12][kR3VS]: corners dz = 0, current voxel plane
  double* hi = lo + 12 * kR3VS;                       // [2][12][kR3VS]: corners dz = 1, current / previous
  double* loa = hi + 2 * 12 * kR3VS;                  // magnitudes, same layout
  double* hia = loa + 12 * kR3VS;
  __shared__ double red[kR3NT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tx = nx < kR3X ? nx : kR3X, ty = ny < kR3Y ? ny : kR3Y, tz = nz < kR3Z ? nz : kR3Z;
  const int etx = tx + 2, nnode = (tx + 2) * (ty + 2);
  const int vtx = tx + 1, nvox = (tx + 1) * (ty + 1);
  const int nzc = nz / tz;
  const int l = blockIdx.z / nzc, zc = blockIdx.z % nzc;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  const int64_t N = a.N;
  const int x0 = blockIdx.x * tx, y0 = blockIdx.y * ty, z0 = zc * tz;
  const int tid = threadIdx.x;
  const double* u = a.u + (int64_t)l * 3 * N;
  const double* em = a.emac + l * 6;
  const double* Eb = a.E + (int64_t)(l / a.lcs) * N;
  const int64_t plane = (int64_t)nx * ny;
  // node of the extended node tile (load) and voxel of the extended voxel tile
  const int nex = tid % etx, ney = tid / etx;
  const int64_t node_xy = (int64_t)((y0 - 1 + ney) & (ny - 1)) * nx + ((x0 - 1 + nex) & (nx - 1));
  const int vex = tid % vtx, vey = tid / vtx;
  const int64_t vox_xy = (int64_t)((y0 - 1 + vey) & (ny - 1)) * nx + ((x0 - 1 + vex) & (nx - 1));

  auto load_plane = [&](int pz, double* dst) {
    if (tid < nnode) {
      const int64_t node = (int64_t)((z0 + pz) & (nz - 1)) * plane + node_xy;
#pragma unroll
      for (int j = 0; j < 3; ++j) dst[j * kR3NES + tid] = u[j * N + node];
    }
  };
  load_plane(-1, un);
  double acc = 0.0, acca = 0.0;
  int cur = 0;
  for (int zz = -1; zz < tz; ++zz) {
    load_plane(zz + 1, un + ((zz + 2) & 1) * 3 * kR3NES);
    __syncthreads();
    if (tid < nvox) {
      const double* p0 = un + ((zz + 1) & 1) * 3 * kR3NES;   // node plane zz
      const double* p1 = un + ((zz + 2) & 1) * 3 * kR3NES;   // node plane zz + 1
      double uc[8][3];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int i = (vey + ((c >> 1) & 1)) * etx + vex + (c & 1);
        const double* src = (c & 4) ? p1 : p0;
#pragma unroll
        for (int j = 0; j < 3; ++j) uc[c][j] = src[j * kR3NES + i];
      }
      const double e = Eb[(int64_t)((z0 + zz) & (nz - 1)) * plane + vox_xy];
      double f[8][3], fa[8][3];
#pragma unroll
      for (int c = 0; c < 8; ++c) f[c][0] = f[c][1] = f[c][2] = fa[c][0] = fa[c][1] = fa[c][2] = 0.0;
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
        const int v1 = 1 << pa, v2 = v1 | (1 << pb);
        double H[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          H[pa][j] = (uc[v1][j] - uc[0][j]) * a.ih[pa];
          H[pb][j] = (uc[v2][j] - uc[v1][j]) * a.ih[pb];
          H[pc][j] = (uc[7][j] - uc[v2][j]) * a.ih[pc];
        }
        double eps[6], sg[6];
        eps[0] = em[0] + H[0][0];
        eps[1] = em[1] + H[1][1];
        eps[2] = em[2] + H[2][2];
        eps[3] = em[3] + kInvSqrt2 * (H[1][2] + H[2][1]);
        eps[4] = em[4] + kInvSqrt2 * (H[0][2] + H[2][0]);
        eps[5] = em[5] + kInvSqrt2 * (H[0][1] + H[1][0]);
        stress_3d(eps, e, a.lam, a.mu2, sg);
        double S[3][3];
        S[0][0] = sg[0]; S[1][1] = sg[1]; S[2][2] = sg[2];
        S[1][2] = S[2][1] = kInvSqrt2 * sg[3];
        S[0][2] = S[2][0] = kInvSqrt2 * sg[4];
        S[0][1] = S[1][0] = kInvSqrt2 * sg[5];
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
      double* hc = hi + cur * 12 * kR3VS;
      double* hca = hia + cur * 12 * kR3VS;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          lo[(c * 3 + j) * kR3VS + tid] = f[c][j];
          loa[(c * 3 + j) * kR3VS + tid] = fa[c][j];
          hc[(c * 3 + j) * kR3VS + tid] = f[c + 4][j];
          hca[(c * 3 + j) * kR3VS + tid] = fa[c + 4][j];
        }
    }
    __syncthreads();
    if (zz >= 0 && tid < tx * ty) {
      // node (x0 + lx, y0 + ly, z0 + zz): corner (dx, dy, dz) of voxel (x - dx, y - dy, z - dz)
      const int lx = tid % tx, ly = tid / tx;
      const double* hp = hi + (cur ^ 1) * 12 * kR3VS;
      const double* hpa = hia + (cur ^ 1) * 12 * kR3VS;
      double fn[3] = {0, 0, 0}, fna[3] = {0, 0, 0};
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int i = (ly + 1 - dy) * vtx + (lx + 1 - dx);
          const int c = dx + 2 * dy;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            fn[j] += lo[(c * 3 + j) * kR3VS + i] + hp[(c * 3 + j) * kR3VS + i];
            fna[j] += loa[(c * 3 + j) * kR3VS + i] + hpa[(c * 3 + j) * kR3VS + i];
          }
        }
      const int64_t node = ((int64_t)(z0 + zz) * ny + (y0 + ly)) * nx + x0 + lx;
      if (a.fout_f32) {
        float* fo = (float*)a.fout + (int64_t)l * 3 * N;
#pragma unroll
        for (int j = 0; j < 3; ++j) fo[j * N + node] = (float)fn[j];
      } else {
        double* fo = (double*)a.fout + (int64_t)l * 3 * N;
#pragma unroll
        for (int j = 0; j < 3; ++j) fo[j * N + node] = fn[j];
      }
      acc += fn[0] * fn[0] + fn[1] * fn[1] + fn[2] * fn[2];
      acca += fna[0] * fna[0] + fna[1] * fna[1] + fna[2] * fna[2];
    }
    cur ^= 1;
    __syncthreads();
  }
  const double s = block_sum<kR3NT>(acc, red);
  const double sa = block_sum<kR3NT>(acca, red);
  const int nblk = gridDim.x * gridDim.y * nzc;
  const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc);
  double* part = a.part + (int64_t)l * a.part_stride;
  double* parta = part + a.part_stride / 2;
  if (threadIdx.x == 0) parta[blk] = sa;
  if (publish_partial(s, part, &cg->cnt_r, blk, nblk, &flag)) {
    const double t = sum_partials<kR3NT>(part, nblk, red);
    const double ta = sum_partials<kR3NT>(parta, nblk, red);
    if (threadIdx.x == 0) { cg->fn2 = t; cg->fa2 = ta; cg->cnt_r = 0; }
  }
}

inline cudaError_t launch_residual_3d(const Fp64Args& a, cudaStream_t s) {
  const int tx = a.n[0] < kR3X ? a.n[0] : kR3X, ty = a.n[1] < kR3Y ? a.n[1] : kR3Y;
  const int tz = a.n[2] < kR3Z ? a.n[2] : kR3Z;
  const size_t sm = residual_3d_smem();
  static DeviceOnce attr;
  attr.run(current_device(), [&] { cudaFuncSetAttribute(residual_3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); });
  dim3 grid(a.n[0] / tx, a.n[1] / ty, (a.n[2] / tz) * a.L);
  residual_3d<<<grid, kR3NT, sm, s>>>(a);
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
