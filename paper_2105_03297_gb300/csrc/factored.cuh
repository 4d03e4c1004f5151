// Factored nodal form of the projected operator (same operator, other order):
//   G C p = B (B^H B)^-1 B^H F[C p] = B_r K^-1 B_r^T (C p),
// with B_r the real-space strain stencil of the elements, B_r^T its adjoint
// (nodal forces) and K^-1 = F^-1 (B^H B)^-1 F a 3x3 (2x2) Fourier multiplier
// on nodal fields.  Only the D nodal components go through FFTs.
//
//   force stencil  x += alpha_prev p_old, p = r + beta p_old, sigma = C p,
//                  <p, sigma> -> alpha, f = B_r^T sigma (D per node)
//   FFT passes     f -> w = F^-1 (B^H B)^-1 F f   (existing passes, D components)
//   strain update  q = B_r w, r -= alpha q, <r, r> -> beta, convergence
//
// B_r^T gathers, for every node, the forces of the elements of the 2^D voxels
// it is a corner of.  The force stencil sweeps a tile of nodes plane by plane
// (3D: z-planes; 2D: y-rows), keeps the corner forces of the current and the
// previous voxel plane in shared memory, and recomputes the stresses of a
// one-voxel halo on the low side (those voxels' p is not written: their owner
// block writes it).
#pragma once
#include "pass3d.cuh"

namespace rve {

// ----------------------------------------------------------------- 3D
// Node tile (at most kFX x kFY x kFZ; smaller grids use the whole axis) and
// the voxel tile with its low-side halo.  Corner forces live in shared memory
// as structure of arrays [12][kFVS] (corner-component major) so that
// consecutive voxels hit consecutive banks.
constexpr int kFX = 32, kFY = 8, kFZ = 16;
constexpr int kFVX = kFX + 1, kFVY = kFY + 1, kFVS = kFVX * kFVY;
constexpr int kFNT = 320;                                     // >= kFVS = 297
static_assert(kFNT >= kFVS, "one thread per voxel of the extended tile");

template <typename T> constexpr size_t force_smem_3d() { return sizeof(T) * 36 * kFVS; }

// Stresses (tensor rows, unit-free) of the six tetrahedra of one voxel from
// its p (36 Mandel components at stride N) and the corner forces
// B_e^T sigma_e (8 corners x 3): corner c = dx + 2 dy + 4 dz.
template <typename T>
__device__ __forceinline__ void voxel_corner_forces_3d(const T* pv /*[36]*/, T e, T lam, T mu2, const T* ih,
                                                       T f[8][3]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) f[c][0] = f[c][1] = f[c][2] = 0;
  const T r2 = (T)kInvSqrt2;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const T* p = pv + 6 * t;
    const T tr = lam * (p[0] + p[1] + p[2]);
    T S[3][3];
    S[0][0] = e * (tr + mu2 * p[0]);
    S[1][1] = e * (tr + mu2 * p[1]);
    S[2][2] = e * (tr + mu2 * p[2]);
    S[1][2] = S[2][1] = e * mu2 * p[3] * r2;
    S[0][2] = S[2][0] = e * mu2 * p[4] * r2;
    S[0][1] = S[1][0] = e * mu2 * p[5] * r2;
    const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
    const int v1 = 1 << pa, v2 = v1 | (1 << pb);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T Pa = ih[pa] * S[pa][j], Pb = ih[pb] * S[pb][j], Pc = ih[pc] * S[pc][j];
      f[0][j] -= Pa;
      f[v1][j] += Pa - Pb;
      f[v2][j] += Pb - Pc;
      f[7][j] += Pc;
    }
  }
}

// CG direction update and nodal forces of the material response:
//   x += alpha_prev p_old (owned voxels), p = r + beta p_old -> p_new,
//   f = B_r^T (C p), <p, C p> -> alpha (last block).
// p_old and p_new are different buffers (halo voxels read p_old of voxels
// their owner block rewrites).  grid (n_x/tx, n_y/ty, (n_z/tz) L), kFNT
// threads, force_smem_3d<T>() bytes of dynamic shared memory.
template <typename T>
__global__ void __launch_bounds__(kFNT, sizeof(T) == 4 ? 2 : 1)
    force_stencil_3d(PassArgs<T> a, const T* __restrict__ r, const T* __restrict__ pold, T* __restrict__ pnew,
                     T* __restrict__ x, T* __restrict__ f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* lo = reinterpret_cast<T*>(smem_raw);   // [12][kFVS]: corners dz = 0 of the current voxel plane
  T* hi = lo + 12 * kFVS;                   // [2][12][kFVS]: corners dz = 1 of the current / previous plane
  __shared__ double red[kFNT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tx = nx < kFX ? nx : kFX, ty = ny < kFY ? ny : kFY, tz = nz < kFZ ? nz : kFZ;
  const int vtx = tx + 1, nvox = (tx + 1) * (ty + 1);
  const int nzc = nz / tz;
  const int l = blockIdx.z / nzc, zc = blockIdx.z % nzc;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t N = a.N;
  const int x0 = blockIdx.x * tx, y0 = blockIdx.y * ty, z0 = zc * tz;
  const T beta = (T)cg->beta, alpha_prev = (T)cg->alpha;
  const bool use_old = cg->it > 0;
  const T ih[3] = {a.ih[0], a.ih[1], a.ih[2]};
  const int tid = threadIdx.x;
  const int ex = tid % vtx, ey = tid / vtx;      // voxel of the extended tile
  const bool vox = tid < nvox;
  const int vx = (x0 - 1 + ex) & (nx - 1), vy = (y0 - 1 + ey) & (ny - 1);
  const bool owned_xy = vox && ex > 0 && ey > 0;
  const T* Eb = a.E + (int64_t)(l / a.lcs) * N;
  const int64_t cbase = (int64_t)l * a.m * N;
  T acc = 0;
  int cur = 0;
  for (int zz = -1; zz < tz; ++zz) {
    const int vz = (z0 + zz) & (nz - 1);
    if (vox) {
      const int64_t v = ((int64_t)vz * ny + vy) * nx + vx;
      const bool owned = owned_xy && zz >= 0;
      T pv[36];
#pragma unroll
      for (int c = 0; c < 36; ++c) pv[c] = r[cbase + (int64_t)c * N + v];
      if (use_old) {
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          T po[6];
#pragma unroll
          for (int s = 0; s < 6; ++s) po[s] = pold[cbase + (int64_t)(6 * t + s) * N + v];
#pragma unroll
          for (int s = 0; s < 6; ++s) pv[6 * t + s] += beta * po[s];
          if (owned) {
            T xv[6];
#pragma unroll
            for (int s = 0; s < 6; ++s) xv[s] = x[cbase + (int64_t)(6 * t + s) * N + v];
#pragma unroll
            for (int s = 0; s < 6; ++s) x[cbase + (int64_t)(6 * t + s) * N + v] = xv[s] + alpha_prev * po[s];
          }
        }
      }
      if (owned) {
#pragma unroll
        for (int c = 0; c < 36; ++c) pnew[cbase + (int64_t)c * N + v] = pv[c];
      }
      const T e = Eb[v];
      T fc[8][3];
      voxel_corner_forces_3d<T>(pv, e, a.lam, a.mu2, ih, fc);
      if (owned) {
        // <p, C p> of the owned voxel (p : sigma over its tetrahedra, Mandel)
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const T* p = pv + 6 * t;
          const T tr = a.lam * (p[0] + p[1] + p[2]);
#pragma unroll
          for (int j = 0; j < 3; ++j) acc += p[j] * e * (tr + a.mu2 * p[j]);
#pragma unroll
          for (int j = 3; j < 6; ++j) acc += p[j] * e * a.mu2 * p[j];
        }
      }
      T* hc = hi + cur * 12 * kFVS;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          lo[(c * 3 + j) * kFVS + tid] = fc[c][j];       // corners (dx, dy, 0)
          hc[(c * 3 + j) * kFVS + tid] = fc[c + 4][j];   // corners (dx, dy, 1)
        }
    }
    __syncthreads();
    if (zz >= 0 && tid < tx * ty) {
      // node (x0 + lx, y0 + ly, z0 + zz): corner (dx, dy, dz) of voxel (x - dx, y - dy, z - dz)
      const int lx = tid % tx, ly = tid / tx;
      const T* hp = hi + (cur ^ 1) * 12 * kFVS;
      T fn[3] = {0, 0, 0};
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int i = (ly + 1 - dy) * vtx + (lx + 1 - dx);
          const int c = dx + 2 * dy;
#pragma unroll
          for (int j = 0; j < 3; ++j) fn[j] += lo[(c * 3 + j) * kFVS + i] + hp[(c * 3 + j) * kFVS + i];
        }
      const int64_t node = ((int64_t)(z0 + zz) * ny + (y0 + ly)) * nx + x0 + lx;
#pragma unroll
      for (int j = 0; j < 3; ++j) f[((int64_t)l * 3 + j) * N + node] = fn[j];
    }
    cur ^= 1;
    __syncthreads();
  }
  const double s = block_sum<kFNT>((double)acc, red);
  const int nblk = gridDim.x * gridDim.y * nzc;
  const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
    const double pq = sum_partials<kFNT>(part, nblk, red);
    if (threadIdx.x == 0) finish_alpha(cg, pq);
  }
}

// q = B_r w on every tetrahedron, r -= alpha q, <r, r>.  w: [L][3][N].
// grid (ceil(N / NT), L).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) strain_update_3d(PassArgs<T> a, const T* __restrict__ w, T* __restrict__ r) {
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int l = blockIdx.y;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int64_t N = a.N;
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  const T alpha = (T)cg->alpha;
  T acc = 0;
  if (v < N) {
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
    const T* wl = w + (int64_t)l * 3 * N;
    T uc[8][3];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cx = (x + (c & 1)) & (nx - 1), cy = (y + ((c >> 1) & 1)) & (ny - 1);
      const int cz = (z + ((c >> 2) & 1)) & (nz - 1);
      const int64_t i = ((int64_t)cz * ny + cy) * nx + cx;
#pragma unroll
      for (int j = 0; j < 3; ++j) uc[c][j] = __ldg(wl + j * N + i);
    }
    const int64_t cbase = (int64_t)l * a.m * N + v;
    const T r2 = (T)kInvSqrt2;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
      const int v1 = 1 << pa, v2 = v1 | (1 << pb);
      T H[3][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        H[pa][j] = (uc[v1][j] - uc[0][j]) * a.ih[pa];
        H[pb][j] = (uc[v2][j] - uc[v1][j]) * a.ih[pb];
        H[pc][j] = (uc[7][j] - uc[v2][j]) * a.ih[pc];
      }
      T q[6];
      q[0] = H[0][0]; q[1] = H[1][1]; q[2] = H[2][2];
      q[3] = r2 * (H[1][2] + H[2][1]);
      q[4] = r2 * (H[0][2] + H[2][0]);
      q[5] = r2 * (H[0][1] + H[1][0]);
      T rv[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) rv[s] = r[cbase + (int64_t)(6 * t + s) * N];
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        rv[s] -= alpha * q[s];
        acc += rv[s] * rv[s];
        r[cbase + (int64_t)(6 * t + s) * N] = rv[s];
      }
    }
  }
  const double s = block_sum<NT>((double)acc, red);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_e, blockIdx.x, gridDim.x, &flag)) {
    const double rr = sum_partials<NT>(part, gridDim.x, red);
    if (threadIdx.x == 0) finish_rr(cg, rr, false);
  }
}

// ----------------------------------------------------------------- 2D
constexpr int kGX = 256, kGY = 16;          // node tile (x, at most) and row chunk (y, at most)
constexpr int kGVS = kGX + 1;               // pixel row of the tile with its low-side halo
constexpr int kGNT = 288;                   // >= kGVS
static_assert(kGNT >= kGVS, "one thread per pixel of the extended row");

// Corner forces of the two triangles of one pixel: corner c = dx + 2 dy.
template <typename T>
__device__ __forceinline__ void voxel_corner_forces_2d(const T* pv /*[6]*/, T e, T lam, T mu2, T ihx, T ihy,
                                                       T f[4][2]) {
  const T r2 = (T)kInvSqrt2;
  // element 0 = nodes {00, 10, 01}: grad N_00 = (-ihx, -ihy), N_10 = (ihx, 0), N_01 = (0, ihy)
  // element 1 = nodes {11, 01, 10}: grad N_11 = (ihx, ihy), N_01 = (-ihx, 0), N_10 = (0, -ihy)
  T S[2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const T* p = pv + 3 * q;
    const T tr = lam * (p[0] + p[1]);
    S[q][0] = e * (tr + mu2 * p[0]);   // xx
    S[q][1] = e * (tr + mu2 * p[1]);   // yy
    S[q][2] = e * mu2 * p[2] * r2;     // xy (tensor)
  }
  // force of node i on component j: sum_a grad_a N_i sigma_aj
  f[0][0] = -ihx * S[0][0] - ihy * S[0][2];
  f[0][1] = -ihx * S[0][2] - ihy * S[0][1];
  f[1][0] = ihx * S[0][0] - ihy * S[1][2];
  f[1][1] = ihx * S[0][2] - ihy * S[1][1];
  f[2][0] = ihy * S[0][2] - ihx * S[1][0];
  f[2][1] = ihy * S[0][1] - ihx * S[1][2];
  f[3][0] = ihx * S[1][0] + ihy * S[1][2];
  f[3][1] = ihx * S[1][2] + ihy * S[1][1];
}

// 2D counterpart of force_stencil_3d, sweeping pixel rows.  grid
// (n_x/tx, (n_y/ty) L), kGNT threads; shared memory [3][4][kGVS] (static).
template <typename T>
__global__ void __launch_bounds__(kGNT) force_stencil_2d(PassArgs<T> a, const T* __restrict__ r,
                                                         const T* __restrict__ pold, T* __restrict__ pnew,
                                                         T* __restrict__ x, T* __restrict__ f) {
  __shared__ T lo[4][kGVS];      // corners dy = 0 of the current pixel row
  __shared__ T hi[2][4][kGVS];   // corners dy = 1 of the current / previous row
  __shared__ double red[kGNT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1];
  const int tx = nx < kGX ? nx : kGX, ty = ny < kGY ? ny : kGY;
  const int nyc = ny / ty;
  const int l = blockIdx.y / nyc, yc = blockIdx.y % nyc;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t N = a.N;
  const int x0 = blockIdx.x * tx, y0 = yc * ty;
  const T beta = (T)cg->beta, alpha_prev = (T)cg->alpha;
  const bool use_old = cg->it > 0;
  const int tid = threadIdx.x;
  const bool vox = tid <= tx;
  const int vx = (x0 - 1 + tid) & (nx - 1);
  const T* Eb = a.E + (int64_t)(l / a.lcs) * N;
  const int64_t cbase = (int64_t)l * a.m * N;
  T acc = 0;
  int cur = 0;
  for (int yy = -1; yy < ty; ++yy) {
    const int vy = (y0 + yy) & (ny - 1);
    if (vox) {
      const int64_t v = (int64_t)vy * nx + vx;
      const bool owned = tid > 0 && yy >= 0;
      T pv[6], po[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) pv[c] = r[cbase + (int64_t)c * N + v];
      if (use_old) {
#pragma unroll
        for (int c = 0; c < 6; ++c) po[c] = pold[cbase + (int64_t)c * N + v];
#pragma unroll
        for (int c = 0; c < 6; ++c) pv[c] += beta * po[c];
        if (owned) {
          T xv[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) xv[c] = x[cbase + (int64_t)c * N + v];
#pragma unroll
          for (int c = 0; c < 6; ++c) x[cbase + (int64_t)c * N + v] = xv[c] + alpha_prev * po[c];
        }
      }
      if (owned) {
#pragma unroll
        for (int c = 0; c < 6; ++c) pnew[cbase + (int64_t)c * N + v] = pv[c];
      }
      const T e = Eb[v];
      T fc[4][2];
      voxel_corner_forces_2d<T>(pv, e, a.lam, a.mu2, a.ih[0], a.ih[1], fc);
      if (owned) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const T* p = pv + 3 * q;
          const T tr = a.lam * (p[0] + p[1]);
          acc += p[0] * e * (tr + a.mu2 * p[0]) + p[1] * e * (tr + a.mu2 * p[1]) + p[2] * e * a.mu2 * p[2];
        }
      }
      lo[0][tid] = fc[0][0]; lo[1][tid] = fc[0][1]; lo[2][tid] = fc[1][0]; lo[3][tid] = fc[1][1];
      hi[cur][0][tid] = fc[2][0]; hi[cur][1][tid] = fc[2][1]; hi[cur][2][tid] = fc[3][0]; hi[cur][3][tid] = fc[3][1];
    }
    __syncthreads();
    if (yy >= 0 && tid < tx) {
      // node (x0 + tid, y0 + yy): corner (dx, 0) of pixel (x - dx, y), corner (dx, 1) of pixel (x - dx, y - 1)
      T fn[2] = {0, 0};
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int i = tid + 1 - dx;
#pragma unroll
        for (int j = 0; j < 2; ++j) fn[j] += lo[2 * dx + j][i] + hi[cur ^ 1][2 * dx + j][i];
      }
      const int64_t node = (int64_t)(y0 + yy) * nx + x0 + tid;
      f[((int64_t)l * 2 + 0) * N + node] = fn[0];
      f[((int64_t)l * 2 + 1) * N + node] = fn[1];
    }
    cur ^= 1;
    __syncthreads();
  }
  const double s = block_sum<kGNT>((double)acc, red);
  const int nblk = gridDim.x * nyc;
  const int blk = blockIdx.x + gridDim.x * yc;
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
    const double pq = sum_partials<kGNT>(part, nblk, red);
    if (threadIdx.x == 0) finish_alpha(cg, pq);
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) strain_update_2d(PassArgs<T> a, const T* __restrict__ w, T* __restrict__ r) {
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int l = blockIdx.y;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int nx = a.n[0], ny = a.n[1];
  const int64_t N = a.N;
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  const T alpha = (T)cg->alpha;
  T acc = 0;
  if (v < N) {
    const int x = (int)(v % nx), y = (int)(v / nx);
    const int x1 = (x + 1) & (nx - 1), y1 = (y + 1) & (ny - 1);
    const T* wl = w + (int64_t)l * 2 * N;
    const int64_t i00 = (int64_t)y * nx + x, i10 = (int64_t)y * nx + x1;
    const int64_t i01 = (int64_t)y1 * nx + x, i11 = (int64_t)y1 * nx + x1;
    T u00[2], u10[2], u01[2], u11[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      u00[j] = __ldg(wl + j * N + i00); u10[j] = __ldg(wl + j * N + i10);
      u01[j] = __ldg(wl + j * N + i01); u11[j] = __ldg(wl + j * N + i11);
    }
    const T ihx = a.ih[0], ihy = a.ih[1], r2 = (T)kInvSqrt2;
    T q[6];
    // element 0: d/dx = (u10 - u00) ihx, d/dy = (u01 - u00) ihy
    q[0] = (u10[0] - u00[0]) * ihx;
    q[1] = (u01[1] - u00[1]) * ihy;
    q[2] = r2 * ((u01[0] - u00[0]) * ihy + (u10[1] - u00[1]) * ihx);
    // element 1: d/dx = (u11 - u01) ihx, d/dy = (u11 - u10) ihy
    q[3] = (u11[0] - u01[0]) * ihx;
    q[4] = (u11[1] - u10[1]) * ihy;
    q[5] = r2 * ((u11[0] - u10[0]) * ihy + (u11[1] - u01[1]) * ihx);
    const int64_t cbase = (int64_t)l * a.m * N + v;
    T rv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) rv[c] = r[cbase + (int64_t)c * N];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      rv[c] -= alpha * q[c];
      acc += rv[c] * rv[c];
      r[cbase + (int64_t)c * N] = rv[c];
    }
  }
  const double s = block_sum<NT>((double)acc, red);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_e, blockIdx.x, gridDim.x, &flag)) {
    const double rr = sum_partials<NT>(part, gridDim.x, red);
    if (threadIdx.x == 0) finish_rr(cg, rr, false);
  }
}

// ------------------------------------------------------------ launchers
// pold / pnew: the previous and the new search direction (distinct buffers).
template <typename T>
cudaError_t launch_force_stencil(const PassArgs<T>& a, const T* pold, T* pnew, T* f, cudaStream_t s) {
  if (a.dim == 3) {
    const int tx = a.n[0] < kFX ? a.n[0] : kFX, ty = a.n[1] < kFY ? a.n[1] : kFY;
    const int tz = a.n[2] < kFZ ? a.n[2] : kFZ;
    const size_t sm = force_smem_3d<T>();
    static DeviceOnce attr;
    attr.run(current_device(), [&] { set_smem_attrs(force_stencil_3d<T>, sm); });
    dim3 grid(a.n[0] / tx, a.n[1] / ty, (a.n[2] / tz) * a.L);
    force_stencil_3d<T><<<grid, kFNT, sm, s>>>(a, a.r, pold, pnew, a.x, f);
  } else {
    const int tx = a.n[0] < kGX ? a.n[0] : kGX, ty = a.n[1] < kGY ? a.n[1] : kGY;
    dim3 grid(a.n[0] / tx, (a.n[1] / ty) * a.L);
    force_stencil_2d<T><<<grid, kGNT, 0, s>>>(a, a.r, pold, pnew, a.x, f);
  }
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_strain_update(const PassArgs<T>& a, const T* w, cudaStream_t s) {
  constexpr int NT = 256;
  dim3 grid((unsigned)((a.N + NT - 1) / NT), a.L);
  if (a.dim == 3) strain_update_3d<T, NT><<<grid, NT, 0, s>>>(a, w, a.r);
  else strain_update_2d<T, NT><<<grid, NT, 0, s>>>(a, w, a.r);
  return cudaGetLastError();
}

}  // namespace rve
