// Nodal-state form of the projected CG.  Every CG vector of the strain form
// is compatible (it lies in the range of G = B K^-1 B^T), so it is B applied
// to a nodal field: x = B xi, r = B rho, p = B pi, and q = G C p = B w with
// w = K^-1 B^T C B pi.  Running the same CG on the nodal fields (D
// components per node instead of m per voxel) gives the same iterates; the
// inner products stay those of the strain space:
//   <p, C p> = sum over elements of (B pi) : C (B pi)     (force kernel)
//   <r, r>   = sum over elements of |B rho|^2              (update kernel)
// This is the preconditioned-FE reading of the projection (Sec. 4: the
// operator acts as a preconditioner of the FE stiffness with B^T B in the
// role of the reference stiffness).
//
//   force kernel   pi = rho + beta pi_old, xi += alpha_prev pi_old,
//                  f = B^T C B pi, <B pi, C B pi> -> alpha
//   FFT passes     w = F^-1 (B^H B)^-1 F f    (D components)
//   update kernel  rho_new = rho - alpha w, <B rho_new, B rho_new> -> beta
//
// pi and rho each alternate between two buffers (the kernels read their
// neighbours' old values while owners write new ones).
#pragma once
#include "factored.cuh"

namespace rve {

// ----------------------------------------------------------------- 3D
// Node tile (at most kNX x kNY x kNZ) extended by one node on each side in x
// and y (the corners of the halo voxels), and the voxel tile with its
// low-side halo as in the strain-state force stencil.
constexpr int kNX = 32, kNY = 8, kNZ = 16;
constexpr int kNEX = kNX + 2, kNEY = kNY + 2, kNES = kNEX * kNEY;   // 340 nodes
constexpr int kNVS = (kNX + 1) * (kNY + 1);                        // 297 voxels
constexpr int kNNT = 352;
static_assert(kNNT >= kNES && kNNT >= kNVS, "one thread per node and per voxel of the tile");

// Mandel strains of the six tetrahedra of a voxel from its corner
// displacements uc[c][j], corner c = dx + 2 dy + 4 dz.
template <typename T>
__device__ __forceinline__ void tet_strains_3d(const T uc[8][3], const T* ih, T* pv /*[36]*/) {
  const T r2 = (T)kInvSqrt2;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
    const int v1 = 1 << pa, v2 = v1 | (1 << pb);
    T H[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      H[pa][j] = (uc[v1][j] - uc[0][j]) * ih[pa];
      H[pb][j] = (uc[v2][j] - uc[v1][j]) * ih[pb];
      H[pc][j] = (uc[7][j] - uc[v2][j]) * ih[pc];
    }
    T* q = pv + 6 * t;
    q[0] = H[0][0]; q[1] = H[1][1]; q[2] = H[2][2];
    q[3] = r2 * (H[1][2] + H[2][1]);
    q[4] = r2 * (H[0][2] + H[2][0]);
    q[5] = r2 * (H[0][1] + H[1][0]);
  }
}

// Corner forces B_e^T sigma_e of the six tetrahedra of a voxel straight from
// its corner displacements (strain, stress and force per tetrahedron, so only
// the corner values and the force accumulators stay live), and the voxel's
// share of <B u, C B u>.
template <typename T>
__device__ __forceinline__ void voxel_forces_from_corners_3d(const T uc[8][3], T e, T lam, T mu2, const T* ih,
                                                             T f[8][3], T& pq) {
  const T r2 = (T)kInvSqrt2;
#pragma unroll
  for (int c = 0; c < 8; ++c) f[c][0] = f[c][1] = f[c][2] = 0;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int pa = kuhn_perm(t, 0), pb = kuhn_perm(t, 1), pc = kuhn_perm(t, 2);
    const int v1 = 1 << pa, v2 = v1 | (1 << pb);
    T H[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      H[pa][j] = (uc[v1][j] - uc[0][j]) * ih[pa];
      H[pb][j] = (uc[v2][j] - uc[v1][j]) * ih[pb];
      H[pc][j] = (uc[7][j] - uc[v2][j]) * ih[pc];
    }
    // tensor strain (symmetric part of H) and stress
    const T exx = H[0][0], eyy = H[1][1], ezz = H[2][2];
    const T eyz = (T)0.5 * (H[1][2] + H[2][1]), exz = (T)0.5 * (H[0][2] + H[2][0]);
    const T exy = (T)0.5 * (H[0][1] + H[1][0]);
    const T tr = lam * (exx + eyy + ezz);
    T S[3][3];
    S[0][0] = e * (tr + mu2 * exx);
    S[1][1] = e * (tr + mu2 * eyy);
    S[2][2] = e * (tr + mu2 * ezz);
    S[1][2] = S[2][1] = e * mu2 * eyz;
    S[0][2] = S[2][0] = e * mu2 * exz;
    S[0][1] = S[1][0] = e * mu2 * exy;
    // eps : sigma (tensor contraction = Mandel dot product)
    pq += exx * S[0][0] + eyy * S[1][1] + ezz * S[2][2] + (T)2 * (eyz * S[1][2] + exz * S[0][2] + exy * S[0][1]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T Pa = ih[pa] * S[pa][j], Pb = ih[pb] * S[pb][j], Pc = ih[pc] * S[pc][j];
      f[0][j] -= Pa;
      f[v1][j] += Pa - Pb;
      f[v2][j] += Pb - Pc;
      f[7][j] += Pc;
    }
  }
  (void)r2;
}

// Ring sizes of the plane sweep: two node planes of pi, two voxel planes of
// dz = 0 corner forces and three of dz = 1 corner forces, so that the node
// sums of plane z - 1 and the voxel work of plane z share one barrier
// interval (two barriers per plane).
template <typename T> constexpr size_t nodal_force_smem_3d_v2() { return sizeof(T) * (2 * 3 * kNES + (2 + 3) * 12 * kNVS); }

// grid (n_x/tx, n_y/ty, (n_z/tz) L), kNNT threads, nodal_force_smem_3d_v2<T>()
// bytes of dynamic shared memory.  rho, pold, pnew, xi, f: [L][3][N].
// Loads of the next node plane (rho, pi_old, xi) and of the next voxel
// plane's modulus are issued one plane ahead into registers.
template <typename T>
__global__ void __launch_bounds__(kNNT, sizeof(T) == 4 ? 2 : 1)
    nodal_force_3d(PassArgs<T> a, const T* __restrict__ rho, const T* __restrict__ pold, T* __restrict__ pnew,
                   T* __restrict__ xi, T* __restrict__ f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pn = reinterpret_cast<T*>(smem_raw);   // [2][3][kNES]: pi of two node planes
  T* lo = pn + 2 * 3 * kNES;                // [2][12][kNVS]: corners dz = 0 of two voxel planes
  T* hi = lo + 2 * 12 * kNVS;               // [3][12][kNVS]: corners dz = 1 of three voxel planes
  __shared__ double red[kNNT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tx = nx < kNX ? nx : kNX, ty = ny < kNY ? ny : kNY, tz = nz < kNZ ? nz : kNZ;
  const int etx = tx + 2, nnode = (tx + 2) * (ty + 2);
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
  // node of the extended node tile handled by this thread
  const int nex = tid % etx, ney = tid / etx;
  const bool isnode = tid < nnode;
  const int gx = (x0 - 1 + nex) & (nx - 1), gy = (y0 - 1 + ney) & (ny - 1);
  const bool owned_node_xy = isnode && nex >= 1 && nex <= tx && ney >= 1 && ney <= ty;
  // voxel of the extended voxel tile handled by this thread
  const int vex = tid % vtx, vey = tid / vtx;
  const bool isvox = tid < nvox;
  const int vx = (x0 - 1 + vex) & (nx - 1), vy = (y0 - 1 + vey) & (ny - 1);
  const bool owned_vox_xy = isvox && vex > 0 && vey > 0;
  const T* Eb = a.E + (int64_t)(l / a.lcs) * N;
  const int64_t lbase = (int64_t)l * 3 * N;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t node_xy = (int64_t)gy * nx + gx;
  const int64_t vox_xy = (int64_t)vy * nx + vx;

  // registers of the node plane in flight
  T r_rho[3], r_po[3], r_xi[3];
  auto fetch_plane = [&](int pz) {
    if (!isnode) return;
    const int64_t node = (int64_t)((z0 + pz) & (nz - 1)) * plane + node_xy;
    const bool owned = owned_node_xy && pz >= 0 && pz < tz;
#pragma unroll
    for (int j = 0; j < 3; ++j) r_rho[j] = rho[lbase + (int64_t)j * N + node];
    if (use_old) {
#pragma unroll
      for (int j = 0; j < 3; ++j) r_po[j] = pold[lbase + (int64_t)j * N + node];
      if (owned) {
#pragma unroll
        for (int j = 0; j < 3; ++j) r_xi[j] = xi[lbase + (int64_t)j * N + node];
      }
    }
  };
  // pi of the fetched plane into dst[3][kNES]; owners write pi and xi
  auto commit_plane = [&](int pz, T* dst) {
    if (!isnode) return;
    const int64_t node = (int64_t)((z0 + pz) & (nz - 1)) * plane + node_xy;
    const bool owned = owned_node_xy && pz >= 0 && pz < tz;
    T pv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) pv[j] = use_old ? r_rho[j] + beta * r_po[j] : r_rho[j];
    if (owned) {
#pragma unroll
      for (int j = 0; j < 3; ++j) pnew[lbase + (int64_t)j * N + node] = pv[j];
      if (use_old) {
#pragma unroll
        for (int j = 0; j < 3; ++j) xi[lbase + (int64_t)j * N + node] = r_xi[j] + alpha_prev * r_po[j];
      }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) dst[j * kNES + tid] = pv[j];
  };
  T r_e = 0;
  auto fetch_e = [&](int vz) {
    if (isvox) r_e = Eb[(int64_t)((z0 + vz) & (nz - 1)) * plane + vox_xy];
  };

  fetch_plane(-1);
  commit_plane(-1, pn);
  fetch_plane(0);
  fetch_e(-1);
  T acc = 0;
  for (int zz = -1; zz < tz; ++zz) {
    // (1) pi of node plane zz + 1 (fetched one step ahead) into the ring; the
    //     node sums of plane zz - 1; fetch the next plane and modulus
    commit_plane(zz + 1, pn + ((zz + 2) & 1) * 3 * kNES);
    const T e = r_e;
    if (zz + 2 <= tz) fetch_plane(zz + 2);
    if (zz + 1 < tz) fetch_e(zz + 1);
    if (zz >= 1 && tid < tx * ty) {
      // node (x0 + lx, y0 + ly, z0 + zz - 1): dz = 0 corners of voxel plane zz - 1,
      // dz = 1 corners of voxel plane zz - 2
      const int lx = tid % tx, ly = tid / tx;
      const T* lp = lo + ((zz - 1) & 1) * 12 * kNVS;
      const T* hp = hi + ((zz + 1) % 3) * 12 * kNVS;   // plane zz - 2
      T fn[3] = {0, 0, 0};
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int i = (ly + 1 - dy) * vtx + (lx + 1 - dx);
          const int c = dx + 2 * dy;
#pragma unroll
          for (int j = 0; j < 3; ++j) fn[j] += lp[(c * 3 + j) * kNVS + i] + hp[(c * 3 + j) * kNVS + i];
        }
      const int64_t node = ((int64_t)(z0 + zz - 1) * ny + (y0 + ly)) * nx + x0 + lx;
#pragma unroll
      for (int j = 0; j < 3; ++j) f[lbase + (int64_t)j * N + node] = fn[j];
    }
    __syncthreads();
    // (2) corner forces of voxel plane zz from node planes zz and zz + 1
    if (isvox) {
      const T* p0 = pn + ((zz + 1) & 1) * 3 * kNES;
      const T* p1 = pn + ((zz + 2) & 1) * 3 * kNES;
      T uc[8][3];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int i = (vey + ((c >> 1) & 1)) * etx + vex + (c & 1);
        const T* src = (c & 4) ? p1 : p0;
#pragma unroll
        for (int j = 0; j < 3; ++j) uc[c][j] = src[j * kNES + i];
      }
      T fc[8][3];
      T pq = 0;
      voxel_forces_from_corners_3d<T>(uc, e, a.lam, a.mu2, ih, fc, pq);
      if (owned_vox_xy && zz >= 0) acc += pq;
      T* lc = lo + (zz & 1) * 12 * kNVS;
      T* hc = hi + ((zz + 3) % 3) * 12 * kNVS;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          lc[(c * 3 + j) * kNVS + tid] = fc[c][j];
          hc[(c * 3 + j) * kNVS + tid] = fc[c + 4][j];
        }
    }
    __syncthreads();
  }
  // node sums of the last plane z0 + tz - 1
  if (tid < tx * ty) {
    const int zz = tz;
    const int lx = tid % tx, ly = tid / tx;
    const T* lp = lo + ((zz - 1) & 1) * 12 * kNVS;
    const T* hp = hi + ((zz + 1) % 3) * 12 * kNVS;
    T fn[3] = {0, 0, 0};
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int i = (ly + 1 - dy) * vtx + (lx + 1 - dx);
        const int c = dx + 2 * dy;
#pragma unroll
        for (int j = 0; j < 3; ++j) fn[j] += lp[(c * 3 + j) * kNVS + i] + hp[(c * 3 + j) * kNVS + i];
      }
    const int64_t node = ((int64_t)(z0 + zz - 1) * ny + (y0 + ly)) * nx + x0 + lx;
#pragma unroll
    for (int j = 0; j < 3; ++j) f[lbase + (int64_t)j * N + node] = fn[j];
  }
  const double s = block_sum<kNNT>((double)acc, red);
  const int nblk = gridDim.x * gridDim.y * nzc;
  const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
    const double pq = sum_partials<kNNT>(part, nblk, red);
    if (threadIdx.x == 0) finish_alpha(cg, pq);
  }
}

// rho_new = rho_old - alpha w (init: rho = -w, xi = 0) at every node and
// <B rho_new, B rho_new> over the six tetrahedra of every voxel.  Thread
// (x, y) sweeps z over a chunk of kUZ planes, keeping the updated corner
// values of plane z + 1 for the next step; the node (x, y, z) is written
// once.  NT threads cover bx x by columns, bx = min(n_x, 32), by = NT / bx;
// grid (n_x/bx, n_y/by, (n_z/kUZ) L).
constexpr int kUZ = 16;
template <typename T, int NT>
__global__ void __launch_bounds__(NT) nodal_update_3d(PassArgs<T> a, const T* __restrict__ rho_old,
                                                      const T* __restrict__ w, T* __restrict__ rho_new,
                                                      T* __restrict__ xi, int init) {
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tz = nz < kUZ ? nz : kUZ;
  const int nzc = nz / tz;
  const int l = blockIdx.z / nzc, zc = blockIdx.z % nzc;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t N = a.N;
  const int bx = nx < 32 ? nx : 32, by = NT / bx;
  const int x = blockIdx.x * bx + (threadIdx.x & (bx - 1)), y = blockIdx.y * by + threadIdx.x / bx;
  const int x1 = (x + 1) & (nx - 1), y1 = (y + 1) & (ny - 1);
  const T alpha = init ? (T)0 : (T)cg->alpha;
  const int64_t lbase = (int64_t)l * 3 * N;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t o00 = (int64_t)y * nx + x, o10 = (int64_t)y * nx + x1;
  const int64_t o01 = (int64_t)y1 * nx + x, o11 = (int64_t)y1 * nx + x1;
  const int z0 = zc * tz;
  // updated values of the 4 corners (dx, dy) of one node plane
  auto corners = [&](int z, T c[4][3]) {
    const int64_t pb = lbase + (int64_t)(z & (nz - 1)) * plane;
    const int64_t off[4] = {o00, o10, o01, o11};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int64_t i = pb + (int64_t)j * N + off[k];
        c[k][j] = init ? -__ldg(w + i) : __ldg(rho_old + i) - alpha * __ldg(w + i);
      }
  };
  T lo[4][3], hi[4][3];
  corners(z0, lo);
  T acc = 0;
  for (int z = z0; z < z0 + tz; ++z) {
    corners(z + 1, hi);
    const int64_t v = lbase + (int64_t)z * plane + o00;
#pragma unroll
    for (int j = 0; j < 3; ++j) rho_new[v + (int64_t)j * N] = lo[0][j];
    if (init) {
#pragma unroll
      for (int j = 0; j < 3; ++j) xi[v + (int64_t)j * N] = 0;
    }
    T uc[8][3];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) { uc[k][j] = lo[k][j]; uc[k + 4][j] = hi[k][j]; }
    T pv[36];
    tet_strains_3d<T>(uc, a.ih, pv);
#pragma unroll
    for (int c = 0; c < 36; ++c) acc += pv[c] * pv[c];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) lo[k][j] = hi[k][j];
  }
  const double s = block_sum<NT>((double)acc, red);
  const int nblk = gridDim.x * gridDim.y * nzc;
  const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc);
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_e, blk, nblk, &flag)) {
    const double rr = sum_partials<NT>(part, nblk, red);
    if (threadIdx.x == 0) finish_rr(cg, rr, init != 0);
  }
}

// ----------------------------------------------------------------- 2D
constexpr int kMX = 256, kMY = 16;                 // node tile (x, at most) and row chunk (y, at most)
constexpr int kMEX = kMX + 2, kMVX = kMX + 1;      // node row with both halo nodes, pixel row with low halo
constexpr int kMNT = 288;
static_assert(kMNT >= kMEX, "one thread per node of the extended row");

// Mandel strains of the two triangles of a pixel from its corner
// displacements uc[c][j], corner c = dx + 2 dy.
template <typename T>
__device__ __forceinline__ void tri_strains_2d(const T uc[4][2], T ihx, T ihy, T* q /*[6]*/) {
  const T r2 = (T)kInvSqrt2;
  // element 0 = nodes {00, 10, 01}; element 1 = nodes {11, 01, 10}
  q[0] = (uc[1][0] - uc[0][0]) * ihx;
  q[1] = (uc[2][1] - uc[0][1]) * ihy;
  q[2] = r2 * ((uc[2][0] - uc[0][0]) * ihy + (uc[1][1] - uc[0][1]) * ihx);
  q[3] = (uc[3][0] - uc[2][0]) * ihx;
  q[4] = (uc[3][1] - uc[1][1]) * ihy;
  q[5] = r2 * ((uc[3][0] - uc[1][0]) * ihy + (uc[3][1] - uc[2][1]) * ihx);
}

// grid (n_x/tx, (n_y/ty) L), kMNT threads.  rho, pold, pnew, xi, f: [L][2][N].
template <typename T>
__global__ void __launch_bounds__(kMNT) nodal_force_2d(PassArgs<T> a, const T* __restrict__ rho,
                                                       const T* __restrict__ pold, T* __restrict__ pnew,
                                                       T* __restrict__ xi, T* __restrict__ f) {
  __shared__ T pn[2][2][kMEX];    // pi of two node rows
  __shared__ T lo[4][kMVX];       // corners dy = 0 of the current pixel row
  __shared__ T hi[2][4][kMVX];    // corners dy = 1 of the current / previous row
  __shared__ double red[kMNT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1];
  const int tx = nx < kMX ? nx : kMX, ty = ny < kMY ? ny : kMY;
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
  const bool isnode = tid < tx + 2;
  const int gx = (x0 - 1 + tid) & (nx - 1);
  const bool owned_node_x = isnode && tid >= 1 && tid <= tx;
  const bool isvox = tid <= tx;
  const int vx = (x0 - 1 + tid) & (nx - 1);
  const T* Eb = a.E + (int64_t)(l / a.lcs) * N;
  const int64_t lbase = (int64_t)l * 2 * N;

  auto load_row = [&](int py, T (*dst)[kMEX]) {
    if (!isnode) return;
    const int gy = (y0 + py) & (ny - 1);
    const int64_t node = (int64_t)gy * nx + gx;
    const bool owned = owned_node_x && py >= 0 && py < ty;
    T pv[2], po[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) pv[j] = rho[lbase + (int64_t)j * N + node];
    if (use_old) {
#pragma unroll
      for (int j = 0; j < 2; ++j) po[j] = pold[lbase + (int64_t)j * N + node];
#pragma unroll
      for (int j = 0; j < 2; ++j) pv[j] += beta * po[j];
      if (owned) {
#pragma unroll
        for (int j = 0; j < 2; ++j) xi[lbase + (int64_t)j * N + node] += alpha_prev * po[j];
      }
    }
    if (owned) {
#pragma unroll
      for (int j = 0; j < 2; ++j) pnew[lbase + (int64_t)j * N + node] = pv[j];
    }
    dst[0][tid] = pv[0];
    dst[1][tid] = pv[1];
  };

  load_row(-1, pn[0]);
  T acc = 0;
  int cur = 0;
  for (int yy = -1; yy < ty; ++yy) {
    load_row(yy + 1, pn[(yy + 2) & 1]);
    __syncthreads();
    if (isvox) {
      T (*p0)[kMEX] = pn[(yy + 1) & 1];
      T (*p1)[kMEX] = pn[(yy + 2) & 1];
      T uc[4][2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uc[0][j] = p0[j][tid]; uc[1][j] = p0[j][tid + 1];
        uc[2][j] = p1[j][tid]; uc[3][j] = p1[j][tid + 1];
      }
      T pv[6];
      tri_strains_2d<T>(uc, a.ih[0], a.ih[1], pv);
      const int vy = (y0 + yy) & (ny - 1);
      const T e = Eb[(int64_t)vy * nx + vx];
      T fc[4][2];
      voxel_corner_forces_2d<T>(pv, e, a.lam, a.mu2, a.ih[0], a.ih[1], fc);
      if (tid > 0 && yy >= 0) {
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
      T fn[2] = {0, 0};
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int i = tid + 1 - dx;
#pragma unroll
        for (int j = 0; j < 2; ++j) fn[j] += lo[2 * dx + j][i] + hi[cur ^ 1][2 * dx + j][i];
      }
      const int64_t node = (int64_t)(y0 + yy) * nx + x0 + tid;
      f[lbase + node] = fn[0];
      f[lbase + N + node] = fn[1];
    }
    cur ^= 1;
    __syncthreads();
  }
  const double s = block_sum<kMNT>((double)acc, red);
  const int nblk = gridDim.x * nyc;
  const int blk = blockIdx.x + gridDim.x * yc;
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
    const double pq = sum_partials<kMNT>(part, nblk, red);
    if (threadIdx.x == 0) finish_alpha(cg, pq);
  }
}

// 2D counterpart of nodal_update_3d: NT threads cover bx columns (bx =
// min(n_x, NT)) x NT/bx row groups of kUY rows; each thread sweeps its rows
// keeping the updated corner values of row y + 1.  grid (n_x/bx,
// max(1, n_y/(kUY NT/bx)) L); row groups past n_y are idle.
constexpr int kUY = 16;
template <typename T, int NT>
__global__ void __launch_bounds__(NT) nodal_update_2d(PassArgs<T> a, const T* __restrict__ rho_old,
                                                      const T* __restrict__ w, T* __restrict__ rho_new,
                                                      T* __restrict__ xi, int init) {
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int nx = a.n[0], ny = a.n[1];
  const int bx = nx < NT ? nx : NT, by = NT / bx;
  const int rows_blk = by * kUY;
  const int nyb = ny > rows_blk ? ny / rows_blk : 1;
  const int l = blockIdx.y / nyb, yb = blockIdx.y % nyb;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t N = a.N;
  const int x = blockIdx.x * bx + (threadIdx.x % bx);
  const int ys = yb * rows_blk + (threadIdx.x / bx) * kUY;
  const int x1 = (x + 1) & (nx - 1);
  const T alpha = init ? (T)0 : (T)cg->alpha;
  const int64_t lbase = (int64_t)l * 2 * N;
  T acc = 0;
  if (ys < ny) {
    auto corners = [&](int y, T c[2][2]) {
      const int64_t rb = lbase + (int64_t)(y & (ny - 1)) * nx;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int64_t i0 = rb + (int64_t)j * N + x, i1 = rb + (int64_t)j * N + x1;
        c[0][j] = init ? -__ldg(w + i0) : __ldg(rho_old + i0) - alpha * __ldg(w + i0);
        c[1][j] = init ? -__ldg(w + i1) : __ldg(rho_old + i1) - alpha * __ldg(w + i1);
      }
    };
    T lo[2][2], hi[2][2];
    corners(ys, lo);
    for (int y = ys; y < ys + kUY; ++y) {
      corners(y + 1, hi);
      const int64_t v = lbase + (int64_t)y * nx + x;
      rho_new[v] = lo[0][0];
      rho_new[v + N] = lo[0][1];
      if (init) { xi[v] = 0; xi[v + N] = 0; }
      const T uc[4][2] = {{lo[0][0], lo[0][1]}, {lo[1][0], lo[1][1]}, {hi[0][0], hi[0][1]}, {hi[1][0], hi[1][1]}};
      T q[6];
      tri_strains_2d<T>(uc, a.ih[0], a.ih[1], q);
#pragma unroll
      for (int c = 0; c < 6; ++c) acc += q[c] * q[c];
#pragma unroll
      for (int k = 0; k < 2; ++k) { lo[k][0] = hi[k][0]; lo[k][1] = hi[k][1]; }
    }
  }
  const double s = block_sum<NT>((double)acc, red);
  const int nblk = gridDim.x * nyb;
  const int blk = blockIdx.x + gridDim.x * yb;
  double* part = a.part + (int64_t)l * a.part_stride;
  if (publish_partial(s, part, &cg->cnt_e, blk, nblk, &flag)) {
    const double rr = sum_partials<NT>(part, nblk, red);
    if (threadIdx.x == 0) finish_rr(cg, rr, init != 0);
  }
}

// After the CG: xi += alpha pi_last (the deferred update, for load cases that
// ran an iteration and did not break down), then u += xi in FP64.
// grid (ceil(N / NT), L).  pi_even / pi_odd: direction buffers of even / odd
// iterations.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) nodal_finish(PassArgs<T> a, const T* __restrict__ pi_even,
                                                   const T* __restrict__ pi_odd, const T* __restrict__ xi) {
  const int l = blockIdx.y;
  const CgState* cg = a.cg + l;
  if (!cg->active) return;
  const int64_t N = a.N;
  const int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (v >= N) return;
  const bool last = cg->it > 0 && cg->status != ST_BAD;
  const T alpha = last ? (T)cg->alpha : (T)0;
  const T* pl = ((cg->it - 1) & 1) ? pi_odd : pi_even;
  const int64_t lbase = (int64_t)l * a.dim * N;
  for (int j = 0; j < a.dim; ++j) {
    T x = xi[lbase + j * N + v];
    if (last) x += alpha * pl[lbase + j * N + v];
    a.u64[lbase + j * N + v] += (double)x;
  }
}

// ------------------------------------------------------------ launchers
template <typename T>
cudaError_t launch_nodal_force(const PassArgs<T>& a, const T* rho, const T* pold, T* pnew, T* xi, T* f,
                               cudaStream_t s) {
  if (a.dim == 3) {
    const int tx = a.n[0] < kNX ? a.n[0] : kNX, ty = a.n[1] < kNY ? a.n[1] : kNY;
    const int tz = a.n[2] < kNZ ? a.n[2] : kNZ;
    const size_t sm = nodal_force_smem_3d_v2<T>();
    static DeviceOnce attr;
    attr.run(current_device(), [&] { set_smem_attrs(nodal_force_3d<T>, sm); });
    dim3 grid(a.n[0] / tx, a.n[1] / ty, (a.n[2] / tz) * a.L);
    nodal_force_3d<T><<<grid, kNNT, sm, s>>>(a, rho, pold, pnew, xi, f);
  } else {
    const int tx = a.n[0] < kMX ? a.n[0] : kMX, ty = a.n[1] < kMY ? a.n[1] : kMY;
    dim3 grid(a.n[0] / tx, (a.n[1] / ty) * a.L);
    nodal_force_2d<T><<<grid, kMNT, 0, s>>>(a, rho, pold, pnew, xi, f);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nodal_update(const PassArgs<T>& a, const T* rho_old, const T* w, T* rho_new, T* xi, int init,
                                cudaStream_t s) {
  constexpr int NT = 256;
  if (a.dim == 3) {
    const int bx = a.n[0] < 32 ? a.n[0] : 32, by = NT / bx;   // n_y >= 16 >= by
    const int tz = a.n[2] < kUZ ? a.n[2] : kUZ;
    dim3 grid(a.n[0] / bx, a.n[1] / by, (a.n[2] / tz) * a.L);
    nodal_update_3d<T, NT><<<grid, NT, 0, s>>>(a, rho_old, w, rho_new, xi, init);
  } else {
    const int bx = a.n[0] < NT ? a.n[0] : NT, rows_blk = (NT / bx) * kUY;
    const int nyb = a.n[1] > rows_blk ? a.n[1] / rows_blk : 1;
    dim3 grid(a.n[0] / bx, nyb * a.L);
    nodal_update_2d<T, NT><<<grid, NT, 0, s>>>(a, rho_old, w, rho_new, xi, init);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nodal_finish(const PassArgs<T>& a, const T* pi_even, const T* pi_odd, const T* xi,
                                cudaStream_t s) {
  constexpr int NT = 256;
  dim3 grid((unsigned)((a.N + NT - 1) / NT), a.L);
  nodal_finish<T, NT><<<grid, NT, 0, s>>>(a, pi_even, pi_odd, xi);
  return cudaGetLastError();
}

}  // namespace rve
