// 3D projected-operator passes (six Kuhn tetrahedra per voxel).
//
// Real fields are [l][c][z][y][x].  One application of q = G * (C : p):
//   A  material (+ CG direction update, <p, C p>) and forward real FFT along x;
//      writes spec1 as [l][c][k_x][z][y] (y contiguous);
//   B  forward FFT along y of whole y-pencils; writes spec2 as
//      [l][c][k_x][k_y][z] (z contiguous, chunks of TZB z per k_y);
//   C  forward FFT along z, projection G(k) per wavevector, inverse FFT along
//      z, in place on spec2 (all m = 36 components of one (k_x, k_y) pencil);
//   D  inverse FFT along y, spec2 -> spec1;
//   E  inverse real FFT along x, r -= alpha q, <r, r> (x += alpha p is
//      deferred to the next pass A, as in 2D).
#pragma once
#include "pass2d.cuh"
#include "pass3d_pipe.cuh"

namespace rve {

// Kuhn tetrahedron Theta = permutation (a, b, c) of (x, y, z), lexicographic.
__host__ __device__ constexpr int kuhn_perm(int t, int i) {
  // rows: (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0)
  return (t == 0) ? (i == 0 ? 0 : i == 1 ? 1 : 2)
       : (t == 1) ? (i == 0 ? 0 : i == 1 ? 2 : 1)
       : (t == 2) ? (i == 0 ? 1 : i == 1 ? 0 : 2)
       : (t == 3) ? (i == 0 ? 1 : i == 1 ? 2 : 0)
       : (t == 4) ? (i == 0 ? 2 : i == 1 ? 0 : 1)
                  : (i == 0 ? 2 : i == 1 ? 1 : 0);
}

// --------------------------------------------- L2 prefetch of a later tile
// The transform passes run grids of far more blocks than are resident, and
// the blocks start in about linear launch order as earlier ones retire.  With
// a.pf_ahead = D > 0 every block asks the TMA unit to bring the input of
// block b + D (b its own linear index) into L2 (bulk prefetches: no data
// reaches the SM and nothing waits on them), so that DRAM keeps streaming a
// later tile while this block transforms its own (passes A and E: tile
// variants 6 and 4; passes B, C and D: always in FP32; the distances are in
// prefetch_distance).
//
// Block coordinates (x, y, z) of the block a.pf_ahead places after this one in
// launch order; false past the end of the grid.
template <typename T>
__device__ __forceinline__ bool grid_ahead(const PassArgs<T>& a, int& bx, int& by, int& bz) {
  const int64_t nblk = (int64_t)gridDim.x * gridDim.y * gridDim.z;
  const int64_t b = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z) + a.pf_ahead;
  if (b >= nblk) return false;
  bx = (int)(b % gridDim.x);
  const int64_t b1 = b / gridDim.x;
  by = (int)(b1 % gridDim.y);
  bz = (int)(b1 / gridDim.y);
  return true;
}
// Whether load case l still runs (its rows are worth prefetching).
template <typename T> __device__ __forceinline__ bool slot_runs(const PassArgs<T>& a, int l) {
  const CgState* cg = a.cg + l;
  return cg->active && !(a.cgphase && cg->status != ST_RUN);
}
// Passes A and E (grid (n_y/TY, n_z, L*G)): tile (l, grp, z, y0) of the later
// block; false past the end of the grid or for a load case whose CG has stopped.
template <typename T>
__device__ __forceinline__ bool block_ahead(const PassArgs<T>& a, int G, int TY, int& l, int& grp, int& z, int& y0) {
  int bx, bz;
  if (!grid_ahead(a, bx, z, bz)) return false;
  y0 = bx * TY;
  l = bz / G;
  grp = bz % G;
  return slot_runs(a, l);
}

// Pass A (CG mode, stress form): the r, E and (after the first iteration)
// p_old and x rows of the later block: TY contiguous rows of NX values per
// component, 19 requests of TY * NX * sizeof(T) bytes, one per thread.
template <typename T, int NX, int TY>
__device__ __forceinline__ void pass_a_prefetch_ahead(const PassArgs<T>& a, int G) {
  static_assert((TY * NX * sizeof(T)) % 16 == 0, "bulk prefetch sizes are multiples of 16 bytes");
  const int t = threadIdx.x;
  if (t >= 19) return;
  int l, grp, z, y0;
  if (!block_ahead(a, G, TY, l, grp, z, y0)) return;
  if (t >= 7 && a.cg[l].it == 0) return;   // no p_old or x reads in the first iteration
  const int64_t N = a.N;
  const int64_t row0 = ((int64_t)z * a.n[1] + y0) * NX;
  const int64_t comp = ((int64_t)l * a.m + grp * 6) * N + row0;
  const T* src = t < 6 ? a.r + comp + t * N
               : t == 6 ? a.E + (int64_t)(l / a.lcs) * N + row0
               : t < 13 ? a.p + comp + (t - 7) * N
                        : a.x + comp + (t - 13) * N;
  prefetch_l2_bulk(src, (unsigned)(TY * NX * sizeof(T)));
}

// Pass E (CG mode, stress form): the later block's spectrum tile (TY
// contiguous y values for each of its six components and NX/2 + 1 k_x) and its
// r rows.
template <typename T, int NX, int TY>
__device__ __forceinline__ void pass_e_prefetch_ahead(const PassArgs<T>& a, int G) {
  constexpr int KX = NX / 2 + 1;
  static_assert((TY * sizeof(cplx<T>)) % 16 == 0, "bulk prefetch sizes are multiples of 16 bytes");
  static_assert((TY * NX * sizeof(T)) % 16 == 0, "bulk prefetch sizes are multiples of 16 bytes");
  int l, grp, z, y0;
  if (!block_ahead(a, G, TY, l, grp, z, y0)) return;
  const int ny = a.n[1], nz = a.n[2];
  const cplx<T>* s0 = a.spec + ((((int64_t)l * a.m + grp * 6) * KX) * nz + z) * ny + y0;
  const T* r0 = a.r + ((int64_t)l * a.m + grp * 6) * a.N + ((int64_t)z * ny + y0) * NX;
  for (int i = threadIdx.x; i < 6 * KX + 6; i += blockDim.x) {
    if (i < 6 * KX)
      prefetch_l2_bulk(s0 + (int64_t)i * nz * ny, (unsigned)(TY * sizeof(cplx<T>)));   // i = c KX + k_x
    else
      prefetch_l2_bulk(r0 + (int64_t)(i - 6 * KX) * a.N, (unsigned)(TY * NX * sizeof(T)));
  }
}

// ---------------------------------------------------------------- pass A
// Resident blocks per SM the register budget is sized for.
template <typename T, int NT> __host__ __device__ constexpr int pass_a_min_blocks() {
  return sizeof(T) != 4 ? 1 : NT <= 384 ? 3 : NT <= 512 ? 2 : 1;
}

// grid (n_y/TY, n_z, L*G), G = 6 tetrahedra (6 components each) or 1 (nodal, 3).
// NT is either the FFT's thread count or (tile variants 3, 4) the number of
// load units of the tile, so that every thread streams exactly one unit.
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT, pass_a_min_blocks<T, NT>()) pass_a_3d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int GS = 6;
  constexpr int KX = NX / 2 + 1;
  constexpr int LD = ae_ld<NX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [GS][NP][LD]
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const bool nodal = (a.amode == A_NODAL);
  const int G = nodal ? 1 : a.nq;
  const int l = blockIdx.z / G, grp = blockIdx.z % G;
  const int z = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1], nz = a.n[2];
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int c0 = nodal ? 0 : grp * 6;
  T beta = 0, alpha_prev = 0;
  bool use_old = false;
  if (a.amode == A_CG) { beta = (T)cg->beta; alpha_prev = (T)cg->alpha; use_old = cg->it > 0; }
  if (a.pf_ahead > 0 && a.amode == A_CG && !nodal) pass_a_prefetch_ahead<T, NX, TY>(a, G);
  // two columns per unit: 6 components x 2 rows x (r, p, x) stay in registers
  const T acc = pass_a_load<T, NX, TY, GS, NT, LD, 2>(a, buf, l, c0, ((int64_t)z * ny + y0) * NX, nodal, beta,
                                                      alpha_prev, use_old);
  __syncthreads();
  smem_fft<T, NX, GS * NP, LD, NT, -1>(buf, a.tw[0]);
  pass_a_store<T, NX, TY, NT, LD>(buf, nodal ? 3 : 6,
                                  a.spec + ((((int64_t)l * a.m + c0) * KX) * nz + z) * ny + y0,
                                  (int64_t)KX * nz * ny, (int64_t)nz * ny);

  if (a.amode == A_CG) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y * G;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * grp);
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
      const double pq = sum_partials<NT>(part, nblk, red);
      if (threadIdx.x == 0) finish_alpha(cg, pq);
    }
  }
}

// ---------------------------------------------------------------- pass B / D
// FFT along y.  grid (n_z/TZB, n_x/2+1, L*Cc).  FWD: spec1 pencils -> spec2
// chunks; !FWD: spec2 chunks -> spec1 pencils.
template <typename T, int NY, int TZB, int NT, bool FWD, int V = 0>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT <= 256 ? 4 : 2) : 1) pass_y_3d(PassArgs<T> a, int Cc) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LD = FftSplit<NY, V>::LDO;  // odd: the chunk transposes are conflict-free
  C* buf = reinterpret_cast<C*>(smem_raw);  // [TZB][LD]
  const int l = blockIdx.z / Cc, c = blockIdx.z % Cc;
  const int kx = blockIdx.y, z0 = blockIdx.x * TZB;
  const int nz = a.n[2], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t cbase = (((int64_t)l * a.m + c) * KX + kx);
  C* pencils = a.spec + (cbase * nz + z0) * NY;  // [zz][y], y contiguous
  C* chunks = a.spec2 + cbase * NY * nz + z0;     // [k_y][zz], zz contiguous
  // L2 prefetch of the later block's input (see grid_ahead): forward, its
  // TZB contiguous y-pencils (one request); inverse, its NY z-chunks of TZB
  // values
  int zb2, kx2, lc2;
  if (a.pf_ahead > 0 && grid_ahead(a, zb2, kx2, lc2) && slot_runs(a, lc2 / Cc)) {
    static_assert((TZB * sizeof(C)) % 16 == 0, "bulk prefetch sizes are multiples of 16 bytes");
    const int64_t cb2 = (((int64_t)(lc2 / Cc) * a.m + lc2 % Cc) * KX + kx2);
    const int z2 = zb2 * TZB;
    if (FWD) {
      if (threadIdx.x == 0) prefetch_l2_bulk(a.spec + (cb2 * nz + z2) * NY, (unsigned)(TZB * NY * sizeof(C)));
    } else {
      for (int k = threadIdx.x; k < NY; k += blockDim.x)
        prefetch_l2_bulk(a.spec2 + cb2 * NY * nz + z2 + (int64_t)k * nz, (unsigned)(TZB * sizeof(C)));
    }
  }
  if (FWD) {
    // step 1 reads whole y-pencils, step 2 writes z-chunks (zz fastest)
    auto ld = [&](int zz, int y) -> C { return pencils[(int64_t)zz * NY + y]; };
    auto st = [&](int zz, int k, C v) { chunks[(int64_t)k * nz + zz] = v; };
    fft4<T, NY, TZB, LD, NT, -1, false, false, false, true, V>(buf, a.tw[1], ld, st);
  } else {
    auto ld = [&](int zz, int k) -> C { return chunks[(int64_t)k * nz + zz]; };
    auto st = [&](int zz, int y, C v) { pencils[(int64_t)zz * NY + y] = v; };
    fft4<T, NY, TZB, LD, NT, +1, false, false, true, false, V>(buf, a.tw[1], ld, st);
  }
}

// ---------------------------------------------------------------- pass C
// Projection at one wavevector of the column kz of buf ([36][LD] in shared
// memory), in place, streaming the components so that only the element
// gradients, B^H B and t live in registers.
//   mode P_G:         s (36) -> B (B^H B)^-1 B^H s
//   mode P_NODAL_IN:  rows 0..2 = f^ -> B (B^H B)^-1 f^   (36 out)
//   mode P_NODAL_OUT: s (36) -> (B^H B)^-1 B^H s           (3 out, rows 0..2)
template <typename T, int LD>
__device__ __forceinline__ void project_3d(cplx<T>* col, const cplx<T>* e, const T* ih, T scale, int mode) {
  using C = cplx<T>;
  const C one = mkc<T>(1, 0);
  C d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = cscale(csub(e[i], one), ih[i]);
  const C e01 = cmul(e[0], e[1]), e02 = cmul(e[0], e[2]), e12 = cmul(e[1], e[2]);
  // element gradients g[t][axis] of the Kuhn tetrahedra {0, e_a, e_a+e_b, 1}
  C g[6][3];
  g[0][0] = d[0];             g[0][1] = cmul(e[0], d[1]);  g[0][2] = cmul(e01, d[2]);   // (x,y,z)
  g[1][0] = d[0];             g[1][1] = cmul(e02, d[1]);   g[1][2] = cmul(e[0], d[2]);  // (x,z,y)
  g[2][0] = cmul(e[1], d[0]); g[2][1] = d[1];              g[2][2] = cmul(e01, d[2]);   // (y,x,z)
  g[3][0] = cmul(e12, d[0]);  g[3][1] = d[1];              g[3][2] = cmul(e[1], d[2]);  // (y,z,x)
  g[4][0] = cmul(e[2], d[0]); g[4][1] = cmul(e02, d[1]);   g[4][2] = d[2];              // (z,x,y)
  g[5][0] = cmul(e12, d[0]);  g[5][1] = cmul(e[2], d[1]);  g[5][2] = d[2];              // (z,y,x)
  // M = B^H B = 1/2 sum_t (|g|^2 I + g g^H)
  T mdiag[3] = {0, 0, 0};
  C m01 = mkc<T>(0, 0), m02 = mkc<T>(0, 0), m12 = mkc<T>(0, 0);
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const T a0 = cabs2(g[t][0]), a1 = cabs2(g[t][1]), a2 = cabs2(g[t][2]);
    const T nn = a0 + a1 + a2;
    mdiag[0] += (T)0.5 * (nn + a0);
    mdiag[1] += (T)0.5 * (nn + a1);
    mdiag[2] += (T)0.5 * (nn + a2);
    m01 = cadd(m01, cscale(cmul(g[t][0], cconj(g[t][1])), (T)0.5));
    m02 = cadd(m02, cscale(cmul(g[t][0], cconj(g[t][2])), (T)0.5));
    m12 = cadd(m12, cscale(cmul(g[t][1], cconj(g[t][2])), (T)0.5));
  }
  const T r2 = (T)kInvSqrt2;
  C t3[3];
  if (mode == P_NODAL_IN || mode == P_SOLVE) {
    t3[0] = col[0]; t3[1] = col[LD]; t3[2] = col[2 * LD];
  } else {
    // t = B^H s: t_j = sum_t sum_a conj(g_ta) sigma_t,aj
    t3[0] = t3[1] = t3[2] = mkc<T>(0, 0);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const C* sp = col + 6 * t * LD;
      const C sxx = sp[0], syy = sp[LD], szz = sp[2 * LD];
      const C syz = cscale(sp[3 * LD], r2), sxz = cscale(sp[4 * LD], r2), sxy = cscale(sp[5 * LD], r2);
      t3[0] = cadd(t3[0], cadd(cadd(cjmul(g[t][0], sxx), cjmul(g[t][1], sxy)), cjmul(g[t][2], sxz)));
      t3[1] = cadd(t3[1], cadd(cadd(cjmul(g[t][0], sxy), cjmul(g[t][1], syy)), cjmul(g[t][2], syz)));
      t3[2] = cadd(t3[2], cadd(cadd(cjmul(g[t][0], sxz), cjmul(g[t][1], syz)), cjmul(g[t][2], szz)));
    }
  }
  // w = M^-1 t by the adjugate of the Hermitian matrix
  // M = [[A, m01, m02], [conj m01, B, m12], [conj m02, conj m12, Cc]]
  const T A = mdiag[0], B = mdiag[1], Cc = mdiag[2];
  const T A00 = B * Cc - cabs2(m12);
  const T A11 = A * Cc - cabs2(m02);
  const T A22 = A * B - cabs2(m01);
  // adj[0][1] = m02 conj(m12) - m01 Cc ; adj[0][2] = m01 m12 - m02 B ; adj[1][2] = m02 conj(m01) - A m12
  const C A01 = csub(cmul(m02, cconj(m12)), cscale(m01, Cc));
  const C A02 = csub(cmul(m01, m12), cscale(m02, B));
  const C A12 = csub(cmul(m02, cconj(m01)), cscale(m12, A));
  const T det = A * A00 + (cmul(m01, cconj(A01))).x + (cmul(m02, cconj(A02))).x;
  const T id = scale / det;
  C w[3];
  w[0] = cscale(cadd(cadd(cscale(t3[0], A00), cmul(A01, t3[1])), cmul(A02, t3[2])), id);
  w[1] = cscale(cadd(cadd(cjmul(A01, t3[0]), cscale(t3[1], A11)), cmul(A12, t3[2])), id);
  w[2] = cscale(cadd(cadd(cjmul(A02, t3[0]), cjmul(A12, t3[1])), cscale(t3[2], A22)), id);
  if (mode == P_NODAL_OUT || mode == P_SOLVE) {
    col[0] = w[0]; col[LD] = w[1]; col[2 * LD] = w[2];
    return;
  }
  // eps^ = B w: Mandel components of sym(g_t (x) w)
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    C* sp = col + 6 * t * LD;
    sp[0] = cmul(g[t][0], w[0]);
    sp[LD] = cmul(g[t][1], w[1]);
    sp[2 * LD] = cmul(g[t][2], w[2]);
    sp[3 * LD] = cscale(cadd(cmul(g[t][1], w[2]), cmul(g[t][2], w[1])), r2);
    sp[4 * LD] = cscale(cadd(cmul(g[t][0], w[2]), cmul(g[t][2], w[0])), r2);
    sp[5 * LD] = cscale(cadd(cmul(g[t][0], w[1]), cmul(g[t][1], w[0])), r2);
  }
}

// The same projection done by a pair of adjacent lanes: lane half h handles
// tetrahedra 3h..3h+2 (their gradients, their share of B^H B and of
// t = B^H s), the pair exchanges its partial sums by warp shuffle, both
// solve the 3x3 system, and each writes the outputs of its own tetrahedra.
// All 32 lanes of a warp must call it together (it exchanges partial sums
// with __shfl_xor_sync over the full warp): the k = 0 wavevector is handled by
// the `zero` flag, which only changes what is written at the end.
template <typename T, int LD>
__device__ __forceinline__ void project_3d_pair(cplx<T>* col, const cplx<T>* e, const T* ih, T scale, int mode,
                                                int half, bool zero) {
  using C = cplx<T>;
  const C one = mkc<T>(1, 0);
  C d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = cscale(csub(e[i], one), ih[i]);
  const C e01 = cmul(e[0], e[1]), e02 = cmul(e[0], e[2]), e12 = cmul(e[1], e[2]);
  // gradients of this lane's tetrahedra {0, e_a, e_a+e_b, 1}
  C g[3][3];
  if (half == 0) {
    g[0][0] = d[0];             g[0][1] = cmul(e[0], d[1]);  g[0][2] = cmul(e01, d[2]);   // (x,y,z)
    g[1][0] = d[0];             g[1][1] = cmul(e02, d[1]);   g[1][2] = cmul(e[0], d[2]);  // (x,z,y)
    g[2][0] = cmul(e[1], d[0]); g[2][1] = d[1];              g[2][2] = cmul(e01, d[2]);   // (y,x,z)
  } else {
    g[0][0] = cmul(e12, d[0]);  g[0][1] = d[1];              g[0][2] = cmul(e[1], d[2]);  // (y,z,x)
    g[1][0] = cmul(e[2], d[0]); g[1][1] = cmul(e02, d[1]);   g[1][2] = d[2];              // (z,x,y)
    g[2][0] = cmul(e12, d[0]);  g[2][1] = cmul(e[2], d[1]);  g[2][2] = d[2];              // (z,y,x)
  }
  // partial M = B^H B over this lane's tetrahedra
  T md[3] = {0, 0, 0};
  C m01 = mkc<T>(0, 0), m02 = mkc<T>(0, 0), m12 = mkc<T>(0, 0);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const T a0 = cabs2(g[t][0]), a1 = cabs2(g[t][1]), a2 = cabs2(g[t][2]);
    const T nn = a0 + a1 + a2;
    md[0] += (T)0.5 * (nn + a0);
    md[1] += (T)0.5 * (nn + a1);
    md[2] += (T)0.5 * (nn + a2);
    m01 = cadd(m01, cscale(cmul(g[t][0], cconj(g[t][1])), (T)0.5));
    m02 = cadd(m02, cscale(cmul(g[t][0], cconj(g[t][2])), (T)0.5));
    m12 = cadd(m12, cscale(cmul(g[t][1], cconj(g[t][2])), (T)0.5));
  }
  const T r2 = (T)kInvSqrt2;
  C t3[3];
  cplx<T>* own = col + 18 * half * LD;  // rows of this lane's tetrahedra
  const bool nodal_in = (mode == P_NODAL_IN || mode == P_SOLVE);
  if (nodal_in) {
    t3[0] = col[0]; t3[1] = col[LD]; t3[2] = col[2 * LD];
  } else {
    t3[0] = t3[1] = t3[2] = mkc<T>(0, 0);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const C* sp = own + 6 * t * LD;
      const C sxx = sp[0], syy = sp[LD], szz = sp[2 * LD];
      const C syz = cscale(sp[3 * LD], r2), sxz = cscale(sp[4 * LD], r2), sxy = cscale(sp[5 * LD], r2);
      t3[0] = cadd(t3[0], cadd(cadd(cjmul(g[t][0], sxx), cjmul(g[t][1], sxy)), cjmul(g[t][2], sxz)));
      t3[1] = cadd(t3[1], cadd(cadd(cjmul(g[t][0], sxy), cjmul(g[t][1], syy)), cjmul(g[t][2], syz)));
      t3[2] = cadd(t3[2], cadd(cadd(cjmul(g[t][0], sxz), cjmul(g[t][1], syz)), cjmul(g[t][2], szz)));
    }
  }
  // pair sums
  auto xs = [](T v) { return v + __shfl_xor_sync(0xffffffffu, v, 1); };
#pragma unroll
  for (int i = 0; i < 3; ++i) md[i] = xs(md[i]);
  m01.x = xs(m01.x); m01.y = xs(m01.y);
  m02.x = xs(m02.x); m02.y = xs(m02.y);
  m12.x = xs(m12.x); m12.y = xs(m12.y);
  if (!nodal_in) {
#pragma unroll
    for (int i = 0; i < 3; ++i) { t3[i].x = xs(t3[i].x); t3[i].y = xs(t3[i].y); }
  }
  const T A = md[0], B = md[1], Cc = md[2];
  const T A00 = B * Cc - cabs2(m12);
  const T A11 = A * Cc - cabs2(m02);
  const T A22 = A * B - cabs2(m01);
  const C A01 = csub(cmul(m02, cconj(m12)), cscale(m01, Cc));
  const C A02 = csub(cmul(m01, m12), cscale(m02, B));
  const C A12 = csub(cmul(m02, cconj(m01)), cscale(m12, A));
  const T det = A * A00 + (cmul(m01, cconj(A01))).x + (cmul(m02, cconj(A02))).x;
  const T id = scale / det;
  C w[3];
  w[0] = cscale(cadd(cadd(cscale(t3[0], A00), cmul(A01, t3[1])), cmul(A02, t3[2])), id);
  w[1] = cscale(cadd(cadd(cjmul(A01, t3[0]), cscale(t3[1], A11)), cmul(A12, t3[2])), id);
  w[2] = cscale(cadd(cadd(cjmul(A02, t3[0]), cjmul(A12, t3[1])), cscale(t3[2], A22)), id);
  const bool nodal_out = (mode == P_NODAL_OUT || mode == P_SOLVE);
  if (zero) {
    // k = 0: G(0) = 0, the fluctuation has no mean (w is not finite here)
    const C z = mkc<T>(0, 0);
    if (nodal_out) {
      if (half == 0) { col[0] = z; col[LD] = z; col[2 * LD] = z; }
    } else {
#pragma unroll
      for (int r = 0; r < 18; ++r) own[r * LD] = z;
    }
    return;
  }
  if (nodal_out) {
    if (half == 0) { col[0] = w[0]; col[LD] = w[1]; col[2 * LD] = w[2]; }
    return;
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    C* sp = own + 6 * t * LD;
    sp[0] = cmul(g[t][0], w[0]);
    sp[LD] = cmul(g[t][1], w[1]);
    sp[2 * LD] = cmul(g[t][2], w[2]);
    sp[3 * LD] = cscale(cadd(cmul(g[t][1], w[2]), cmul(g[t][2], w[1])), r2);
    sp[4 * LD] = cscale(cadd(cmul(g[t][0], w[2]), cmul(g[t][2], w[0])), r2);
    sp[5 * LD] = cscale(cadd(cmul(g[t][0], w[1]), cmul(g[t][1], w[0])), r2);
  }
}

// Row stride of the pass C buffer: at least the FFT's leading dimension, and
// chosen so that the two lanes of a wavevector (rows c and c + 18, same
// column) fall into different halves of a shared-memory bank window: the row
// offset 18 LD sizeof(complex) is then an odd multiple of 64 bytes and the
// lane-pair projection's accesses are free of bank conflicts.
template <typename T, int NZ, int V = 0> __host__ __device__ constexpr int pass_c_ld() {
  constexpr int base = FftSplit<NZ, V>::LD;
  constexpr int mod = sizeof(T) == 4 ? 8 : 4, want = sizeof(T) == 4 ? 4 : 2;
  return base + ((want - base % mod) + mod) % mod;
}

// grid (n_x/2+1, n_y, L): one (k_x, k_y) pencil of all components per block.
template <typename T, int NZ, int NT, int V = 0>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT <= 576) ? 2 : 1) pass_c_3d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int M = 36;
  constexpr int LD = pass_c_ld<T, NZ, V>();
  static_assert((18 * LD * (int)sizeof(cplx<T>)) % 128 == 64, "lane pairs must not share a bank");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [M][LD]
  const int kx = blockIdx.x, ky = blockIdx.y, l = blockIdx.z;
  const int ny = a.n[1], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int cin = (a.pmode == P_NODAL_IN || a.pmode == P_SOLVE) ? 3 : M;
  const int cout = (a.pmode == P_NODAL_OUT || a.pmode == P_SOLVE) ? 3 : M;
  const int64_t stride_c = (int64_t)KX * ny * NZ;
  C* pen = a.spec2 + (int64_t)l * M * stride_c + ((int64_t)kx * ny + ky) * NZ;
  // L2 prefetch of the later block's pencil (see grid_ahead): one request of
  // NZ values per component
  int kx2, ky2, l2;
  if (a.pf_ahead > 0 && threadIdx.x < M && grid_ahead(a, kx2, ky2, l2) && slot_runs(a, l2))
    prefetch_l2_bulk(a.spec2 + (int64_t)l2 * M * stride_c + ((int64_t)kx2 * ny + ky2) * NZ + threadIdx.x * stride_c,
                     (unsigned)(NZ * sizeof(C)));
  auto ld_g = [&](int c, int z) -> C { return pen[c * stride_c + z]; };
  auto st_s = [&](int c, int k, C v) { buf[c * LD + k] = v; };
  if (cin == M) fft4<T, NZ, M, LD, NT, -1, false, true, false, false, V>(buf, a.tw[2], ld_g, st_s);
  else fft4<T, NZ, 3, LD, NT, -1, false, true, false, false, V>(buf, a.tw[2], ld_g, st_s);
  C e[3];
  e[0] = a.ph[0][kx];
  e[1] = a.ph[1][ky];
  // two lanes per wavevector (NT >= 2 NZ, and 2 NZ is a whole number of warps)
  static_assert(NT >= 2 * NZ && (2 * NZ) % 32 == 0, "pass C needs two lanes per wavevector");
  if (threadIdx.x < 2 * NZ) {  // whole warps: every lane of them calls the pair projection
    const int kz = threadIdx.x >> 1, half = threadIdx.x & 1;
    e[2] = a.ph[2][kz];
    project_3d_pair<T, LD>(buf + kz, e, a.ih, a.inv_n, a.pmode, half, kx == 0 && ky == 0 && kz == 0);
  }
  __syncthreads();
  auto ld_s = [&](int c, int z) -> C { return buf[c * LD + z]; };
  auto st_g = [&](int c, int k, C v) { pen[c * stride_c + k] = v; };
  if (cout == M) fft4<T, NZ, M, LD, NT, +1, true, false, false, false, V>(buf, a.tw[2], ld_s, st_g);
  else fft4<T, NZ, 3, LD, NT, +1, true, false, false, false, V>(buf, a.tw[2], ld_s, st_g);
}

// Pass C for the nodal solve w^ = (B^H B)^-1 f^ (P_SOLVE, 3 components in
// and out): P pencils (k_x, k_y0 + i), i < P, per block, so that a block has
// as many transforms as the 36-component pass.  Row b of the buffer is
// component b % 3 of pencil b / 3.  grid (n_x/2+1, n_y/P, L).
template <typename T, int NZ, int P, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) pass_c_3d_nodal(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int M = 36, R = 3 * P;
  constexpr int LD = FftSplit<NZ>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [R][LD]
  const int kx = blockIdx.x, ky0 = blockIdx.y * P, l = blockIdx.z;
  const int ny = a.n[1], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t stride_c = (int64_t)KX * ny * NZ;
  C* base = a.spec2 + (int64_t)l * M * stride_c + ((int64_t)kx * ny + ky0) * NZ;
  auto ld_g = [&](int b, int z) -> C { return base[(b % 3) * stride_c + (b / 3) * NZ + z]; };
  auto st_s = [&](int b, int k, C v) { buf[b * LD + k] = v; };
  fft4<T, NZ, R, LD, NT, -1, false, true, false, false>(buf, a.tw[2], ld_g, st_s);
  for (int i = threadIdx.x; i < P * NZ; i += NT) {
    const int pc = i / NZ, kz = i % NZ;
    C* col = buf + 3 * pc * LD + kz;
    if (kx == 0 && ky0 + pc == 0 && kz == 0) {
      // k = 0: the nodal solve has no mean (w^(0) = 0)
      col[0] = col[LD] = col[2 * LD] = mkc<T>(0, 0);
    } else {
      const C e[3] = {a.ph[0][kx], a.ph[1][ky0 + pc], a.ph[2][kz]};
      project_3d<T, LD>(col, e, a.ih, a.inv_n, P_SOLVE);
    }
  }
  __syncthreads();
  auto ld_s = [&](int b, int z) -> C { return buf[b * LD + z]; };
  auto st_g = [&](int b, int k, C v) { base[(b % 3) * stride_c + (b / 3) * NZ + k] = v; };
  fft4<T, NZ, R, LD, NT, +1, true, false, false, false>(buf, a.tw[2], ld_s, st_g);
}

// Pass C for one evaluation point per voxel (the derivatives of Secs. 2.3-2.5,
// m = 6): P = 6 pencils (k_x, k_y0 + i) of the 6 components per block, so
// that a block has the 36 transforms of the finite-element pass; row b is
// component b % 6 of pencil b / 6.  grid (n_x/2+1, ceil(n_y/P), L).
template <typename T, int NZ, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) pass_c_3d_q1(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int P = 6, R = 36;
  constexpr int LD = FftSplit<NZ>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [R][LD]
  const int kx = blockIdx.x, ky0 = blockIdx.y * P, l = blockIdx.z;
  const int ny = a.n[1], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t stride_c = (int64_t)KX * ny * NZ;
  C* base = a.spec2 + (int64_t)l * a.m * stride_c + ((int64_t)kx * ny + ky0) * NZ;
  auto ld_g = [&](int b, int z) -> C {
    return (ky0 + b / 6 < ny) ? base[(b % 6) * stride_c + (b / 6) * NZ + z] : mkc<T>(0, 0);
  };
  auto st_s = [&](int b, int k, C v) { buf[b * LD + k] = v; };
  fft4<T, NZ, R, LD, NT, -1, false, true, false, false>(buf, a.tw[2], ld_g, st_s);
  for (int i = threadIdx.x; i < P * NZ; i += NT) {
    const int pc = i / NZ, kz = i % NZ, ky = ky0 + pc;
    if (ky >= ny) continue;
    C sv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) sv[c] = buf[(6 * pc + c) * LD + kz];
    if (kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
      for (int c = 0; c < 6; ++c) sv[c] = mkc<T>(0, 0);
    } else {
      const int j[3] = {kx, ky, kz};
      const C e[3] = {a.ph[0][kx], a.ph[1][ky], a.ph[2][kz]};
      C g[2][3];
      const int nq = deriv_symbols<T, 3>(a.deriv, j, a.n, e, a.ih, g);
      project_generic<T, 3>(sv, g, nq, a.inv_n);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) buf[(6 * pc + c) * LD + kz] = sv[c];
  }
  __syncthreads();
  auto ld_s = [&](int b, int z) -> C { return buf[b * LD + z]; };
  auto st_g = [&](int b, int k, C v) {
    if (ky0 + b / 6 < ny) base[(b % 6) * stride_c + (b / 6) * NZ + k] = v;
  };
  fft4<T, NZ, R, LD, NT, +1, true, false, false, false>(buf, a.tw[2], ld_s, st_g);
}

// Pass C for finite strain (P_FINITE): one (k_x, k_y) pencil of the 54
// deformation-gradient components (6 tetrahedra x 3 x 3) per block.
// grid (n_x/2+1, n_y, L).
template <typename T, int NZ, int NT>
__global__ void __launch_bounds__(NT, 1) pass_c_3d_fs(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int R = 54;
  constexpr int LD = FftSplit<NZ>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [R][LD]
  const int kx = blockIdx.x, ky = blockIdx.y, l = blockIdx.z;
  const int ny = a.n[1], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t stride_c = (int64_t)KX * ny * NZ;
  C* pen = a.spec2 + (int64_t)l * a.m * stride_c + ((int64_t)kx * ny + ky) * NZ;
  auto ld_g = [&](int c, int z) -> C { return pen[c * stride_c + z]; };
  auto st_s = [&](int c, int k, C v) { buf[c * LD + k] = v; };
  fft4<T, NZ, R, LD, NT, -1, false, true, false, false>(buf, a.tw[2], ld_g, st_s);
  for (int kz = threadIdx.x; kz < NZ; kz += NT) {
    const C e[3] = {a.ph[0][kx], a.ph[1][ky], a.ph[2][kz]};
    C g[6][3];
    fe_gradients<T, 3>(e, a.ih, g);
    auto col = [&](int c) -> C& { return buf[c * LD + kz]; };
    project_finite<T, 3, 6>(col, g, a.inv_n, kx == 0 && ky == 0 && kz == 0);
  }
  __syncthreads();
  auto ld_s = [&](int c, int z) -> C { return buf[c * LD + z]; };
  auto st_g = [&](int c, int k, C v) { pen[c * stride_c + k] = v; };
  fft4<T, NZ, R, LD, NT, +1, true, false, false, false>(buf, a.tw[2], ld_s, st_g);
}

// ---------------------------------------------------------------- pass E
// grid (n_y/TY, n_z, L*G): G = 6 tetrahedra (6 components each) or one group
// of the 3 nodal components (E_NODAL); inverse real FFT along x and update.
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT <= 384) ? 3 : 1) pass_e_3d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int KX = NX / 2 + 1;
  constexpr int GE = 6;
  constexpr int LD = ae_ld<NX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [GE][NP][LD]
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const bool nodal = (a.emode == E_NODAL || a.emode == E_NOUT);
  const int G = nodal ? 1 : a.nq;
  const int l = blockIdx.z / G, grp = blockIdx.z % G;
  const int z = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1], nz = a.n[2];
  const int64_t N = a.N;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int ge = nodal ? 3 : GE;
  const int c0 = nodal ? 0 : grp * GE;
  // the r rows this tile updates after its inverse FFT: start their DRAM reads
  // now so that they overlap the spectrum loads and the transform (measured at
  // 256^3: pass E 1.92 -> 1.88 ms; the same prefetch slowed the 2D pass E, whose
  // 4 KB rows compete with the spectrum loads at the start of the block)
  if (a.emode == E_CG)
    prefetch_rows_l2<T, NX>(a.r + ((int64_t)l * a.m + c0) * N + ((int64_t)z * ny + y0) * NX, ge, TY, N);
  if (a.pf_ahead > 0 && a.emode == E_CG && !nodal) pass_e_prefetch_ahead<T, NX, TY>(a, G);

  pass_e_unpack<T, NX, TY, NT, LD>(buf, a.spec + ((((int64_t)l * a.m + c0) * KX) * nz + z) * ny + y0, ge,
                                   (int64_t)KX * nz * ny, (int64_t)nz * ny);
  __syncthreads();
  T acc = 0;
  const T alpha = (a.emode == E_CG) ? (T)cg->alpha : (T)0;
  auto ld_s = [&](int b, int x) -> C { return buf[b * LD + x]; };
  PassEStore<T, NX, NP> st{&a, ge, ((int64_t)z * ny + y0) * NX, ((int64_t)l * a.m + c0) * N, (int64_t)l * 3 * N,
                           alpha, &acc};
  fft4<T, NX, GE * NP, LD, NT, +1, true, false, false, false, 0, decltype(ld_s), decltype(st), true>(buf, a.tw[0],
                                                                                                  ld_s, st);

  if (a.emode == E_CG || a.emode == E_INIT) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y * G;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * grp);
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(s, part, &cg->cnt_e, blk, nblk, &flag)) {
      const double rr = sum_partials<NT>(part, nblk, red);
      if (threadIdx.x == 0) finish_rr(cg, rr, a.emode == E_INIT);
    }
  }
}

// ------------------------------------------------------------ launchers
template <typename T> struct Tile3D;
template <> struct Tile3D<float> { static constexpr int TY = 8; static constexpr int TZB = 16; };
template <> struct Tile3D<double> { static constexpr int TY = 4; static constexpr int TZB = 8; };

template <typename T> constexpr int tile_rows3(int v) {
  return v == 1 ? Tile3D<T>::TY / 2 : v == 2 ? Tile3D<T>::TY * 2 : Tile3D<T>::TY;
}

// Load units of a pass A tile (see pass_a_load: two rows x one 16-byte vector
// of every component of one half of an element).
template <typename T, int NX, int TY> constexpr int pass_a_units3() { return 2 * (TY / 2) * (NX / Vec16<T>::n); }
template <int A, int B> constexpr int max_i() { return A > B ? A : B; }

// Prefetch distance (blocks ahead, see grid_ahead): the blocks resident at once
// (occ per SM x SMs) divided by div.  What pays is about 4 to 10 MB of
// prefetched rows in flight, so the divisor depends on a block's input.
// Measured at 256^3 (FP32, ms per CG iteration):
//   pass A (152 KB per block, three blocks per SM), div 16 (28 blocks): 2.88
//     without, 2.53 at div 16, 2.56 at div 32 to 152, 2.62 at div 8 and 3.26
//     at div 2 (35 MB in flight crowd L2);
//   pass B (32 KB per block): 0.86 without, 0.81 / 0.77 / 0.72 / 0.69 / 0.72
//     at div 16 / 8 / 4 / 2 / 1;
//   pass C (72 KB per block): 1.52 without, 1.55 / 1.53 / 1.47 / 1.41 / 1.43;
//   pass D (32 KB per block, scattered z-chunks): 0.85 without, 0.83 / 0.82 /
//     0.82 / 0.82 / 0.84;
//   pass E (tile variant 4, 97 KB per block): 1.82 without, 1.80 at div 16, 8
//     and 4, 1.87 at div 2 (the pipelined variant 3, 1.74, stays faster).
inline int prefetch_distance(int occ, int div) {
  const int d = occ * device_sm_count() / div;
  return d > 1 ? d : 1;
}

template <typename T, int NX, int TY, bool BY_UNITS = false>
cudaError_t launch_a_3d_t(const PassArgs<T>& a, cudaStream_t s, bool ahead = false) {
  constexpr int NF = fft_threads<NX, 6 * (TY / 2)>();
  constexpr int NU = (pass_a_units3<T, NX, TY>() + 31) / 32 * 32;
  constexpr int NT = BY_UNITS ? (max_i<NF, NU>() > 1024 ? NF : max_i<NF, NU>()) : NF;
  const size_t sm = sizeof(cplx<T>) * 6 * (TY / 2) * ae_ld<NX>();
  auto k = pass_a_3d<T, NX, TY, NT>;
  static DeviceOnce attr;
  static int occ[kMaxDevices] = {0};
  const int dev = current_device();
  attr.run(dev, [&] {
    set_smem_attrs(k, sm);
    if (dev >= 0 && dev < kMaxDevices) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[dev], k, NT, sm);
  });
  dim3 grid(a.n[1] / TY, a.n[2], a.L * (a.amode == A_NODAL ? 1 : a.nq));
  if (ahead) {
    PassArgs<T> b = a;
    b.pf_ahead = prefetch_distance((dev >= 0 && dev < kMaxDevices) ? occ[dev] : 0, 16);
    k<<<grid, NT, sm, s>>>(b);
  } else {
    k<<<grid, NT, sm, s>>>(a);
  }
  return cudaGetLastError();
}
template <typename T, int NX, int TY>
cudaError_t launch_e_3d_t(const PassArgs<T>& a, cudaStream_t s, bool ahead = false) {
  constexpr int NT = fft_threads<NX, 6 * (TY / 2)>();
  const size_t sm = sizeof(cplx<T>) * 6 * (TY / 2) * ae_ld<NX>();
  auto k = pass_e_3d<T, NX, TY, NT>;
  static DeviceOnce attr;
  static int occ[kMaxDevices] = {0};
  const int dev = current_device();
  attr.run(dev, [&] {
    set_smem_attrs(k, sm);
    if (dev >= 0 && dev < kMaxDevices) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[dev], k, NT, sm);
  });
  dim3 grid(a.n[1] / TY, a.n[2], a.L * ((a.emode == E_NODAL || a.emode == E_NOUT) ? 1 : a.nq));
  if (ahead) {
    PassArgs<T> b = a;
    b.pf_ahead = prefetch_distance((dev >= 0 && dev < kMaxDevices) ? occ[dev] : 0, 16);
    k<<<grid, NT, sm, s>>>(b);
  } else {
    k<<<grid, NT, sm, s>>>(a);
  }
  return cudaGetLastError();
}
// Tile variants of pass A: 0 default rows per block, 1 half, 2 double (threads
// = the FFT's); 3 default rows and 4 half rows with one thread per load unit;
// 5 (FP32, n_x >= 128, CG iterations) the pipelined persistent pass with
// bulk-copied rows (pass3d_pipe.cuh); other modes of variant 5 use variant 0;
// 6 variant 0 with the L2 prefetch of a later block's rows.
template <typename T, int NX>
cudaError_t launch_a_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && NX >= 128) {
    if (a.var_a == 5 && a.amode == A_CG && a.L <= kPipeMaxL && a.n[1] >= 4) return launch_a_3d_pipe<NX>(a, s);
  }
  if constexpr (NX >= 64) {
    if (a.var_a == 1) return launch_a_3d_t<T, NX, tile_rows3<T>(1)>(a, s);
    if (a.var_a == 2 && a.n[1] >= tile_rows3<T>(2)) return launch_a_3d_t<T, NX, tile_rows3<T>(2)>(a, s);
    if (a.var_a == 3) return launch_a_3d_t<T, NX, tile_rows3<T>(0), true>(a, s);
    if (a.var_a == 4) return launch_a_3d_t<T, NX, tile_rows3<T>(1), true>(a, s);
    if (a.var_a == 6) return launch_a_3d_t<T, NX, tile_rows3<T>(0)>(a, s, true);
  }
  return launch_a_3d_t<T, NX, tile_rows3<T>(0)>(a, s);
}
// Tile variants of pass E: 0 default rows per block, 1 half, 2 double; 3
// (FP32, n_x >= 128, CG iterations, with the spectrum's tensor map) the
// pipelined persistent pass (pass3d_pipe.cuh); other modes of 3 use 0; 4
// variant 0 with the L2 prefetch of a later block's spectrum tile and rows.
template <typename T, int NX>
cudaError_t launch_e_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && NX >= 128) {
    if (a.var_e == 3 && a.emode == E_CG && a.tm_spec && a.L <= kPipeMaxL && a.n[1] >= kPipeETY)
      return launch_e_3d_pipe<NX>(a, s);
  }
  if constexpr (NX >= 64) {
    if (a.var_e == 1) return launch_e_3d_t<T, NX, tile_rows3<T>(1)>(a, s);
    if (a.var_e == 2 && a.n[1] >= tile_rows3<T>(2)) return launch_e_3d_t<T, NX, tile_rows3<T>(2)>(a, s);
    if (a.var_e == 4) return launch_e_3d_t<T, NX, tile_rows3<T>(0)>(a, s, true);
  }
  return launch_e_3d_t<T, NX, tile_rows3<T>(0)>(a, s);
}
template <typename T, int NY, bool FWD, int V>
cudaError_t launch_y_3d_v(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int TZB = Tile3D<T>::TZB;
  constexpr int NT = fft_threads<NY, TZB, V>();
  const size_t sm = sizeof(cplx<T>) * TZB * FftSplit<NY, V>::LDO;
  auto k = pass_y_3d<T, NY, TZB, NT, FWD, V>;
  static DeviceOnce attr;
  static int occ[kMaxDevices] = {0};
  const int dev = current_device();
  attr.run(dev, [&] {
    set_smem_attrs(k, sm);
    if (dev >= 0 && dev < kMaxDevices) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[dev], k, NT, sm);
  });
  const bool din = (a.pmode == P_NODAL_IN || a.pmode == P_SOLVE);
  const bool dout = (a.pmode == P_NODAL_OUT || a.pmode == P_SOLVE);
  const int Cc = FWD ? (din ? 3 : a.m) : (dout ? 3 : a.m);
  dim3 grid(a.n[2] / TZB, a.kx, a.L * Cc);
  if (sizeof(T) == 4) {
    PassArgs<T> b = a;
    b.pf_ahead = prefetch_distance((dev >= 0 && dev < kMaxDevices) ? occ[dev] : 0, 2);
    k<<<grid, NT, sm, s>>>(b, Cc);
  } else {
    k<<<grid, NT, sm, s>>>(a, Cc);
  }
  return cudaGetLastError();
}
// Split variant of the y transforms (passes B and D): a.var_y.
template <typename T, int NY, bool FWD>
cudaError_t launch_y_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  if constexpr (fft_split_count<NY>() > 1) {
    if (a.var_y == 1) return launch_y_3d_v<T, NY, FWD, 1>(a, s);
  }
  return launch_y_3d_v<T, NY, FWD, 0>(a, s);
}
template <typename T, int NY> cudaError_t launch_yf_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  return launch_y_3d_n<T, NY, true>(a, s);
}
template <typename T, int NY> cudaError_t launch_yb_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  return launch_y_3d_n<T, NY, false>(a, s);
}
// Pass C of the finite-element stress form with split variant V (a.var_c).
template <typename T, int NZ, int V>
cudaError_t launch_c_3d_v(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NT = fft_threads<NZ, 36, V>();
  const size_t sm = sizeof(cplx<T>) * 36 * pass_c_ld<T, NZ, V>();
  auto k = pass_c_3d<T, NZ, NT, V>;
  static DeviceOnce attr;
  static int occ[kMaxDevices] = {0};
  const int dev = current_device();
  attr.run(dev, [&] {
    set_smem_attrs(k, sm);
    if (dev >= 0 && dev < kMaxDevices) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[dev], k, NT, sm);
  });
  dim3 grid(a.kx, a.n[1], a.L);
  if (sizeof(T) == 4) {
    PassArgs<T> b = a;
    b.pf_ahead = prefetch_distance((dev >= 0 && dev < kMaxDevices) ? occ[dev] : 0, 2);
    k<<<grid, NT, sm, s>>>(b);
  } else {
    k<<<grid, NT, sm, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int NZ>
cudaError_t launch_c_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  if (a.pmode == P_SOLVE) {
    constexpr int P = 8;  // n_y >= 16
    constexpr int NTn = fft_threads<NZ, 3 * P>();
    const size_t smn = sizeof(cplx<T>) * 3 * P * FftSplit<NZ>::LD;
    auto kn = pass_c_3d_nodal<T, NZ, P, NTn>;
    static DeviceOnce attr_n;
    attr_n.run(current_device(), [&] { set_smem_attrs(kn, smn); });
    dim3 gridn(a.kx, a.n[1] / P, a.L);
    kn<<<gridn, NTn, smn, s>>>(a);
    return cudaGetLastError();
  }
  if (a.pmode == P_FINITE) {
    constexpr int NTf = fft_threads<NZ, 54>();
    const size_t smf = sizeof(cplx<T>) * 54 * FftSplit<NZ>::LD;
    if (smf > 227 * 1024) return cudaErrorInvalidConfiguration;   // FP64 at n_z = 256
    auto kf = pass_c_3d_fs<T, NZ, NTf>;
    static DeviceOnce attrf;
    attrf.run(current_device(), [&] { set_smem_attrs(kf, smf); });
    kf<<<dim3(a.kx, a.n[1], a.L), NTf, smf, s>>>(a);
    return cudaGetLastError();
  }
  if (a.nq == 1) {
    constexpr int NT1 = fft_threads<NZ, 36>();
    const size_t sm1 = sizeof(cplx<T>) * 36 * FftSplit<NZ>::LD;
    auto k1 = pass_c_3d_q1<T, NZ, NT1>;
    static DeviceOnce attr1;
    attr1.run(current_device(), [&] { set_smem_attrs(k1, sm1); });
    k1<<<dim3(a.kx, (a.n[1] + 5) / 6, a.L), NT1, sm1, s>>>(a);
    return cudaGetLastError();
  }
  if constexpr (fft_split_count<NZ>() > 1) {
    if (a.var_c == 1) return launch_c_3d_v<T, NZ, 1>(a, s);
  }
  return launch_c_3d_v<T, NZ, 0>(a, s);
}

#define RVE_DISPATCH_N3(nval, FN, ...)                     \
  switch (nval) {                                          \
    case 16: return FN<T, 16>(__VA_ARGS__);                \
    case 32: return FN<T, 32>(__VA_ARGS__);                \
    case 64: return FN<T, 64>(__VA_ARGS__);                \
    case 128: return FN<T, 128>(__VA_ARGS__);              \
    case 256: return FN<T, 256>(__VA_ARGS__);              \
    default: return cudaErrorInvalidValue;                 \
  }

template <typename T> cudaError_t launch_pass_a_3d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N3(a.n[0], launch_a_3d_n, a, s)
}
template <typename T> cudaError_t launch_pass_b_3d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N3(a.n[1], launch_yf_3d_n, a, s)
}
template <typename T> cudaError_t launch_pass_c_3d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N3(a.n[2], launch_c_3d_n, a, s)
}
template <typename T> cudaError_t launch_pass_d_3d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N3(a.n[1], launch_yb_3d_n, a, s)
}
template <typename T> cudaError_t launch_pass_e_3d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N3(a.n[0], launch_e_3d_n, a, s)
}

}  // namespace rve
