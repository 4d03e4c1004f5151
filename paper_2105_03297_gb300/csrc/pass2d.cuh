// 2D projected-operator passes (two linear triangles per pixel, Sec. 2.6).
//
// One application of q = G * (C : p) is three launches:
//   A  material (+ fused CG direction update and <p, C p>) and forward real
//      FFT along x; writes the half spectrum transposed, [l][c][k_x][y], so
//      that the next pass reads whole y-columns contiguously;
//   C  forward FFT along y, the projection G(k) = B (B^H B)^-1 B^H per
//      wavevector (k = 0 set to zero), inverse FFT along y, in place;
//   E  inverse real FFT along x, then r -= alpha q and <r, r> (q never
//      touches memory).  x += alpha p of iteration k is deferred to pass A of
//      iteration k+1, which reads p anyway (one vector stream less per
//      iteration); cg_finish_x applies the last one.
// DFT convention of Appendix A; the 1/N of the inverse is applied in pass C.
// Two real rows (y, y+1) share one complex FFT (X_y + i X_{y+1}).
#pragma once
#include "rve_internal.h"

namespace rve {

constexpr double kInvSqrt2 = 0.70710678118654752440;
}  // namespace rve
#include "deriv.cuh"
#include "finite.cuh"
namespace rve {

// CG scalars: last-block finalisation of <p, C p> (pass A)
__device__ __forceinline__ void finish_alpha(CgState* cg, double pq) {
  cg->pq = pq;
  if (!(pq > 0.0) || !isfinite(pq)) { cg->status = ST_BAD; cg->alpha = 0.0; }
  else cg->alpha = cg->rr / pq;
  cg->cnt_a = 0;
}
// ... and of <r, r> (pass E)
__device__ __forceinline__ void finish_rr(CgState* cg, double rr, bool init) {
  if (init) {
    cg->rr0 = rr; cg->rr = rr; cg->it = 0; cg->beta = 0.0;
    // a held slot (ST_HOLD) stays held until the host releases it
    cg->status = !isfinite(rr) ? ST_BAD : (rr == 0.0 ? ST_CONV : (cg->status == ST_HOLD ? ST_HOLD : ST_RUN));
  } else {
    cg->it += 1;
    if (!isfinite(rr)) { cg->status = ST_BAD; }
    else {
      cg->beta = rr / cg->rr;
      cg->rr = rr;
      if (rr <= cg->tol2 * cg->rr0) cg->status = ST_CONV;
      else if (cg->it >= cg->maxit) cg->status = ST_MAXIT;
    }
  }
  cg->cnt_e = 0;
}

// ------------------------------------------------------------------------
// Pass A body, shared by 2D (GS = 3 components per element) and 3D (GS = 6):
// stream TY rows of NX voxels starting at voxel v0, apply the material, and
// pack the stress of component j, rows (2 pr, 2 pr + 1), as one complex row
// buf[(j*NP + pr)*LD + x] = sigma(2 pr, x) + i sigma(2 pr + 1, x).  A thread
// handles a unit of two rows x VL columns (16-byte loads of both rows of every
// component in flight together; 2-complex stores to shared memory).  Returns
// this thread's share of <p, C p>.
template <typename T, int NX, int TY, int GS, int NT, int LD, int VL = Vec16<T>::n>
__device__ __forceinline__ T pass_a_load(const PassArgs<T>& a, cplx<T>* buf, int l, int c0, int64_t v0,
                                         bool nodal, T beta, T alpha_prev, bool use_old) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int D = (GS == 3) ? 2 : 3;
  // In 3D a unit covers either the three normal or the three shear components
  // of an element (the material couples only the normal ones through the
  // trace), which halves the registers a unit needs.
  constexpr int HALVES = (GS == 6) ? 2 : 1;
  constexpr int GH = GS / HALVES;
  constexpr int NU = HALVES * NP * (NX / VL);
  static_assert(LD % 2 == 0, "row starts must stay 16-byte aligned");
  static_assert(VL % 2 == 0, "units pair complex values");
  const int64_t N = a.N;
  T acc = 0;
  for (int i = threadIdx.x; i < NU; i += NT) {
    const int half = i / (NP * (NX / VL));
    const int iu = i % (NP * (NX / VL));
    const int pr = iu / (NX / VL), x0 = (iu % (NX / VL)) * VL;
    const int j0 = half * GH;
    const int64_t va = v0 + (int64_t)(2 * pr) * NX + x0;
    T pv[2][GH][VL];
    T ev[2][VL];
    if (nodal) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < GH; ++j) {
          if (j0 + j < a.dim) vloadn<T, VL>(pv[h][j], a.in + ((int64_t)l * a.dim + j0 + j) * N + va + h * NX);
          else {
#pragma unroll
            for (int q = 0; q < VL; ++q) pv[h][j][q] = 0;
          }
        }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (a.amode != A_BARE) vloadn<T, VL>(ev[h], a.E + (int64_t)(l / a.lcs) * N + va + h * NX);
#pragma unroll
        for (int j = 0; j < GH; ++j) {
          const int64_t idx = ((int64_t)l * a.m + c0 + j0 + j) * N + va + h * NX;
          if (a.amode == A_CG) {
            vloadn<T, VL>(pv[h][j], a.r + idx);
          } else if (a.amode == A_MACRO) {
#pragma unroll
            for (int q = 0; q < VL; ++q) pv[h][j][q] = (T)a.emac[l * GS + j0 + j];
          } else {
            vloadn<T, VL>(pv[h][j], a.in + idx);
          }
        }
      }
      if (a.amode == A_CG && use_old) {
        // deferred update of the previous iteration: x += alpha_prev p_old,
        // then the new direction p = r + beta p_old
        T po[2][GH][VL], xo[2][GH][VL];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < GH; ++j) {
            const int64_t idx = ((int64_t)l * a.m + c0 + j0 + j) * N + va + h * NX;
            vloadn<T, VL>(po[h][j], a.p + idx);
            vloadn<T, VL>(xo[h][j], a.x + idx);
          }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < GH; ++j) {
#pragma unroll
            for (int q = 0; q < VL; ++q) {
              pv[h][j][q] += beta * po[h][j][q];
              xo[h][j][q] += alpha_prev * po[h][j][q];
            }
            vstoren<T, VL>(a.x + ((int64_t)l * a.m + c0 + j0 + j) * N + va + h * NX, xo[h][j]);
          }
      }
      if (a.amode == A_CG) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < GH; ++j)
            vstoren<T, VL>(a.p + ((int64_t)l * a.m + c0 + j0 + j) * N + va + h * NX, pv[h][j]);
      }
    }
    T sv[2][GH][VL];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < VL; ++q) {
        if (nodal || a.amode == A_BARE) {
#pragma unroll
          for (int j = 0; j < GH; ++j) sv[h][j][q] = pv[h][j][q];
        } else {
          // isotropic material, unit-modulus Lame constants times E_v:
          // normal components lambda tr + 2 mu eps, shear components 2 mu eps
          const T e = ev[h][q];
          if (HALVES == 1 || half == 0) {
            T tr = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) tr += pv[h][j][q];
            tr *= a.lam;
#pragma unroll
            for (int j = 0; j < GH; ++j) sv[h][j][q] = (j < D) ? e * (tr + a.mu2 * pv[h][j][q]) : e * (a.mu2 * pv[h][j][q]);
          } else {
#pragma unroll
            for (int j = 0; j < GH; ++j) sv[h][j][q] = e * (a.mu2 * pv[h][j][q]);
          }
          if (a.amode == A_CG) {
#pragma unroll
            for (int j = 0; j < GH; ++j) acc += pv[h][j][q] * sv[h][j][q];
          }
        }
      }
#pragma unroll
    for (int j = 0; j < GH; ++j) {
      C* dst = buf + ((j0 + j) * NP + pr) * LD + x0;
#pragma unroll
      for (int q = 0; q < VL; q += 2)
        cstore2<T>(dst + q, mkc<T>(sv[0][j][q], sv[1][j][q]), mkc<T>(sv[0][j][q + 1], sv[1][j][q + 1]));
    }
  }
  return acc;
}

// Two-for-one post-processing of the packed rows and transposed store:
// spectrum element (k, y0 + 2 pr (+1)) of component c0 + j goes to
// base + j*comp_stride + k*k_stride + 2 pr (+1).
template <typename T, int NX, int TY, int NT, int LD>
__device__ __forceinline__ void pass_a_store(const cplx<T>* buf, int gs, cplx<T>* base, int64_t comp_stride,
                                             int64_t k_stride) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int KX = NX / 2 + 1;
  for (int i = threadIdx.x; i < gs * KX * NP; i += NT) {
    const int pr = i % NP, k = (i / NP) % KX, j = i / (NP * KX);
    const C* row = buf + (j * NP + pr) * LD;
    const C A = row[k];
    const C Bc = cconj(row[(NX - k) & (NX - 1)]);
    const C xa = cscale(cadd(A, Bc), (T)0.5);
    const C d = csub(A, Bc);
    const C xb = mkc<T>((T)0.5 * d.y, (T)-0.5 * d.x);
    cstore2<T>(base + j * comp_stride + (int64_t)k * k_stride + 2 * pr, xa, xb);
  }
}

// ---------------------------------------------------------------- pass A
// grid (n_y/TY, groups, L), groups = n_q element blocks (n_s components each)
// or one block of D nodal components (A_NODAL).
// Resident blocks per SM the register budget of pass A is sized for.
template <typename T, int NT> __host__ __device__ constexpr int pass_a2_min_blocks() {
  return sizeof(T) != 4 ? 1 : NT <= 512 ? 2 : 1;
}

// NT is either the FFT's thread count or (tile variants 3, 4) the number of
// load units of the tile, so that every thread streams exactly one unit.
// PAIR (n_x = 512 or 1024, tile variant 5): the x transform spreads each
// 32-point register FFT of its first step over a lane pair (smem_fft_pair),
// NT = 2 N1 per transform, three blocks per SM.
template <typename T, int NX, int TY, int NT, bool PAIR = false>
__global__ void __launch_bounds__(NT, PAIR ? 3 : pass_a2_min_blocks<T, NT>()) pass_a_2d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int GS = 3;
  constexpr int KX = NX / 2 + 1;
  constexpr int LD = ae_ld<NX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [GS][NP][LD]
  __shared__ double red[NT / 32];
  __shared__ int flag;

  const int l = blockIdx.z, grp = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1];
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const bool nodal = (a.amode == A_NODAL);
  const int c0 = nodal ? 0 : grp * 3;
  T beta = 0, alpha_prev = 0;
  bool use_old = false;
  if (a.amode == A_CG) { beta = (T)cg->beta; alpha_prev = (T)cg->alpha; use_old = cg->it > 0; }
  // the lane-pair variant runs three blocks per SM: units of two columns (8-byte
  // loads, as in 3D) keep the load phase within its registers
  const T acc = pass_a_load<T, NX, TY, GS, NT, LD, PAIR ? 2 : Vec16<T>::n>(a, buf, l, c0, (int64_t)y0 * NX, nodal,
                                                                          beta, alpha_prev, use_old);
  __syncthreads();
  if constexpr (PAIR) smem_fft_pair<T, NX, GS * NP, LD, NT, -1>(buf, a.tw[0]);
  else smem_fft<T, NX, GS * NP, LD, NT, -1>(buf, a.tw[0]);
  pass_a_store<T, NX, TY, NT, LD>(buf, nodal ? 2 : 3, a.spec + (((int64_t)l * a.m + c0) * KX) * ny + y0,
                                  (int64_t)KX * ny, ny);

  if (a.amode == A_CG) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y;
    const int blk = blockIdx.x + gridDim.x * blockIdx.y;
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
      const double pq = sum_partials<NT>(part, nblk, red);
      if (threadIdx.x == 0) finish_alpha(cg, pq);
    }
  }
}

// ---------------------------------------------------------------- pass C
// Projection of the m = 6 spectra at one wavevector, in place.
//   mode P_G:         s (6) -> B (B^H B)^-1 B^H s
//   mode P_NODAL_IN:  s[0..1] = f^ -> B (B^H B)^-1 f^   (6 out)
//   mode P_NODAL_OUT: s (6) -> (B^H B)^-1 B^H s           (2 out, in s[0..1])
template <typename T>
__device__ __forceinline__ void project_2d(cplx<T>* s, cplx<T> ex, cplx<T> ey, T ihx, T ihy, T scale, int mode) {
  using C = cplx<T>;
  const C one = mkc<T>(1, 0);
  C g[2][2];
  const C dx = cscale(csub(ex, one), ihx), dy = cscale(csub(ey, one), ihy);
  g[0][0] = dx; g[0][1] = dy;                       // nodes {00,10,01}
  g[1][0] = cmul(ey, dx); g[1][1] = cmul(ex, dy);   // nodes {11,01,10}
  // M = B^H B = 1/2 sum (|g|^2 I + g g^H)
  T m00 = 0, m11 = 0; C m01 = mkc<T>(0, 0);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const T ax = cabs2(g[q][0]), ay = cabs2(g[q][1]);
    m00 += ax + (T)0.5 * ay;
    m11 += (T)0.5 * ax + ay;
    m01 = cadd(m01, cscale(cmul(g[q][0], cconj(g[q][1])), (T)0.5));
  }
  C t0, t1;
  if (mode == P_NODAL_IN || mode == P_SOLVE) {
    t0 = s[0]; t1 = s[1];
  } else {
    // t = B^H s: t_j = sum_q sum_a conj(g_qa) sigma_q,aj
    t0 = mkc<T>(0, 0); t1 = mkc<T>(0, 0);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const C sxx = s[3 * q], syy = s[3 * q + 1], sxy = cscale(s[3 * q + 2], (T)kInvSqrt2);
      t0 = cadd(t0, cadd(cjmul(g[q][0], sxx), cjmul(g[q][1], sxy)));
      t1 = cadd(t1, cadd(cjmul(g[q][0], sxy), cjmul(g[q][1], syy)));
    }
  }
  const T det = m00 * m11 - cabs2(m01);
  const T id = scale / det;
  // w = M^-1 t,  M^-1 = [[m11, -m01], [-conj(m01), m00]] / det
  const C w0 = cscale(csub(cscale(t0, m11), cmul(m01, t1)), id);
  const C w1 = cscale(csub(cscale(t1, m00), cjmul(m01, t0)), id);
  if (mode == P_NODAL_OUT || mode == P_SOLVE) {
    s[0] = w0; s[1] = w1;
    return;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    s[3 * q] = cmul(g[q][0], w0);
    s[3 * q + 1] = cmul(g[q][1], w1);
    s[3 * q + 2] = cscale(cadd(cmul(g[q][0], w1), cmul(g[q][1], w0)), (T)kInvSqrt2);
  }
}

// grid (n_x/2+1, L); one k_x column of all six spectra per block.  The forward
// FFT reads the column straight from the spectrum, the inverse FFT writes it
// straight back; only the middle transposes and the projection use shared
// memory.
template <typename T, int NY, int NQ, int NT, int V = 0>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 1) pass_c_2d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int M = 3 * NQ;   // 6 for the finite elements and two-point Fourier, 3 for one point,
                              // 9 for finite-strain gradients (8 + padding)
  constexpr int LD = FftSplit<NY, V>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [M][LD]
  const int kx = blockIdx.x, l = blockIdx.y;
  const int KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int cin = (a.pmode == P_NODAL_IN || a.pmode == P_SOLVE) ? 2 : M;
  const int cout = (a.pmode == P_NODAL_OUT || a.pmode == P_SOLVE) ? 2 : M;
  C* col = a.spec + (((int64_t)l * M) * KX + kx) * NY;
  const int64_t cstride = (int64_t)KX * NY;
  auto ld_g = [&](int c, int y) -> C { return col[c * cstride + y]; };
  auto st_s = [&](int c, int k, C v) { buf[c * LD + k] = v; };
  if (cin == M) fft4<T, NY, M, LD, NT, -1, false, true, false, false, V>(buf, a.tw[1], ld_g, st_s);
  else fft4<T, NY, 2, LD, NT, -1, false, true, false, false, V>(buf, a.tw[1], ld_g, st_s);

  const C ex = a.ph[0][kx];
  for (int ky = threadIdx.x; ky < NY; ky += NT) {
    C s[M];
#pragma unroll
    for (int c = 0; c < M; ++c) s[c] = (c < cin) ? buf[c * LD + ky] : mkc<T>(0, 0);
    if constexpr (NQ == 3) {
      // finite strain: deformation gradients of the two triangles (+ padding)
      const C e2[2] = {ex, a.ph[1][ky]};
      C g[6][3];
      fe_gradients<T, 2>(e2, a.ih, g);
      auto col = [&](int c) -> C& { return s[c]; };
      project_finite<T, 2, 2>(col, g, a.inv_n, kx == 0 && ky == 0);
    } else if (kx == 0 && ky == 0) {
#pragma unroll
      for (int c = 0; c < M; ++c) s[c] = mkc<T>(0, 0);
    } else if (NQ == 2 && a.deriv == D_FE) {
      project_2d<T>(s, ex, a.ph[1][ky], a.ih[0], a.ih[1], a.inv_n, a.pmode);
    } else {
      const int j[2] = {kx, ky};
      const C e[2] = {ex, a.ph[1][ky]};
      C g[2][3];
      const int nq = deriv_symbols<T, 2>(a.deriv, j, a.n, e, a.ih, g);
      project_generic<T, 2>(s, g, nq, a.inv_n);
    }
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < cout) buf[c * LD + ky] = s[c];
  }
  __syncthreads();
  auto ld_s = [&](int c, int y) -> C { return buf[c * LD + y]; };
  auto st_g = [&](int c, int k, C v) { col[c * cstride + k] = v; };
  if (cout == M) fft4<T, NY, M, LD, NT, +1, true, false, false, false, V>(buf, a.tw[1], ld_s, st_g);
  else fft4<T, NY, 2, LD, NT, +1, true, false, false, false, V>(buf, a.tw[1], ld_s, st_g);
}

// Pass C for the nodal solve w^ = (B^H B)^-1 f^ (P_SOLVE, 2 components in and
// out): P k_x columns per block so that a block holds as many transforms as
// the 6-component pass.  Row b is component b % 2 of column kx0 + b / 2;
// columns past n_x/2 are skipped.  grid (ceil((n_x/2+1) / P), L).
template <typename T, int NY, int P, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) pass_c_2d_nodal(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int M = 6, R = 2 * P;
  constexpr int LD = FftSplit<NY>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [R][LD]
  const int kx0 = blockIdx.x * P, l = blockIdx.y;
  const int KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t cstride = (int64_t)KX * NY;
  C* base = a.spec + ((int64_t)l * M * KX + kx0) * NY;
  auto ld_g = [&](int b, int y) -> C {
    return (kx0 + b / 2 < KX) ? base[(b % 2) * cstride + (int64_t)(b / 2) * NY + y] : mkc<T>(0, 0);
  };
  auto st_s = [&](int b, int k, C v) { buf[b * LD + k] = v; };
  fft4<T, NY, R, LD, NT, -1, false, true, false, false>(buf, a.tw[1], ld_g, st_s);
  for (int i = threadIdx.x; i < P * NY; i += NT) {
    const int pc = i / NY, ky = i % NY, kx = kx0 + pc;
    if (kx >= KX) continue;
    C s2[M];
    s2[0] = buf[2 * pc * LD + ky];
    s2[1] = buf[(2 * pc + 1) * LD + ky];
    if (kx == 0 && ky == 0) {
      s2[0] = s2[1] = mkc<T>(0, 0);   // k = 0: the nodal solve has no mean
    } else {
      project_2d<T>(s2, a.ph[0][kx], a.ph[1][ky], a.ih[0], a.ih[1], a.inv_n, P_SOLVE);
    }
    buf[2 * pc * LD + ky] = s2[0];
    buf[(2 * pc + 1) * LD + ky] = s2[1];
  }
  __syncthreads();
  auto ld_s = [&](int b, int y) -> C { return buf[b * LD + y]; };
  auto st_g = [&](int b, int k, C v) {
    if (kx0 + b / 2 < KX) base[(b % 2) * cstride + (int64_t)(b / 2) * NY + k] = v;
  };
  fft4<T, NY, R, LD, NT, +1, true, false, false, false>(buf, a.tw[1], ld_s, st_g);
}

// ------------------------------------------------------------------------
// Pass E body shared by 2D and 3D: load the (k, y-pair) spectra of ge
// components into packed rows (component j at src + j*comp_stride +
// k*k_stride + y-offset, rows j*NP + pr), ready for the inverse FFT.
// Each thread has up to UB of its loads in flight before it writes any of
// them to shared memory (a load per loop trip would leave one in flight).
template <typename T, int NX, int TY, int NT, int LD>
__device__ __forceinline__ void pass_e_unpack(cplx<T>* buf, const cplx<T>* src, int ge, int64_t comp_stride,
                                              int64_t k_stride) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int KX = NX / 2 + 1;
  constexpr int UB = 8;
  const int total = ge * KX * NP;
  for (int i0 = threadIdx.x; i0 < total; i0 += UB * NT) {
    C ab[UB][2];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int i = i0 + u * NT;
      if (i < total) {
        const int pr = i % NP, k = (i / NP) % KX, j = i / (NP * KX);
        cload2<T>(ab[u], src + j * comp_stride + (int64_t)k * k_stride + 2 * pr);
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int i = i0 + u * NT;
      if (i < total) {
        const int pr = i % NP, k = (i / NP) % KX, j = i / (NP * KX);
        C xa = ab[u][0], xb = ab[u][1];
        if (k == 0 || k == NX / 2) { xa.y = 0; xb.y = 0; }  // C2R ignores these imaginary parts
        C* row = buf + (j * NP + pr) * LD;
        row[k] = mkc<T>(xa.x - xb.y, xa.y + xb.x);                                  // X_a + i X_b
        if (k > 0 && k < NX / 2) row[NX - k] = mkc<T>(xa.x + xb.y, xb.x - xa.y);    // conj(X_a) + i conj(X_b)
      }
    }
  }
}

// The inverse FFT of pass E hands each output q(b, x) (b = j*NP + pr: rows
// 2 pr and 2 pr + 1 of component j, real and imaginary part) to this update:
// CG: r -= alpha q and <r, r>; INIT: r = -q, x = 0; OUT: out = q; NODAL: u += q
// in FP64.  Consecutive threads handle consecutive x, so every access is
// coalesced.  idx0 / uidx0: offsets of the first component's [N] slab in the
// CG vectors / the FP64 nodal field; v0: first voxel of the tile.
template <typename T, int NX, int NP>
struct PassEStore {
  const PassArgs<T>* a;
  int ge;
  int64_t v0, idx0, uidx0;
  T alpha;
  T* acc;
  // outputs x = k2 + N2 k1 (k1 < N1) of rows (2 pr, 2 pr + 1) of component j:
  // all loads of r (or u) are issued before any store
  __device__ __forceinline__ void batch(int b, int k2, const cplx<T>* q) const {
    constexpr int N1 = FftSplit<NX>::N1, N2 = FftSplit<NX>::N2;
    const int j = b / NP, pr = b % NP;
    if (j >= ge) return;
    const int64_t off = (int64_t)j * a->N + v0 + (int64_t)(2 * pr) * NX + k2;
    const int em = a->emode;
    if (em == E_CG) {
      // chunks of up to 8 outputs: 16 loads in flight, bounded registers
      constexpr int CH = N1 < 8 ? N1 : 8;
      T* r = a->r + idx0 + off;
      T s = 0;
#pragma unroll
      for (int c0 = 0; c0 < N1; c0 += CH) {
        T rv[2][CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) { rv[0][k] = r[N2 * (c0 + k)]; rv[1][k] = r[NX + N2 * (c0 + k)]; }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
          rv[0][k] -= alpha * q[c0 + k].x;
          rv[1][k] -= alpha * q[c0 + k].y;
          s += rv[0][k] * rv[0][k] + rv[1][k] * rv[1][k];
          r[N2 * (c0 + k)] = rv[0][k];
          r[NX + N2 * (c0 + k)] = rv[1][k];
        }
      }
      *acc += s;
    } else if (em == E_INIT) {
      T* r = a->r + idx0 + off;
      T* x = a->x + idx0 + off;
      T s = 0;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        r[N2 * k1] = -q[k1].x;
        r[NX + N2 * k1] = -q[k1].y;
        x[N2 * k1] = 0;
        x[NX + N2 * k1] = 0;
        s += q[k1].x * q[k1].x + q[k1].y * q[k1].y;
      }
      *acc += s;
    } else if (em == E_NOUT) {
      T* o = a->out + uidx0 + off;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) { o[N2 * k1] = q[k1].x; o[NX + N2 * k1] = q[k1].y; }
    } else if (em == E_OUT) {
      T* o = a->out + idx0 + off;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) { o[N2 * k1] = q[k1].x; o[NX + N2 * k1] = q[k1].y; }
    } else {
      double* u = a->u64 + uidx0 + off;
      double uv[2][N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) { uv[0][k1] = u[N2 * k1]; uv[1][k1] = u[NX + N2 * k1]; }
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        u[N2 * k1] = uv[0][k1] + (double)q[k1].x;
        u[NX + N2 * k1] = uv[1][k1] + (double)q[k1].y;
      }
    }
  }
  __device__ __forceinline__ void operator()(int, int, cplx<T>) const {}
};

// ---------------------------------------------------------------- pass E
// grid (n_y/TY, groups, L): groups = n_q elements (3 components each) or one
// group of the D = 2 nodal components (E_NODAL); inverse real FFT along x.
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT <= 384) ? 2 : 1) pass_e_2d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int KX = NX / 2 + 1;
  constexpr int GE = 3;
  constexpr int LD = ae_ld<NX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [GE][NP][LD]
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int l = blockIdx.z, grp = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1];
  const int64_t N = a.N;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const bool nodal = (a.emode == E_NODAL || a.emode == E_NOUT);
  const int ge = nodal ? 2 : GE;
  const int c0 = nodal ? 0 : grp * GE;

  pass_e_unpack<T, NX, TY, NT, LD>(buf, a.spec + (((int64_t)l * a.m + c0) * KX) * ny + y0, ge, (int64_t)KX * ny, ny);
  __syncthreads();
  T acc = 0;
  const T alpha = (a.emode == E_CG) ? (T)cg->alpha : (T)0;
  auto ld_s = [&](int b, int x) -> C { return buf[b * LD + x]; };
  PassEStore<T, NX, NP> st{&a, ge, (int64_t)y0 * NX, ((int64_t)l * a.m + c0) * N, (int64_t)l * 2 * N, alpha, &acc};
  fft4<T, NX, GE * NP, LD, NT, +1, true, false, false, false, 0, decltype(ld_s), decltype(st), true>(buf, a.tw[0],
                                                                                                  ld_s, st);

  if (a.emode == E_CG || a.emode == E_INIT) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y;
    const int blk = blockIdx.x + gridDim.x * blockIdx.y;
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(s, part, &cg->cnt_e, blk, nblk, &flag)) {
      const double rr = sum_partials<NT>(part, nblk, red);
      if (threadIdx.x == 0) finish_rr(cg, rr, a.emode == E_INIT);
    }
  }
}

// x += alpha p for every load case that ran at least one iteration: the
// update the last CG iteration deferred.  grid (ceil(m N / (VL*NT)), L).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) cg_finish_x(PassArgs<T> a) {
  constexpr int VL = Vec16<T>::n;
  const int l = blockIdx.y;
  const CgState* cg = a.cg + l;
  if (!cg->active || cg->it == 0 || cg->status == ST_BAD) return;
  const T alpha = (T)cg->alpha;
  const int64_t nv = (int64_t)a.m * a.N / VL;
  const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (i >= nv) return;
  const int64_t idx = (int64_t)l * a.m * a.N + i * VL;
  T xv[VL], pv[VL];
  vload(xv, a.x + idx);
  // the factored form alternates the direction between p (even iterations) and p2 (odd)
  const T* pl = (a.p2 != nullptr && ((cg->it - 1) & 1)) ? a.p2 : a.p;
  vload(pv, pl + idx);
#pragma unroll
  for (int w = 0; w < VL; ++w) xv[w] += alpha * pv[w];
  vstore(a.x + idx, xv);
}

template <typename T> cudaError_t launch_cg_finish_x(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NT = 256;
  const int64_t nv = (int64_t)a.m * a.N / Vec16<T>::n;
  dim3 grid((unsigned)((nv + NT - 1) / NT), a.L);
  cg_finish_x<T, NT><<<grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------ launchers
template <typename T> struct Tile2D;
template <> struct Tile2D<float> { static constexpr int TY = 8; };
template <> struct Tile2D<double> { static constexpr int TY = 4; };

// Tile variants: rows per block TY = default, half, double (the autotuner
// times them on the live buffers and keeps the fastest).
template <typename T> constexpr int tile_rows(int v) {
  return v == 1 ? Tile2D<T>::TY / 2 : v == 2 ? Tile2D<T>::TY * 2 : Tile2D<T>::TY;
}

template <typename T, int NX, int TY, bool BY_UNITS = false, bool PAIR = false>
cudaError_t launch_a_2d_t(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NF = PAIR ? 2 * FftSplit<NX>::N1 * 3 * (TY / 2) : fft_threads<NX, 3 * (TY / 2)>();
  constexpr int NU = ((TY / 2) * (NX / Vec16<T>::n) + 31) / 32 * 32;   // load units of a tile
  constexpr int NT = (BY_UNITS && NU > NF && NU <= 1024) ? NU : NF;
  static_assert(NT <= 1024, "threads per block");
  const size_t sm = sizeof(cplx<T>) * 3 * (TY / 2) * ae_ld<NX>();
  auto k = pass_a_2d<T, NX, TY, NT, PAIR>;
  static DeviceOnce attr;
  attr.run(current_device(), [&] { set_smem_attrs(k, sm); });
  dim3 grid(a.n[1] / TY, a.amode == A_NODAL ? 1 : a.nq, a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int NX, int TY>
cudaError_t launch_e_2d_t(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NT = fft_threads<NX, 3 * (TY / 2)>();
  const size_t sm = sizeof(cplx<T>) * 3 * (TY / 2) * ae_ld<NX>();
  auto k = pass_e_2d<T, NX, TY, NT>;
  static DeviceOnce attr;
  attr.run(current_device(), [&] { set_smem_attrs(k, sm); });
  dim3 grid(a.n[1] / TY, (a.emode == E_NODAL || a.emode == E_NOUT) ? 1 : a.nq, a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}
// Tile variants of the 2D pass A: 0 default rows per block, 1 half, 2 double
// (threads = the FFT's); 3 default rows and 4 half rows with one thread per
// load unit; 5 (FP32, n_x = 512 or 1024) the lane-pair x transform with 384
// threads (default rows at 512, half rows at 1024).
template <typename T, int NX>
cudaError_t launch_a_2d_n(const PassArgs<T>& a, cudaStream_t s) {
  if constexpr ((NX == 512 || NX == 1024) && sizeof(T) == 4) {
    if (a.var_a == 5) return launch_a_2d_t<T, NX, NX == 1024 ? tile_rows<T>(1) : tile_rows<T>(0), false, true>(a, s);
  }
  if constexpr (NX >= 64) {
    if (a.var_a == 1) return launch_a_2d_t<T, NX, tile_rows<T>(1)>(a, s);
    if (a.var_a == 2 && a.n[1] >= tile_rows<T>(2)) return launch_a_2d_t<T, NX, tile_rows<T>(2)>(a, s);
    if (a.var_a == 3) return launch_a_2d_t<T, NX, tile_rows<T>(0), true>(a, s);
    if (a.var_a == 4) return launch_a_2d_t<T, NX, tile_rows<T>(1), true>(a, s);
  }
  return launch_a_2d_t<T, NX, tile_rows<T>(0)>(a, s);
}
// Tile variants of the 2D pass E: 0 default rows per block, 1 half, 2 double.
// (The lane-pair x transform of pass A's variant 5 made pass E slower at
// 1024^2: 0.091 against 0.083 ms per iteration for three load cases.)
template <typename T, int NX>
cudaError_t launch_e_2d_n(const PassArgs<T>& a, cudaStream_t s) {
  if constexpr (NX >= 64) {
    if (a.var_e == 1) return launch_e_2d_t<T, NX, tile_rows<T>(1)>(a, s);
    if (a.var_e == 2 && a.n[1] >= tile_rows<T>(2)) return launch_e_2d_t<T, NX, tile_rows<T>(2)>(a, s);
  }
  return launch_e_2d_t<T, NX, tile_rows<T>(0)>(a, s);
}
// Pass C of the finite elements (two triangles) with split variant V (a.var_c).
template <typename T, int NY, int V>
cudaError_t launch_c_2d_v(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NT = fft_threads<NY, 6, V>();
  const size_t sm = sizeof(cplx<T>) * 6 * FftSplit<NY, V>::LD;
  auto k = pass_c_2d<T, NY, 2, NT, V>;
  static DeviceOnce attr;
  attr.run(current_device(), [&] { set_smem_attrs(k, sm); });
  dim3 grid(a.kx, a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int NY>
cudaError_t launch_c_2d_n(const PassArgs<T>& a, cudaStream_t s) {
  if (a.pmode == P_SOLVE) {
    constexpr int P = 3;
    constexpr int NTn = fft_threads<NY, 2 * P>();
    const size_t smn = sizeof(cplx<T>) * 2 * P * FftSplit<NY>::LD;
    auto kn = pass_c_2d_nodal<T, NY, P, NTn>;
    static DeviceOnce attr_n;
    attr_n.run(current_device(), [&] { set_smem_attrs(kn, smn); });
    dim3 gridn((a.kx + P - 1) / P, a.L);
    kn<<<gridn, NTn, smn, s>>>(a);
    return cudaGetLastError();
  }
  if (a.nq == 3) {
    constexpr int NT3 = fft_threads<NY, 9>();
    const size_t sm3 = sizeof(cplx<T>) * 9 * FftSplit<NY>::LD;
    auto k3 = pass_c_2d<T, NY, 3, NT3>;
    static DeviceOnce attr3;
    attr3.run(current_device(), [&] { set_smem_attrs(k3, sm3); });
    k3<<<dim3(a.kx, a.L), NT3, sm3, s>>>(a);
    return cudaGetLastError();
  }
  if (a.nq == 1) {
    constexpr int NT1 = fft_threads<NY, 3>();
    const size_t sm1 = sizeof(cplx<T>) * 3 * FftSplit<NY>::LD;
    auto k1 = pass_c_2d<T, NY, 1, NT1>;
    static DeviceOnce attr1;
    attr1.run(current_device(), [&] { set_smem_attrs(k1, sm1); });
    k1<<<dim3(a.kx, a.L), NT1, sm1, s>>>(a);
    return cudaGetLastError();
  }
  if constexpr (fft_split_count<NY>() > 1) {
    if (a.var_c == 1) return launch_c_2d_v<T, NY, 1>(a, s);
  }
  return launch_c_2d_v<T, NY, 0>(a, s);
}

#define RVE_DISPATCH_N(nval, FN, ...)                      \
  switch (nval) {                                          \
    case 16: return FN<T, 16>(__VA_ARGS__);                \
    case 32: return FN<T, 32>(__VA_ARGS__);                \
    case 64: return FN<T, 64>(__VA_ARGS__);                \
    case 128: return FN<T, 128>(__VA_ARGS__);              \
    case 256: return FN<T, 256>(__VA_ARGS__);              \
    case 512: return FN<T, 512>(__VA_ARGS__);              \
    case 1024: return FN<T, 1024>(__VA_ARGS__);            \
    default: return cudaErrorInvalidValue;                 \
  }

template <typename T> cudaError_t launch_pass_a_2d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N(a.n[0], launch_a_2d_n, a, s)
}
template <typename T> cudaError_t launch_pass_e_2d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N(a.n[0], launch_e_2d_n, a, s)
}
template <typename T> cudaError_t launch_pass_c_2d(const PassArgs<T>& a, cudaStream_t s) {
  RVE_DISPATCH_N(a.n[1], launch_c_2d_n, a, s)
}

}  // namespace rve
