// 2D projected-operator passes (two linear triangles per pixel, Sec. 2.6).
//
// One application of q = G * (C : p) is three launches:
//   A  material (+ fused CG direction update and <p, C p>) and forward real
//      FFT along x; writes the half spectrum transposed, [l][c][k_x][y], so
//      that the next pass reads whole y-columns contiguously;
//   C  forward FFT along y, the projection G(k) = B (B^H B)^-1 B^H per
//      wavevector (k = 0 set to zero), inverse FFT along y, in place;
//   E  inverse real FFT along x, then x += alpha p, r -= alpha q and <r, r>
//      (q never touches memory).
// DFT convention of Appendix A; the 1/N of the inverse is applied in pass C.
#pragma once
#include "rve_internal.h"

namespace rve {

constexpr double kInvSqrt2 = 0.70710678118654752440;

// ---------------------------------------------------------------- pass A
// grid (n_y/TY, groups, L), groups = n_q element blocks (n_s components each)
// or one block of D nodal components (A_NODAL).
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT) pass_a_2d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;   // two real rows per complex row
  constexpr int GS = 3;        // components per block (n_s; D = 2 for nodal)
  constexpr int KX = NX / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [GS][NP][NX]
  __shared__ double red[NT / 32];
  __shared__ int flag;

  const int l = blockIdx.z, grp = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1];
  const int64_t N = a.N;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const bool nodal = (a.amode == A_NODAL);
  const int gs = nodal ? 2 : 3;
  const int c0 = nodal ? 0 : grp * 3;
  T beta = 0;
  bool use_old = false;
  if (a.amode == A_CG) { beta = (T)cg->beta; use_old = cg->it > 0; }
  T acc = 0;

  for (int i = threadIdx.x; i < TY * NX; i += NT) {
    const int yy = i / NX, xx = i % NX;
    const int64_t v = (int64_t)(y0 + yy) * NX + xx;
    T s[GS];
    if (nodal) {
      s[0] = a.in[((int64_t)l * 2 + 0) * N + v];
      s[1] = a.in[((int64_t)l * 2 + 1) * N + v];
      s[2] = 0;
    } else {
      T pv[GS];
#pragma unroll
      for (int j = 0; j < GS; ++j) {
        const int64_t idx = ((int64_t)l * a.m + c0 + j) * N + v;
        if (a.amode == A_CG) {
          T t = a.r[idx];
          if (use_old) t += beta * a.p[idx];
          a.p[idx] = t;
          pv[j] = t;
        } else if (a.amode == A_MACRO) {
          pv[j] = (T)a.emac[l * 3 + j];
        } else {
          pv[j] = a.in[idx];
        }
      }
      if (a.amode == A_BARE) {
        s[0] = pv[0]; s[1] = pv[1]; s[2] = pv[2];
      } else {
        const T e = a.E[v];
        const T tr = a.lam * (pv[0] + pv[1]);
        s[0] = e * (tr + a.mu2 * pv[0]);
        s[1] = e * (tr + a.mu2 * pv[1]);
        s[2] = e * (a.mu2 * pv[2]);
      }
      if (a.amode == A_CG) acc += pv[0] * s[0] + pv[1] * s[1] + pv[2] * s[2];
    }
#pragma unroll
    for (int j = 0; j < GS; ++j)
      reinterpret_cast<T*>(&buf[(j * NP + yy / 2) * NX + xx])[yy & 1] = s[j];
  }
  __syncthreads();
  smem_fft<T, NX, GS * NP, NX, NT, -1>(buf, a.tw[0]);

  // two-for-one real FFT: rows (y, y+1) were packed as Z = X_y + i X_{y+1}
  for (int i = threadIdx.x; i < gs * KX * NP; i += NT) {
    const int pr = i % NP, k = (i / NP) % KX, j = i / (NP * KX);
    const C* row = buf + (j * NP + pr) * NX;
    const C A = row[k];
    const C Bc = cconj(row[(NX - k) & (NX - 1)]);
    const C xa = cscale(cadd(A, Bc), (T)0.5);
    const C d = csub(A, Bc);
    const C xb = mkc<T>((T)0.5 * d.y, (T)-0.5 * d.x);
    C* dst = a.spec + (((int64_t)l * a.m + c0 + j) * KX + k) * ny + y0 + 2 * pr;
    dst[0] = xa;
    dst[1] = xb;
  }

  if (a.amode == A_CG) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y;
    const int blk = blockIdx.x + gridDim.x * blockIdx.y;
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(s, part, &cg->cnt_a, blk, nblk, &flag)) {
      const double pq = sum_partials<NT>(part, nblk, red);
      if (threadIdx.x == 0) {
        cg->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) { cg->status = ST_BAD; cg->alpha = 0.0; }
        else cg->alpha = cg->rr / pq;
        cg->cnt_a = 0;
      }
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
  if (mode == P_NODAL_IN) {
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
  if (mode == P_NODAL_OUT) {
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

// grid (n_x/2+1, L); one k_x column of all six spectra per block.
template <typename T, int NY, int NT>
__global__ void __launch_bounds__(NT) pass_c_2d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int M = 6;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [M][NY]
  const int kx = blockIdx.x, l = blockIdx.y;
  const int KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int cin = (a.pmode == P_NODAL_IN) ? 2 : M;
  const int cout = (a.pmode == P_NODAL_OUT) ? 2 : M;
  for (int i = threadIdx.x; i < cin * NY; i += NT) {
    const int c = i / NY, y = i % NY;
    buf[c * NY + y] = a.spec[(((int64_t)l * M + c) * KX + kx) * NY + y];
  }
  __syncthreads();
  if (cin == M) smem_fft<T, NY, M, NY, NT, -1>(buf, a.tw[1]);
  else smem_fft<T, NY, 2, NY, NT, -1>(buf, a.tw[1]);

  const C ex = a.ph[0][kx];
  for (int ky = threadIdx.x; ky < NY; ky += NT) {
    C s[M];
#pragma unroll
    for (int c = 0; c < M; ++c) s[c] = (c < cin) ? buf[c * NY + ky] : mkc<T>(0, 0);
    if (kx == 0 && ky == 0) {
#pragma unroll
      for (int c = 0; c < M; ++c) s[c] = mkc<T>(0, 0);
    } else {
      project_2d<T>(s, ex, a.ph[1][ky], a.ih[0], a.ih[1], a.inv_n, a.pmode);
    }
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < cout) buf[c * NY + ky] = s[c];
  }
  __syncthreads();
  if (cout == M) smem_fft<T, NY, M, NY, NT, +1>(buf, a.tw[1]);
  else smem_fft<T, NY, 2, NY, NT, +1>(buf, a.tw[1]);
  for (int i = threadIdx.x; i < cout * NY; i += NT) {
    const int c = i / NY, y = i % NY;
    a.spec[(((int64_t)l * M + c) * KX + kx) * NY + y] = buf[c * NY + y];
  }
}

// ---------------------------------------------------------------- pass E
// grid (n_y/TY, components, L); inverse real FFT along x of one component.
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT) pass_e_2d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int KX = NX / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [NP][NX]
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int l = blockIdx.z, c = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1];
  const int64_t N = a.N;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;

  for (int i = threadIdx.x; i < KX * NP; i += NT) {
    const int pr = i % NP, k = i / NP;
    const C* src = a.spec + (((int64_t)l * a.m + c) * KX + k) * ny + y0 + 2 * pr;
    C xa = src[0], xb = src[1];
    if (k == 0 || k == NX / 2) { xa.y = 0; xb.y = 0; }  // C2R ignores these imaginary parts
    buf[pr * NX + k] = mkc<T>(xa.x - xb.y, xa.y + xb.x);           // X_a + i X_b
    if (k > 0 && k < NX / 2) buf[pr * NX + NX - k] = mkc<T>(xa.x + xb.y, xb.x - xa.y);  // conj(X_a) + i conj(X_b)
  }
  __syncthreads();
  smem_fft<T, NX, NP, NX, NT, +1>(buf, a.tw[0]);

  T acc = 0;
  const T alpha = (a.emode == E_CG) ? (T)cg->alpha : (T)0;
  for (int i = threadIdx.x; i < TY * NX; i += NT) {
    const int yy = i / NX, xx = i % NX;
    const int64_t v = (int64_t)(y0 + yy) * NX + xx;
    const T q = reinterpret_cast<const T*>(&buf[(yy / 2) * NX + xx])[yy & 1];
    if (a.emode == E_NODAL) {
      a.u64[((int64_t)l * 2 + c) * N + v] += (double)q;
      continue;
    }
    const int64_t idx = ((int64_t)l * a.m + c) * N + v;
    if (a.emode == E_CG) {
      a.x[idx] += alpha * a.p[idx];
      const T rv = a.r[idx] - alpha * q;
      a.r[idx] = rv;
      acc += rv * rv;
    } else if (a.emode == E_INIT) {
      const T rv = -q;
      a.r[idx] = rv;
      a.x[idx] = 0;
      acc += rv * rv;
    } else {
      a.out[idx] = q;
    }
  }

  if (a.emode == E_CG || a.emode == E_INIT) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y;
    const int blk = blockIdx.x + gridDim.x * blockIdx.y;
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(s, part, &cg->cnt_e, blk, nblk, &flag)) {
      const double rr = sum_partials<NT>(part, nblk, red);
      if (threadIdx.x == 0) {
        if (a.emode == E_INIT) {
          cg->rr0 = rr; cg->rr = rr; cg->it = 0; cg->beta = 0.0;
          cg->status = !isfinite(rr) ? ST_BAD : (rr == 0.0 ? ST_CONV : ST_RUN);
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
    }
  }
}

// ------------------------------------------------------------ launchers
template <typename T> struct Tile2D;
template <> struct Tile2D<float> { static constexpr int TY = 8; };
template <> struct Tile2D<double> { static constexpr int TY = 4; };

template <typename T, int NX>
cudaError_t launch_a_2d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int TY = Tile2D<T>::TY, NT = 256;
  const size_t sm = sizeof(cplx<T>) * 3 * (TY / 2) * NX;
  auto k = pass_a_2d<T, NX, TY, NT>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.n[1] / TY, a.amode == A_NODAL ? 1 : 2, a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int NX>
cudaError_t launch_e_2d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int TY = Tile2D<T>::TY, NT = 256;
  const size_t sm = sizeof(cplx<T>) * (TY / 2) * NX;
  auto k = pass_e_2d<T, NX, TY, NT>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.n[1] / TY, a.emode == E_NODAL ? 2 : 6, a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int NY>
cudaError_t launch_c_2d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NT = (NY >= 512) ? 512 : 256;
  const size_t sm = sizeof(cplx<T>) * 6 * NY;
  auto k = pass_c_2d<T, NY, NT>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.kx, a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
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

