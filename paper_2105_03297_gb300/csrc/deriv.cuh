// Fourier symbols of the discrete derivatives other than the linear finite
// elements (Secs. 2.3-2.5 and Appendix C) and the projection
// G = B (B^H B)^-1 B^H for them, one wavevector per call.  Every derivative
// has n_q <= 2 evaluation points per voxel; B(k) maps a nodal amplitude w to
// the Mandel strains sym(g_q (x) w) of the evaluation points.
//
//   forward:  g_a = (e_a - 1) / h_a                     (Eq. forward-difference-derivative-fourier)
//   central:  g_a = i sin(theta_a) / h_a                (Eq. central-difference-derivative-fourier)
//   lsq:      g_a = (e_a - 1) / h_a prod_{b != a} (1 + e_b) / 2   (Sec. 2.5, voxel-averaged)
//   fourier:  g_a = i theta_a / h_a                     (the derivative of Eq. original-G)
//   fourier2: g_{1,a} = i theta_a / h_a exp(-i phi), g_{2,a} = i theta_a / h_a exp(+i phi),
//             phi = (theta_x + theta_y) / 6             (Appendix C, 2D)
//
// e_a = exp(i theta_a), theta_a = 2 pi j_a / n_a.  theta is wrapped to
// (-pi, pi) and set to 0 at the Nyquist index of an even axis (the average of
// the two grid choices of Sec. 2.7); sin(theta) and 1 + e are exactly 0 at
// theta = pi.  Where every g vanishes (k = 0, and the zeros of central
// differences, least squares and the Fourier derivative) G = 0.
#pragma once
#include "rve_device.cuh"
#include "rve_internal.h"

namespace rve {

// wrapped angle of index j on an axis of n points (exactly 0 at j = 0 and j = n/2)
template <typename T> __device__ __forceinline__ T wrapped_theta(int j, int n) {
  int w = (2 * j < n) ? j : j - n;
  if (2 * j == n) w = 0;
  return (T)(6.283185307179586477 * (double)w / (double)n);
}

template <typename T> __device__ __forceinline__ void sincos_t(T x, T* s, T* c);
template <> __device__ __forceinline__ void sincos_t<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <> __device__ __forceinline__ void sincos_t<double>(double x, double* s, double* c) { sincos(x, s, c); }

// g[q][a] of the non-FE derivatives at the wavevector with indices j[a];
// e[a] = exp(2 pi i j_a / n_a) from the phase tables.  Returns n_q.
template <typename T, int D>
__device__ __forceinline__ int deriv_symbols(int deriv, const int* j, const int* n, const cplx<T>* e, const T* ih,
                                             cplx<T> g[2][3]) {
  using C = cplx<T>;
  if (deriv == D_FORWARD) {
#pragma unroll
    for (int a = 0; a < D; ++a) g[0][a] = mkc<T>((e[a].x - (T)1) * ih[a], e[a].y * ih[a]);
    return 1;
  }
  if (deriv == D_CENTRAL) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool zero = (j[a] == 0) || (2 * j[a] == n[a]);
      g[0][a] = mkc<T>((T)0, zero ? (T)0 : e[a].y * ih[a]);
    }
    return 1;
  }
  if (deriv == D_LSQ) {
    C half1p[3];
#pragma unroll
    for (int b = 0; b < D; ++b)
      half1p[b] = (2 * j[b] == n[b]) ? mkc<T>(0, 0) : mkc<T>((T)0.5 * ((T)1 + e[b].x), (T)0.5 * e[b].y);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      C v = mkc<T>((e[a].x - (T)1) * ih[a], e[a].y * ih[a]);
#pragma unroll
      for (int b = 0; b < D; ++b)
        if (b != a) v = cmul(v, half1p[b]);
      g[0][a] = v;
    }
    return 1;
  }
  T th[3];
#pragma unroll
  for (int a = 0; a < D; ++a) th[a] = wrapped_theta<T>(j[a], n[a]);
  if (deriv == D_FOURIER) {
#pragma unroll
    for (int a = 0; a < D; ++a) g[0][a] = mkc<T>((T)0, th[a] * ih[a]);
    return 1;
  }
  // D_FOURIER2 (2D)
  T sp, cp;
  sincos_t<T>((th[0] + th[1]) / (T)6, &sp, &cp);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T k = th[a] * ih[a];
    // i k exp(-+ i phi) = (k sin phi, k cos phi) and (-k sin phi, k cos phi)
    g[0][a] = mkc<T>(k * sp, k * cp);
    g[1][a] = mkc<T>(-k * sp, k * cp);
  }
  return 2;
}

// s (nq * n_s Mandel components, element major) -> B (B^H B)^-1 B^H s * scale.
// M = B^H B = 1/2 sum_q (|g_q|^2 I + g_q conj(g_q)^T); G = 0 where all g = 0.
template <typename T, int D>
__device__ __forceinline__ void project_generic(cplx<T>* s, const cplx<T> g[2][3], int nq, T scale) {
  using C = cplx<T>;
  constexpr int NS = (D == 2) ? 3 : 6;
  const T r2 = (T)kInvSqrt2;
  T md[3] = {0, 0, 0};
  C mo[3] = {mkc<T>(0, 0), mkc<T>(0, 0), mkc<T>(0, 0)};   // (0,1), (0,2), (1,2)
  C t[3] = {mkc<T>(0, 0), mkc<T>(0, 0), mkc<T>(0, 0)};
  T gn = 0;
  for (int q = 0; q < nq; ++q) {
    T a2[3], nn = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) { a2[a] = cabs2(g[q][a]); nn += a2[a]; }
    gn += nn;
#pragma unroll
    for (int a = 0; a < D; ++a) md[a] += (T)0.5 * (nn + a2[a]);
    mo[0] = cadd(mo[0], cscale(cmul(g[q][0], cconj(g[q][1])), (T)0.5));
    if (D == 3) {
      mo[1] = cadd(mo[1], cscale(cmul(g[q][0], cconj(g[q][2])), (T)0.5));
      mo[2] = cadd(mo[2], cscale(cmul(g[q][1], cconj(g[q][2])), (T)0.5));
    }
    // t = B^H s: t_j = sum_a conj(g_a) sigma_aj (tensor stress from Mandel)
    const C* sq = s + q * NS;
    if (D == 2) {
      const C sxx = sq[0], syy = sq[1], sxy = cscale(sq[2], r2);
      t[0] = cadd(t[0], cadd(cjmul(g[q][0], sxx), cjmul(g[q][1], sxy)));
      t[1] = cadd(t[1], cadd(cjmul(g[q][0], sxy), cjmul(g[q][1], syy)));
    } else {
      const C sxx = sq[0], syy = sq[1], szz = sq[2];
      const C syz = cscale(sq[3], r2), sxz = cscale(sq[4], r2), sxy = cscale(sq[5], r2);
      t[0] = cadd(t[0], cadd(cadd(cjmul(g[q][0], sxx), cjmul(g[q][1], sxy)), cjmul(g[q][2], sxz)));
      t[1] = cadd(t[1], cadd(cadd(cjmul(g[q][0], sxy), cjmul(g[q][1], syy)), cjmul(g[q][2], syz)));
      t[2] = cadd(t[2], cadd(cadd(cjmul(g[q][0], sxz), cjmul(g[q][1], syz)), cjmul(g[q][2], szz)));
    }
  }
  if (!(gn > (T)0)) {
    for (int c = 0; c < nq * NS; ++c) s[c] = mkc<T>(0, 0);
    return;
  }
  C w[3];
  if (D == 2) {
    const T det = md[0] * md[1] - cabs2(mo[0]);
    const T id = scale / det;
    w[0] = cscale(csub(cscale(t[0], md[1]), cmul(mo[0], t[1])), id);
    w[1] = cscale(csub(cscale(t[1], md[0]), cjmul(mo[0], t[0])), id);
  } else {
    // adjugate of M = [[A, m01, m02], [conj m01, B, m12], [conj m02, conj m12, Cc]]
    const T A = md[0], B = md[1], Cc = md[2];
    const C m01 = mo[0], m02 = mo[1], m12 = mo[2];
    const T A00 = B * Cc - cabs2(m12);
    const T A11 = A * Cc - cabs2(m02);
    const T A22 = A * B - cabs2(m01);
    const C A01 = csub(cmul(m02, cconj(m12)), cscale(m01, Cc));
    const C A02 = csub(cmul(m01, m12), cscale(m02, B));
    const C A12 = csub(cmul(m02, cconj(m01)), cscale(m12, A));
    const T det = A * A00 + (cmul(m01, cconj(A01))).x + (cmul(m02, cconj(A02))).x;
    const T id = scale / det;
    w[0] = cscale(cadd(cadd(cscale(t[0], A00), cmul(A01, t[1])), cmul(A02, t[2])), id);
    w[1] = cscale(cadd(cadd(cjmul(A01, t[0]), cscale(t[1], A11)), cmul(A12, t[2])), id);
    w[2] = cscale(cadd(cadd(cjmul(A02, t[0]), cjmul(A12, t[1])), cscale(t[2], A22)), id);
  }
  for (int q = 0; q < nq; ++q) {
    C* sq = s + q * NS;
    if (D == 2) {
      sq[0] = cmul(g[q][0], w[0]);
      sq[1] = cmul(g[q][1], w[1]);
      sq[2] = cscale(cadd(cmul(g[q][0], w[1]), cmul(g[q][1], w[0])), r2);
    } else {
      sq[0] = cmul(g[q][0], w[0]);
      sq[1] = cmul(g[q][1], w[1]);
      sq[2] = cmul(g[q][2], w[2]);
      sq[3] = cscale(cadd(cmul(g[q][1], w[2]), cmul(g[q][2], w[1])), r2);
      sq[4] = cscale(cadd(cmul(g[q][0], w[2]), cmul(g[q][2], w[0])), r2);
      sq[5] = cscale(cadd(cmul(g[q][0], w[1]), cmul(g[q][1], w[0])), r2);
    }
  }
}

}  // namespace rve
