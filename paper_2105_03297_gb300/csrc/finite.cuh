// Finite strain: the projection of deformation-gradient fields (Eq.
// original-G with the discrete element derivatives of Eq.
// discrete_projection_op) for pass C.  A gradient field holds, per voxel,
// n_q elements x D x D components F_{Theta,i,a} = d chi_i / d r_a at index
// Theta D^2 + i D + a (2D: 8 components padded to 9 so that passes A and E
// see three groups of three).  G acts on the gradient index a of every row i:
//
//   t_i = sum_{Theta,a} conj(g_Theta,a) H_{Theta,i,a},  w_i = t_i / S,
//   H_{Theta,i,a} <- g_Theta,a w_i,                     S = sum |g_Theta,a|^2,
//
// G = 0 where S = 0 (k = 0).
#pragma once
#include "rve_device.cuh"

namespace rve {

// Element gradient symbols of the linear finite elements (the same stencils
// as the small-strain projection): 2D nodes {00,10,01} and {11,01,10}; 3D
// Kuhn tetrahedra {0, e_a, e_a+e_b, 1} in lexicographic order of (a,b,c).
template <typename T, int D>
__device__ __forceinline__ void fe_gradients(const cplx<T>* e, const T* ih, cplx<T> g[6][3]) {
  using C = cplx<T>;
  const C one = mkc<T>(1, 0);
  C d[3];
#pragma unroll
  for (int i = 0; i < D; ++i) d[i] = cscale(csub(e[i], one), ih[i]);
  if (D == 2) {
    g[0][0] = d[0]; g[0][1] = d[1];
    g[1][0] = cmul(e[1], d[0]); g[1][1] = cmul(e[0], d[1]);
  } else {
    const C e01 = cmul(e[0], e[1]), e02 = cmul(e[0], e[2]), e12 = cmul(e[1], e[2]);
    g[0][0] = d[0];             g[0][1] = cmul(e[0], d[1]);  g[0][2] = cmul(e01, d[2]);   // (x,y,z)
    g[1][0] = d[0];             g[1][1] = cmul(e02, d[1]);   g[1][2] = cmul(e[0], d[2]);  // (x,z,y)
    g[2][0] = cmul(e[1], d[0]); g[2][1] = d[1];              g[2][2] = cmul(e01, d[2]);   // (y,x,z)
    g[3][0] = cmul(e12, d[0]);  g[3][1] = d[1];              g[3][2] = cmul(e[1], d[2]);  // (y,z,x)
    g[4][0] = cmul(e[2], d[0]); g[4][1] = cmul(e02, d[1]);   g[4][2] = d[2];              // (z,x,y)
    g[5][0] = cmul(e12, d[0]);  g[5][1] = cmul(e[2], d[1]);  g[5][2] = d[2];              // (z,y,x)
  }
}

// One wavevector: s (n_q D^2 components, element major, padding untouched)
// -> G s * scale.  col(c) addresses component c.
template <typename T, int D, int NQ, class Col>
__device__ __forceinline__ void project_finite(Col col, const cplx<T> g[6][3], T scale, bool zero) {
  using C = cplx<T>;
  T S = 0;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int a = 0; a < D; ++a) S += cabs2(g[q][a]);
  const T id = (zero || !(S > (T)0)) ? (T)0 : scale / S;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    C t = mkc<T>(0, 0);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int a = 0; a < D; ++a) t = cadd(t, cjmul(g[q][a], col(q * D * D + i * D + a)));
    const C w = cscale(t, id);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int a = 0; a < D; ++a) col(q * D * D + i * D + a) = cmul(g[q][a], w);
  }
}

}  // namespace rve
