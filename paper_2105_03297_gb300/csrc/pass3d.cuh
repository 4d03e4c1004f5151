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
//   E  inverse real FFT along x, x += alpha p, r -= alpha q, <r, r>.
#pragma once
#include "pass2d.cuh"

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

// Mandel material sigma = e * (lam tr(eps) 1 + 2 mu eps)
template <typename T> __device__ __forceinline__ void material6(const T* p, T e, T lam, T mu2, T* s) {
  const T tr = lam * (p[0] + p[1] + p[2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) s[j] = e * (tr + mu2 * p[j]);
#pragma unroll
  for (int j = 3; j < 6; ++j) s[j] = e * (mu2 * p[j]);
}

// ---------------------------------------------------------------- pass A
// grid (n_y/TY, n_z, L*G), G = 6 tetrahedra (6 components each) or 1 (nodal, 3).
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT) pass_a_3d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int GS = 6;
  constexpr int KX = NX / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [GS][NP][NX]
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const bool nodal = (a.amode == A_NODAL);
  const int G = nodal ? 1 : 6;
  const int l = blockIdx.z / G, grp = blockIdx.z % G;
  const int z = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1], nz = a.n[2];
  const int64_t N = a.N;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int gs = nodal ? 3 : 6;
  const int c0 = nodal ? 0 : grp * 6;
  T beta = 0;
  bool use_old = false;
  if (a.amode == A_CG) { beta = (T)cg->beta; use_old = cg->it > 0; }
  T acc = 0;
  const int64_t base_v = ((int64_t)z * ny + y0) * NX;

  for (int i = threadIdx.x; i < TY * NX; i += NT) {
    const int yy = i / NX, xx = i % NX;
    const int64_t v = base_v + i;
    T s[GS];
    if (nodal) {
#pragma unroll
      for (int j = 0; j < 3; ++j) s[j] = a.in[((int64_t)l * 3 + j) * N + v];
      s[3] = s[4] = s[5] = 0;
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
          pv[j] = (T)a.emac[l * 6 + j];
        } else {
          pv[j] = a.in[idx];
        }
      }
      if (a.amode == A_BARE) {
#pragma unroll
        for (int j = 0; j < GS; ++j) s[j] = pv[j];
      } else {
        material6<T>(pv, a.E[v], a.lam, a.mu2, s);
      }
      if (a.amode == A_CG) {
#pragma unroll
        for (int j = 0; j < GS; ++j) acc += pv[j] * s[j];
      }
    }
#pragma unroll
    for (int j = 0; j < GS; ++j)
      reinterpret_cast<T*>(&buf[(j * NP + yy / 2) * NX + xx])[yy & 1] = s[j];
  }
  __syncthreads();
  smem_fft<T, NX, GS * NP, NX, NT, -1>(buf, a.tw[0]);

  for (int i = threadIdx.x; i < gs * KX * NP; i += NT) {
    const int pr = i % NP, k = (i / NP) % KX, j = i / (NP * KX);
    const C* row = buf + (j * NP + pr) * NX;
    const C A = row[k];
    const C Bc = cconj(row[(NX - k) & (NX - 1)]);
    const C xa = cscale(cadd(A, Bc), (T)0.5);
    const C d = csub(A, Bc);
    const C xb = mkc<T>((T)0.5 * d.y, (T)-0.5 * d.x);
    C* dst = a.spec + ((((int64_t)l * a.m + c0 + j) * KX + k) * nz + z) * ny + y0 + 2 * pr;
    dst[0] = xa;
    dst[1] = xb;
  }

  if (a.amode == A_CG) {
    const double s = block_sum<NT>((double)acc, red);
    const int nblk = gridDim.x * gridDim.y * G;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * grp);
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

// ---------------------------------------------------------------- pass B / D
// FFT along y.  grid (n_z/TZB, n_x/2+1, L*Cc).  FWD: spec1 pencils -> spec2
// chunks; !FWD: spec2 chunks -> spec1 pencils.
template <typename T, int NY, int TZB, int NT, bool FWD>
__global__ void __launch_bounds__(NT) pass_y_3d(PassArgs<T> a, int Cc) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [TZB][NY]
  const int l = blockIdx.z / Cc, c = blockIdx.z % Cc;
  const int kx = blockIdx.y, z0 = blockIdx.x * TZB;
  const int nz = a.n[2], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int64_t cbase = (((int64_t)l * a.m + c) * KX + kx);
  if (FWD) {
    const C* src = a.spec + (cbase * nz + z0) * NY;
    for (int i = threadIdx.x; i < TZB * NY; i += NT) buf[i] = src[i];
  } else {
    const C* src = a.spec2 + cbase * NY * nz + z0;
    for (int i = threadIdx.x; i < TZB * NY; i += NT) {
      const int zz = i % TZB, ky = i / TZB;
      buf[zz * NY + ky] = src[(int64_t)ky * nz + zz];
    }
  }
  __syncthreads();
  smem_fft<T, NY, TZB, NY, NT, FWD ? -1 : +1>(buf, a.tw[1]);
  if (FWD) {
    C* dst = a.spec2 + cbase * NY * nz + z0;
    for (int i = threadIdx.x; i < TZB * NY; i += NT) {
      const int zz = i % TZB, ky = i / TZB;
      dst[(int64_t)ky * nz + zz] = buf[zz * NY + ky];
    }
  } else {
    C* dst = a.spec + (cbase * nz + z0) * NY;
    for (int i = threadIdx.x; i < TZB * NY; i += NT) dst[i] = buf[i];
  }
}

// ---------------------------------------------------------------- pass C
// Projection of the 36 spectra at one wavevector (modes as in 2D).
template <typename T>
__device__ __forceinline__ void project_3d(cplx<T>* s, const cplx<T>* e, const T* ih, T scale, int mode) {
  using C = cplx<T>;
  const C one = mkc<T>(1, 0);
  C d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = cscale(csub(e[i], one), ih[i]);
  const C e01 = cmul(e[0], e[1]), e02 = cmul(e[0], e[2]), e12 = cmul(e[1], e[2]);
  // element gradients g[t][axis]
  C g[6][3];
  g[0][0] = d[0];           g[0][1] = cmul(e[0], d[1]);  g[0][2] = cmul(e01, d[2]);   // (x,y,z)
  g[1][0] = d[0];           g[1][1] = cmul(e02, d[1]);   g[1][2] = cmul(e[0], d[2]);  // (x,z,y)
  g[2][0] = cmul(e[1], d[0]); g[2][1] = d[1];            g[2][2] = cmul(e01, d[2]);   // (y,x,z)
  g[3][0] = cmul(e12, d[0]);  g[3][1] = d[1];            g[3][2] = cmul(e[1], d[2]);  // (y,z,x)
  g[4][0] = cmul(e[2], d[0]); g[4][1] = cmul(e02, d[1]); g[4][2] = d[2];              // (z,x,y)
  g[5][0] = cmul(e12, d[0]);  g[5][1] = cmul(e[2], d[1]); g[5][2] = d[2];             // (z,y,x)
  // M = 1/2 sum_t (|g|^2 I + g g^H)
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
  C t3[3];
  if (mode == P_NODAL_IN) {
    t3[0] = s[0]; t3[1] = s[1]; t3[2] = s[2];
  } else {
    t3[0] = t3[1] = t3[2] = mkc<T>(0, 0);
    const T r2 = (T)kInvSqrt2;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const C sxx = s[6 * t], syy = s[6 * t + 1], szz = s[6 * t + 2];
      const C syz = cscale(s[6 * t + 3], r2), sxz = cscale(s[6 * t + 4], r2), sxy = cscale(s[6 * t + 5], r2);
      t3[0] = cadd(t3[0], cadd(cadd(cjmul(g[t][0], sxx), cjmul(g[t][1], sxy)), cjmul(g[t][2], sxz)));
      t3[1] = cadd(t3[1], cadd(cadd(cjmul(g[t][0], sxy), cjmul(g[t][1], syy)), cjmul(g[t][2], syz)));
      t3[2] = cadd(t3[2], cadd(cadd(cjmul(g[t][0], sxz), cjmul(g[t][1], syz)), cjmul(g[t][2], szz)));
    }
  }
  // w = M^-1 t by the adjugate of the Hermitian matrix
  // M = [[a, m01, m02], [conj m01, b, m12], [conj m02, conj m12, c]]
  const T A = mdiag[0], B = mdiag[1], Cc = mdiag[2];
  const C A00 = mkc<T>(B * Cc - cabs2(m12), 0);
  const C A11 = mkc<T>(A * Cc - cabs2(m02), 0);
  const C A22 = mkc<T>(A * B - cabs2(m01), 0);
  // adj[0][1] = m02 conj(m12) - m01 c ; adj[0][2] = m01 m12 - m02 b ; adj[1][2] = m02 conj(m01) - a m12
  const C A01 = csub(cmul(m02, cconj(m12)), cscale(m01, Cc));
  const C A02 = csub(cmul(m01, m12), cscale(m02, B));
  const C A12 = csub(cmul(m02, cconj(m01)), cscale(m12, A));
  const T det = A * A00.x + (cmul(m01, cconj(A01))).x + (cmul(m02, cconj(A02))).x;
  const T id = scale / det;
  C w[3];
  w[0] = cscale(cadd(cadd(cscale(t3[0], A00.x), cmul(A01, t3[1])), cmul(A02, t3[2])), id);
  w[1] = cscale(cadd(cadd(cjmul(A01, t3[0]), cscale(t3[1], A11.x)), cmul(A12, t3[2])), id);
  w[2] = cscale(cadd(cadd(cjmul(A02, t3[0]), cjmul(A12, t3[1])), cscale(t3[2], A22.x)), id);
  if (mode == P_NODAL_OUT) {
    s[0] = w[0]; s[1] = w[1]; s[2] = w[2];
    return;
  }
  const T r2 = (T)kInvSqrt2;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    s[6 * t] = cmul(g[t][0], w[0]);
    s[6 * t + 1] = cmul(g[t][1], w[1]);
    s[6 * t + 2] = cmul(g[t][2], w[2]);
    s[6 * t + 3] = cscale(cadd(cmul(g[t][1], w[2]), cmul(g[t][2], w[1])), r2);
    s[6 * t + 4] = cscale(cadd(cmul(g[t][0], w[2]), cmul(g[t][2], w[0])), r2);
    s[6 * t + 5] = cscale(cadd(cmul(g[t][0], w[1]), cmul(g[t][1], w[0])), r2);
  }
}

// grid (n_x/2+1, n_y, L): one (k_x, k_y) pencil of all components per block.
template <typename T, int NZ, int NT>
__global__ void __launch_bounds__(NT) pass_c_3d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int M = 36;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [M][NZ]
  const int kx = blockIdx.x, ky = blockIdx.y, l = blockIdx.z;
  const int ny = a.n[1], KX = a.kx;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;
  const int cin = (a.pmode == P_NODAL_IN) ? 3 : M;
  const int cout = (a.pmode == P_NODAL_OUT) ? 3 : M;
  const int64_t stride_c = (int64_t)KX * ny * NZ;
  const C* src = a.spec2 + (int64_t)l * M * stride_c + ((int64_t)kx * ny + ky) * NZ;
  for (int i = threadIdx.x; i < cin * NZ; i += NT) {
    const int c = i / NZ, z = i % NZ;
    buf[c * NZ + z] = src[c * stride_c + z];
  }
  __syncthreads();
  if (cin == M) smem_fft<T, NZ, M, NZ, NT, -1>(buf, a.tw[2]);
  else smem_fft<T, NZ, 3, NZ, NT, -1>(buf, a.tw[2]);
  C e[3];
  e[0] = a.ph[0][kx];
  e[1] = a.ph[1][ky];
  for (int kz = threadIdx.x; kz < NZ; kz += NT) {
    C s[M];
#pragma unroll
    for (int c = 0; c < M; ++c) s[c] = (c < cin) ? buf[c * NZ + kz] : mkc<T>(0, 0);
    e[2] = a.ph[2][kz];
    if (kx == 0 && ky == 0 && kz == 0) {
#pragma unroll
      for (int c = 0; c < M; ++c) s[c] = mkc<T>(0, 0);
    } else {
      project_3d<T>(s, e, a.ih, a.inv_n, a.pmode);
    }
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < cout) buf[c * NZ + kz] = s[c];
  }
  __syncthreads();
  if (cout == M) smem_fft<T, NZ, M, NZ, NT, +1>(buf, a.tw[2]);
  else smem_fft<T, NZ, 3, NZ, NT, +1>(buf, a.tw[2]);
  C* dst = a.spec2 + (int64_t)l * M * stride_c + ((int64_t)kx * ny + ky) * NZ;
  for (int i = threadIdx.x; i < cout * NZ; i += NT) {
    const int c = i / NZ, z = i % NZ;
    dst[c * stride_c + z] = buf[c * NZ + z];
  }
}

// ---------------------------------------------------------------- pass E
// grid (n_y/TY, n_z, L*Cc), Cc = m or D (nodal).
template <typename T, int NX, int TY, int NT>
__global__ void __launch_bounds__(NT) pass_e_3d(PassArgs<T> a) {
  using C = cplx<T>;
  constexpr int NP = TY / 2;
  constexpr int KX = NX / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);  // [NP][NX]
  __shared__ double red[NT / 32];
  __shared__ int flag;
  const int Cc = (a.emode == E_NODAL) ? 3 : a.m;
  const int l = blockIdx.z / Cc, c = blockIdx.z % Cc;
  const int z = blockIdx.y, y0 = blockIdx.x * TY;
  const int ny = a.n[1], nz = a.n[2];
  const int64_t N = a.N;
  CgState* cg = a.cg + l;
  if (!cg->active) return;
  if (a.cgphase && cg->status != ST_RUN) return;

  for (int i = threadIdx.x; i < KX * NP; i += NT) {
    const int pr = i % NP, k = i / NP;
    const C* src = a.spec + ((((int64_t)l * a.m + c) * KX + k) * nz + z) * ny + y0 + 2 * pr;
    C xa = src[0], xb = src[1];
    if (k == 0 || k == NX / 2) { xa.y = 0; xb.y = 0; }
    buf[pr * NX + k] = mkc<T>(xa.x - xb.y, xa.y + xb.x);
    if (k > 0 && k < NX / 2) buf[pr * NX + NX - k] = mkc<T>(xa.x + xb.y, xb.x - xa.y);
  }
  __syncthreads();
  smem_fft<T, NX, NP, NX, NT, +1>(buf, a.tw[0]);

  T acc = 0;
  const T alpha = (a.emode == E_CG) ? (T)cg->alpha : (T)0;
  const int64_t base_v = ((int64_t)z * ny + y0) * NX;
  for (int i = threadIdx.x; i < TY * NX; i += NT) {
    const int yy = i / NX, xx = i % NX;
    const int64_t v = base_v + i;
    const T q = reinterpret_cast<const T*>(&buf[(yy / 2) * NX + xx])[yy & 1];
    if (a.emode == E_NODAL) {
      a.u64[((int64_t)l * 3 + c) * N + v] += (double)q;
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
    const int nblk = gridDim.x * gridDim.y * Cc;
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * c);
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
template <typename T> struct Tile3D;
template <> struct Tile3D<float> { static constexpr int TY = 8; static constexpr int TZB = 16; };
template <> struct Tile3D<double> { static constexpr int TY = 4; static constexpr int TZB = 8; };

template <typename T, int NX>
cudaError_t launch_a_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int TY = Tile3D<T>::TY, NT = 256;
  const size_t sm = sizeof(cplx<T>) * 6 * (TY / 2) * NX;
  auto k = pass_a_3d<T, NX, TY, NT>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.n[1] / TY, a.n[2], a.L * (a.amode == A_NODAL ? 1 : 6));
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int NX>
cudaError_t launch_e_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int TY = Tile3D<T>::TY, NT = 256;
  const size_t sm = sizeof(cplx<T>) * (TY / 2) * NX;
  auto k = pass_e_3d<T, NX, TY, NT>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.n[1] / TY, a.n[2], a.L * (a.emode == E_NODAL ? 3 : a.m));
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int NY, bool FWD>
cudaError_t launch_y_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int TZB = Tile3D<T>::TZB, NT = 256;
  const size_t sm = sizeof(cplx<T>) * TZB * NY;
  auto k = pass_y_3d<T, NY, TZB, NT, FWD>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  const int Cc = FWD ? (a.pmode == P_NODAL_IN ? 3 : a.m) : (a.pmode == P_NODAL_OUT ? 3 : a.m);
  dim3 grid(a.n[2] / TZB, a.kx, a.L * Cc);
  k<<<grid, NT, sm, s>>>(a, Cc);
  return cudaGetLastError();
}
template <typename T, int NY> cudaError_t launch_yf_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  return launch_y_3d_n<T, NY, true>(a, s);
}
template <typename T, int NY> cudaError_t launch_yb_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  return launch_y_3d_n<T, NY, false>(a, s);
}
template <typename T, int NZ>
cudaError_t launch_c_3d_n(const PassArgs<T>& a, cudaStream_t s) {
  constexpr int NT = (sizeof(T) == 8 || NZ >= 256) ? 512 : 256;
  const size_t sm = sizeof(cplx<T>) * 36 * NZ;
  auto k = pass_c_3d<T, NZ, NT>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); attr = true; }
  dim3 grid(a.kx, a.n[1], a.L);
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
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
