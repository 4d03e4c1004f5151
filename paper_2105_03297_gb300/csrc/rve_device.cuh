// Device-side building blocks shared by the projected-CG pass kernels:
// complex arithmetic on float2/double2, the batched shared-memory Stockham
// FFT, block reductions with a deterministic last-block finalisation, and the
// per-load-case CG state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rve {

// ---------------------------------------------------------------- complex
template <typename T> struct CT;
template <> struct CT<float> { using c = float2; };
template <> struct CT<double> { using c = double2; };
template <typename T> using cplx = typename CT<T>::c;

template <typename T> __device__ __forceinline__ cplx<T> mkc(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cjmul(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// multiply by +i (S > 0) or -i (S < 0)
template <int S, typename C> __device__ __forceinline__ C cmul_i(C a) {
  C r; if (S > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r;
}
template <typename C> __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------------------------- CG state
// One per load case, in device memory.  status: 0 running, 1 converged,
// 2 iteration limit reached, 3 non-finite value or breakdown.
struct CgState {
  double rr, rr0, pq, alpha, beta, tol2;
  double fn2;        // squared FP64 nodal residual norm (last residual pass)
  int it, maxit, status, active;  // active: the outer refinement still runs this load case
  unsigned cnt_a, cnt_e, cnt_r, pad;
};

enum { ST_RUN = 0, ST_CONV = 1, ST_MAXIT = 2, ST_BAD = 3 };

// ------------------------------------------------------- Stockham FFT
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// R-point DFT of v in place, sign S (-1 forward, +1 inverse).
template <int S, int R, typename C> __device__ __forceinline__ void dft_small(C* v) {
  if constexpr (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    C a2 = cadd(v[1], v[3]), a3 = cmul_i<S>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2); v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3); v[3] = csub(a1, a3);
  } else if constexpr (R == 8) {
    using T = decltype(v[0].x);
    const T h = (T)0.70710678118654752440;
    // two radix-4 on even/odd, then combine with W8^r
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<S, 4>(e);
    dft_small<S, 4>(o);
    // o[r] *= exp(S*2*pi*i*r/8)
    C o1; o1.x = h * (o[1].x - (T)S * o[1].y); o1.y = h * (o[1].y + (T)S * o[1].x);
    C o2 = cmul_i<S>(o[2]);
    C o3; o3.x = h * (-o[3].x - (T)S * o[3].y); o3.y = h * (-o[3].y + (T)S * o[3].x);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
}

// One Stockham autosort stage of radix R with NS = product of the previous
// radices, over NB transforms of length N stored at buf + b*LD.  Values are
// staged in registers so the stage is in place; two barriers per stage.
// tw[t] = exp(-2 pi i t / N) (host FP64 libm, rounded to T).
template <typename T, int N, int NB, int LD, int NT, int S, int R, int NS>
__device__ __forceinline__ void stockham_stage(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int NBF = NB * (N / R);
  constexpr int PER = (NBF + NT - 1) / NT;
  C v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int f = threadIdx.x + i * NT;
    if ((NBF % NT) == 0 || f < NBF) {
      const int b = f / (N / R), j = f % (N / R);
      const C* src = buf + b * LD + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = src[r * (N / R)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int f = threadIdx.x + i * NT;
    if ((NBF % NT) == 0 || f < NBF) {
      const int b = f / (N / R), j = f % (N / R);
      const int k = j % NS;
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = __ldg(tw + r * k * (N / (NS * R)));
          if (S > 0) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      dft_small<S, R>(v[i]);
      C* dst = buf + b * LD + (j / NS) * NS * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) dst[q * NS] = v[i][q];
    }
  }
  __syncthreads();
}

template <typename T, int N, int NB, int LD, int NT, int S, int NS>
__device__ __forceinline__ void stockham_from(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  if constexpr (NS * 8 <= N && (ilog2c(N / NS) % 3) == 0) {
    stockham_stage<T, N, NB, LD, NT, S, 8, NS>(buf, tw);
    stockham_from<T, N, NB, LD, NT, S, NS * 8>(buf, tw);
  } else if constexpr (NS * 4 <= N) {
    stockham_stage<T, N, NB, LD, NT, S, 4, NS>(buf, tw);
    stockham_from<T, N, NB, LD, NT, S, NS * 4>(buf, tw);
  } else if constexpr (NS * 2 <= N) {
    stockham_stage<T, N, NB, LD, NT, S, 2, NS>(buf, tw);
  }
}

// Batched in-place FFT (unnormalised) of NB transforms of length N in shared
// memory.  Caller must __syncthreads() before (data written) — the function
// ends with a barrier.
template <typename T, int N, int NB, int LD, int NT, int S>
__device__ __forceinline__ void smem_fft(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  stockham_from<T, N, NB, LD, NT, S, 1>(buf, tw);
}

// ------------------------------------------------------------ reductions
template <int NT> __device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  }
  return s;  // valid in thread 0
}

// Publish this block's partial and report whether it is the last block of
// the load case to do so.  The last block then sums all partials in block
// order, so the result does not depend on scheduling.
__device__ __forceinline__ bool publish_partial(double s, double* part, unsigned* cnt, int blk, int nblk,
                                                int* flag_smem) {
  if (threadIdx.x == 0) {
    part[blk] = s;
    __threadfence();
    unsigned t = atomicAdd(cnt, 1u);
    *flag_smem = (t == (unsigned)(nblk - 1));
  }
  __syncthreads();
  return *flag_smem != 0;
}

// Sum of nblk partials in index order (called by the whole last block).
template <int NT> __device__ __forceinline__ double sum_partials(const double* part, int nblk, double* red) {
  __threadfence();
  // each thread sums a fixed strided subset, then a fixed-order tree
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += NT) s += __ldcg(part + i);
  return block_sum<NT>(s, red);
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

}  // namespace rve
