// Device-side building blocks shared by the projected-CG pass kernels:
// complex arithmetic on float2/double2, the batched shared-memory Stockham
// FFT, block reductions with a deterministic last-block finalisation, and the
// per-load-case CG state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_once.h"

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
  double fa2;        // squared norm of the summed magnitudes of the terms of f (round-off scale)
  int it, maxit, status, active;  // active: the outer refinement still runs this load case
  unsigned cnt_a, cnt_e, cnt_r, pad;
};

// ST_HOLD: set up for a new inner solve but not yet released to the CG
// kernels (a batch handle whose next refinement step is being prepared while
// the batch graph still runs the other handles).
enum { ST_RUN = 0, ST_CONV = 1, ST_MAXIT = 2, ST_BAD = 3, ST_HOLD = 4 };
// CgState::pad of a slot whose kernel gave up a bounded device-side wait
// (status ST_BAD); the host reports RVE_ERR_TIMEOUT for it.
constexpr unsigned kTimeoutMark = 0x7107u;
// The pipelined persistent passes (pass3d_pipe.cuh): load-case slots their
// per-slot partial sums hold, and the rows per tile of the last pass (the
// height of its spectrum tensor map's box).
constexpr int kPipeMaxL = 64;
constexpr int kPipeETY = 4;

// ------------------------------------------------------- FFT in shared memory
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// cos(2 pi j / 32) for j = 0..8 (first quadrant, FP64 values of the
// mathematical constants); the other twiddles of the register FFTs follow by
// symmetry.
__host__ __device__ constexpr double kCos32q(int j) {
  return j == 0 ? 1.0 : j == 1 ? 0.98078528040323044913 : j == 2 ? 0.92387953251128675613
       : j == 3 ? 0.83146961230254523708 : j == 4 ? 0.70710678118654752440 : j == 5 ? 0.55557023301960222474
       : j == 6 ? 0.38268343236508977173 : j == 7 ? 0.19509032201612826785 : 0.0;
}
__host__ __device__ constexpr double kCos32(int j) {
  return j <= 8 ? kCos32q(j) : j <= 16 ? -kCos32q(16 - j) : j <= 24 ? -kCos32q(j - 16) : kCos32q(32 - j);
}
__host__ __device__ constexpr double kSin32(int j) { return kCos32((j + 24) & 31); }

// In-register FFT of R = 1, 2, 4, 8, 16 or 32 points (natural order in and
// out), sign S: exp(S 2 pi i n k / R).  Radix-2 decimation in time, unrolled.
template <int R, int S, typename C>
__device__ __forceinline__ void fft_reg(C* v) {
  using T = decltype(v[0].x);
  if constexpr (R == 2) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    const C a2 = cadd(v[1], v[3]), a3 = cmul_i<S>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2); v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3); v[3] = csub(a1, a3);
  } else if constexpr (R > 4) {
    C e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    fft_reg<R / 2, S>(e);
    fft_reg<R / 2, S>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      C t = o[k];
      const int j = k * (32 / R);
      if (j == 8) {
        t = cmul_i<S>(o[k]);  // w = exp(S i pi / 2) = S i
      } else if (j == 4 || j == 12) {
        // w = (+-1, S) / sqrt2: one multiplication by 1/sqrt2 per component
        const T c = (T)kCos32(4);
        const T sx = (j == 4) ? (T)1 : (T)-1;
        const T sy = (T)S;
        t.x = c * (sx * o[k].x - sy * o[k].y);
        t.y = c * (sx * o[k].y + sy * o[k].x);
      } else if (k != 0) {
        C w;
        w.x = (T)kCos32(j);
        w.y = (T)(S * kSin32(j));
        t = cmul(o[k], w);
      }
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
}

// Four-step split N = N1 * N2 with N1 <= N2 <= 32 (the radix schedule of one
// transform).  Variant 0 is the most square split; variant 1 halves N1 and
// doubles N2 where N2 stays within the 32-point register FFT (16 = 2 x 8,
// 32 = 2 x 16, 64 = 4 x 16, 128 = 4 x 32, 256 = 8 x 32) and is variant 0
// otherwise (512, 1024).  The autotuner picks one per axis.
template <int N, int V = 0> struct FftSplit {
  static constexpr int N1_0 = (N <= 16) ? 4 : (N == 32) ? 4 : (N == 64) ? 8 : (N == 128) ? 8
                            : (N == 256) ? 16 : (N == 512) ? 16 : 32;
  static constexpr bool ALT = (V == 1) && 2 * (N / N1_0) <= 32;
  static constexpr int N1 = ALT ? N1_0 / 2 : N1_0;
  static constexpr int N2 = N / N1;
  // leading dimension of one transform in shared memory (room for the padded
  // transpose of the middle step)
  static constexpr int LD = N + N2;
  // odd leading dimension for buffers that are also read or written across
  // transforms (transposes): consecutive transforms then fall on different banks
  static constexpr int LDO = N + N2 + 1;
};

// Work items of the two steps of the four-step FFT below (step 1: (b, n1),
// one per transform b and n1 < N1; step 2: (b, k2), k2 < N2).
//   Warp mapping (WARP): when the split is square (N2 = N1) or N2 = 2 N1, the
//   items are ordered transform-major in both steps and NT is a whole number
//   of warps, warp w owns T = 32 / N2 whole transforms in both steps: step 1
//   gives them to its first T N1 lanes (all lanes when square, half when
//   N2 = 2 N1), step 2 to all of its lanes.  Every transform's data then stays
//   inside one warp, and the barriers between the steps only have to order
//   that warp's threads (__syncwarp orders their shared-memory accesses too).
//   Otherwise items are numbered across the block (transform fastest where
//   B*_FAST) and the steps need block-wide barriers.
template <int N, int NB, int NT, bool B1_FAST = false, bool B2_FAST = false, int V = 0> struct FftItems {
  static constexpr int N1 = FftSplit<N, V>::N1, N2 = FftSplit<N, V>::N2;
  static constexpr bool WARP =
      !B1_FAST && !B2_FAST && (N2 == N1 || N2 == 2 * N1) && NT % 32 == 0 && 32 % N2 == 0;
  static constexpr int T = 32 / N2;                         // transforms per warp (warp mapping)
  static constexpr int WB = (NT / 32) * T;                  // transforms per iteration (warp mapping)
  static constexpr int W1 = NB * N1, W2 = NB * N2;
  static constexpr int I1 = WARP ? (NB + WB - 1) / WB : (W1 + NT - 1) / NT;
  static constexpr int I2 = WARP ? I1 : (W2 + NT - 1) / NT;
  // item i of this thread in step 1 / step 2; false if the thread has none there
  __device__ __forceinline__ static bool step1(int i, int& b, int& n1) {
    if constexpr (WARP) {
      const int lane = threadIdx.x & 31;
      b = i * WB + (threadIdx.x >> 5) * T + lane / N1;
      n1 = lane % N1;
      return (T * N1 == 32 || lane < T * N1) && (NB % WB == 0 || b < NB);
    } else {
      const int it = threadIdx.x + i * NT;
      b = B1_FAST ? it % NB : it / N1;
      n1 = B1_FAST ? it / NB : it % N1;
      return (W1 % NT) == 0 || it < W1;
    }
  }
  __device__ __forceinline__ static bool step2(int i, int& b, int& k2) {
    if constexpr (WARP) {
      const int lane = threadIdx.x & 31;
      b = i * WB + (threadIdx.x >> 5) * T + lane / N2;
      k2 = lane % N2;
      return NB % WB == 0 || b < NB;
    } else {
      const int it = threadIdx.x + i * NT;
      b = B2_FAST ? it % NB : it / N2;
      k2 = B2_FAST ? it / NB : it % N2;
      return (W2 % NT) == 0 || it < W2;
    }
  }
};

// Row stride of the x-transform buffers of the first and last passes: at
// least the FFT's leading dimension, and 4 (mod 16) complex values, so that
// the rows of the NP packed row pairs that consecutive threads read or write
// at the same column (the two-for-one pre- and post-processing, row pairs
// fastest) fall on different shared-memory banks.
template <int N> __host__ __device__ constexpr int ae_ld() {
  return FftSplit<N>::LD + ((4 - FftSplit<N>::LD % 16) + 16) % 16;
}

// Number of distinct splits of a length (1 or 2).
template <int N> __host__ __device__ constexpr int fft_split_count() { return FftSplit<N, 1>::ALT ? 2 : 1; }

// Barrier between two steps of a transform: warp-level when LOCAL.
template <bool LOCAL> __device__ __forceinline__ void fft_step_sync() {
  if constexpr (LOCAL) __syncwarp();
  else __syncthreads();
}

// Threads that give one work item per thread in both steps for NB transforms,
// within [128, 1024], a multiple of 32.
template <int N, int NB, int V = 0> constexpr int fft_threads() {
  constexpr int w = NB * FftSplit<N, V>::N2;
  constexpr int t = w < 128 ? 128 : (w > 1024 ? 1024 : w);
  return (t + 31) / 32 * 32;
}

// Batched in-place FFT (unnormalised, sign S) of NB transforms of length N
// stored at buf + b*LD, natural order in and out.
//   step 1: for every (b, n1): FFT over n2 of x[n1 + N1 n2] in registers,
//           twiddle by exp(S 2 pi i n1 k2 / N), store transposed with a padded
//           stride (N1 + 1) so that both access patterns are conflict-free;
//   step 2: for every (b, k2): FFT over n1 in registers, store X[k2 + N2 k1].
// tw[t] = exp(-2 pi i t / N) (host FP64 libm, rounded to T).  The caller must
// __syncthreads() before; the function ends with a barrier.  Every step reads
// and writes only its own transform's row, so with the warp mapping of
// FftItems the barriers inside are warp-level.
template <typename T, int N, int NB, int LD, int NT, int S>
__device__ __forceinline__ void smem_fft(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using It = FftItems<N, NB, NT>;
  constexpr int N1 = It::N1, N2 = It::N2;
  constexpr bool LOCAL = It::WARP;
  static_assert(LD >= N + N2, "leading dimension too small for the padded transpose");
  {
    C v[It::I1][N2];
#pragma unroll
    for (int i = 0; i < It::I1; ++i) {
      int b, n1;
      if (It::step1(i, b, n1)) {
        const C* src = buf + b * LD + n1;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v[i][n2] = src[n2 * N1];
      }
    }
    fft_step_sync<LOCAL>();
#pragma unroll
    for (int i = 0; i < It::I1; ++i) {
      int b, n1;
      if (It::step1(i, b, n1)) {
        fft_reg<N2, S>(v[i]);
        C* dst = buf + b * LD + n1;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          C t = v[i][k2];
          if (k2 > 0 && n1 > 0) {
            C w = __ldg(tw + n1 * k2);
            if (S > 0) w.y = -w.y;
            t = cmul(t, w);
          }
          dst[k2 * (N1 + 1)] = t;
        }
      }
    }
  }
  fft_step_sync<LOCAL>();
  {
    C v[It::I2][N1];
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      int b, k2;
      if (It::step2(i, b, k2)) {
        const C* src = buf + b * LD + k2 * (N1 + 1);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[i][n1] = src[n1];
      }
    }
    fft_step_sync<LOCAL>();
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      int b, k2;
      if (It::step2(i, b, k2)) {
        fft_reg<N1, S>(v[i]);
        C* dst = buf + b * LD + k2;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) dst[k1 * N2] = v[i][k1];
      }
    }
  }
  __syncthreads();
}

// 32-point FFT (sign S, natural order in and out) of one sequence held by the
// lane pair (q, q + 16) of a warp: the lane with h = 0 holds the even-indexed
// inputs x[2 m], the lane with h = 1 the odd-indexed x[2 m + 1] (m < 16), in
// v.  Each lane transforms its 16 points; the odd lane twiddles its outputs
// O_k by w^k = exp(S 2 pi i k / 32); one exchange per k gives lane h the
// outputs X[16 h + k] = E_k +- w^k O_k in v[k] (the last radix-2
// decimation-in-time stage of fft_reg<32>, with the same twiddle constants).
// Every lane of the warp must call it: it shuffles over the full warp.
template <int S, typename C>
__device__ __forceinline__ void fft_reg_pair32(C* v, int h) {
  using T = decltype(v[0].x);
  fft_reg<16, S>(v);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    C t = v[k];
    if (k == 8) {
      t = cmul_i<S>(v[k]);
    } else if (k == 4 || k == 12) {
      const T c = (T)kCos32(4);
      const T sx = (k == 4) ? (T)1 : (T)-1;
      const T sy = (T)S;
      t.x = c * (sx * v[k].x - sy * v[k].y);
      t.y = c * (sx * v[k].y + sy * v[k].x);
    } else if (k != 0) {
      C w;
      w.x = (T)kCos32(k);
      w.y = (T)(S * kSin32(k));
      t = cmul(v[k], w);
    }
    if (!h) t = v[k];                 // the even lane sends E_k, the odd lane w^k O_k
    C o;
    o.x = __shfl_xor_sync(0xffffffffu, t.x, 16);
    o.y = __shfl_xor_sync(0xffffffffu, t.y, 16);
    v[k] = h ? csub(o, t) : cadd(t, o);
  }
}

// Steps of the four-step FFT for N = N1 x 32 (N1 = 32: 1024, N1 = 16: 512)
// with every 32-point register FFT of step 1 spread over a lane pair
// (fft_reg_pair32): half the registers per thread and 2 N1 threads per
// transform.  Step 1 items are pairs (b, n1), 16 per warp (lanes q and q + 16
// form pair q); step 2 items are pairs (b, k2) again when N1 = 32 and single
// lanes (b, k2) with a 16-point register FFT when N1 = 16.  Items are numbered
// across the block, the second index fastest, so that the 16 lanes of each
// half-warp touch consecutive shared-memory columns; the steps are separated
// by block-wide barriers.  NT is a multiple of 32.
template <int N, int NB, int NT> struct FftPairItems {
  static constexpr int N1 = FftSplit<N>::N1, N2 = FftSplit<N>::N2;
  static_assert(N2 == 32 && (N1 == 32 || N1 == 16), "lane-pair transforms need N2 = 32 and N1 = 16 or 32");
  static_assert(NT % 32 == 0, "whole warps");
  static constexpr bool PAIR2 = (N1 == 32);    // step 2 on lane pairs too
  static constexpr int P = NT / 2;             // pairs per round of the block
  static constexpr int W1 = NB * N1;           // step-1 pairs
  static constexpr int I1 = (W1 + P - 1) / P;  // step-1 rounds
  static constexpr int W2 = NB * N2;           // step-2 items (pairs or lanes)
  static constexpr int I2 = PAIR2 ? (W2 + P - 1) / P : (W2 + NT - 1) / NT;
};

// Step 1 (in place on buf, ends with a barrier): for every pair (b, n1), the
// 32-point FFT over n2 of x[n1 + N1 n2], twiddled by exp(S 2 pi i n1 k2 / N)
// and stored transposed with the padded stride N1 + 1.  The caller must
// __syncthreads() before.
template <typename T, int N, int NB, int LD, int NT, int S>
__device__ __forceinline__ void fft_pair_step1(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using It = FftPairItems<N, NB, NT>;
  constexpr int N1 = It::N1, N2 = It::N2;
  static_assert(LD >= N + N2, "leading dimension too small for the padded transpose");
  const int lane = threadIdx.x & 31, h = lane >> 4;
  const int p0 = (threadIdx.x >> 5) * 16 + (lane & 15);
  C v[It::I1][16];
#pragma unroll
  for (int i = 0; i < It::I1; ++i) {
    const int p = p0 + i * It::P;
    if (p < It::W1) {
      const C* src = buf + (p / N1) * LD + p % N1;
#pragma unroll
      for (int m = 0; m < 16; ++m) v[i][m] = src[(2 * m + h) * N1];
    } else {
#pragma unroll
      for (int m = 0; m < 16; ++m) v[i][m] = mkc<T>(0, 0);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < It::I1; ++i) {
    const int p = p0 + i * It::P;
    fft_reg_pair32<S>(v[i], h);
    if (p < It::W1) {
      const int n1 = p % N1;
      C* dst = buf + (p / N1) * LD + n1;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int k2 = 16 * h + k;
        C t = v[i][k];
        if (k2 > 0 && n1 > 0) {
          C w = __ldg(tw + n1 * k2);
          if (S > 0) w.y = -w.y;
          t = cmul(t, w);
        }
        dst[k2 * (N1 + 1)] = t;
      }
    }
  }
  __syncthreads();
}

// Step 2: for every (b, k2), the N1-point FFT over n1 of the transposed row.
// With N1 = 32 a lane pair shares it and lane h ends with the outputs
// X[k2 + 32 k1], k1 = 16 h + k; with N1 = 16 one lane holds all 16 (h = 0).
// The outputs, v[k] for k < 16, go to out(b, k2, h, v): written back to buf by
// smem_fft_pair, passed to the caller's store by a last pass.
template <typename T, int N, int NB, int LD, int NT, int S, bool TO_SMEM, class Out>
__device__ __forceinline__ void fft_pair_step2(cplx<T>* buf, const Out& out) {
  using C = cplx<T>;
  using It = FftPairItems<N, NB, NT>;
  constexpr int N1 = It::N1, N2 = It::N2;
  C v[It::I2][16];
  if constexpr (It::PAIR2) {
    const int lane = threadIdx.x & 31, h = lane >> 4;
    const int p0 = (threadIdx.x >> 5) * 16 + (lane & 15);
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      const int p = p0 + i * It::P;
      if (p < It::W2) {
        const C* src = buf + (p / N2) * LD + (p % N2) * (N1 + 1);
#pragma unroll
        for (int m = 0; m < 16; ++m) v[i][m] = src[2 * m + h];
      } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) v[i][m] = mkc<T>(0, 0);
      }
    }
    if constexpr (TO_SMEM) __syncthreads();
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      const int p = p0 + i * It::P;
      fft_reg_pair32<S>(v[i], h);
      if (p < It::W2) out(p / N2, p % N2, h, v[i]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      const int it = threadIdx.x + i * NT;
      if (it < It::W2) {
        const C* src = buf + (it / N2) * LD + (it % N2) * (N1 + 1);
#pragma unroll
        for (int m = 0; m < 16; ++m) v[i][m] = src[m];
      }
    }
    if constexpr (TO_SMEM) __syncthreads();
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      const int it = threadIdx.x + i * NT;
      if (it < It::W2) {
        fft_reg<16, S>(v[i]);
        out(it / N2, it % N2, 0, v[i]);
      }
    }
  }
}

// smem_fft for N = 512 or 1024 with lane-pair register FFTs (in place,
// natural order; the caller must __syncthreads() before; ends with a barrier).
template <typename T, int N, int NB, int LD, int NT, int S>
__device__ __forceinline__ void smem_fft_pair(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  fft_pair_step1<T, N, NB, LD, NT, S>(buf, tw);
  auto to_buf = [&](int b, int k2, int h, const C* v) {
    C* dst = buf + b * LD + k2;
#pragma unroll
    for (int k = 0; k < 16; ++k) dst[(16 * h + k) * FftSplit<N>::N2] = v[k];
  };
  fft_pair_step2<T, N, NB, LD, NT, S, true>(buf, to_buf);
  __syncthreads();
}

// Four-step FFT with caller-supplied input and output (same algorithm as
// smem_fft): step 1 reads its inputs through load(b, n) (n = n1 + N1 n2), step 2
// hands every output to store(b, k, value) (k = k2 + N2 k1).  The middle
// transpose lives in buf (leading dimension LD >= N + N2 per transform).
//   LOAD_SMEM:  load() reads buf, so the middle transpose waits for all loads;
//   STORE_SMEM: store() writes buf, so the stores wait for all step-2 reads;
//   B1_FAST / B2_FAST: work items of step 1 / step 2 are ordered with the
//   transform index b fastest (else n1 / k2 fastest), to match the global
//   layout the load / store touches;
//   BATCH_STORE: store.batch(b, k2, v) receives the N1 outputs of an item at
//   once (k = k2 + N2 k1), so that it can issue all of its global loads first.
// A load() or store() that touches buf touches only transform b's own row
// (b*LD .. b*LD + LD - 1); so with the warp mapping of FftItems (square splits
// and N2 = 2 N1) the barriers between the steps are warp-level, and only the
// final STORE_SMEM barrier, after which the caller reads across transforms, is
// block-wide.
// V selects the split (FftSplit<N, V>).
template <typename T, int N, int NB, int LD, int NT, int S, bool LOAD_SMEM, bool STORE_SMEM, bool B1_FAST,
          bool B2_FAST, int V = 0, class Load, class Store, bool BATCH_STORE = false>
__device__ __forceinline__ void fft4(cplx<T>* buf, const cplx<T>* __restrict__ tw, Load load, Store store) {
  using C = cplx<T>;
  using It = FftItems<N, NB, NT, B1_FAST, B2_FAST, V>;
  constexpr int N1 = It::N1, N2 = It::N2;
  constexpr bool LOCAL = It::WARP;
  static_assert(LD >= N + N2, "leading dimension too small for the padded transpose");
  {
    C v[It::I1][N2];
#pragma unroll
    for (int i = 0; i < It::I1; ++i) {
      int b, n1;
      if (It::step1(i, b, n1)) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v[i][n2] = load(b, n1 + N1 * n2);
      }
    }
    if (LOAD_SMEM) fft_step_sync<LOCAL>();
#pragma unroll
    for (int i = 0; i < It::I1; ++i) {
      int b, n1;
      if (It::step1(i, b, n1)) {
        fft_reg<N2, S>(v[i]);
        C* dst = buf + b * LD + n1;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          C t = v[i][k2];
          if (k2 > 0 && n1 > 0) {
            C w = __ldg(tw + n1 * k2);
            if (S > 0) w.y = -w.y;
            t = cmul(t, w);
          }
          dst[k2 * (N1 + 1)] = t;
        }
      }
    }
  }
  fft_step_sync<LOCAL>();
  {
    C v[It::I2][N1];
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      int b, k2;
      if (It::step2(i, b, k2)) {
        const C* src = buf + b * LD + k2 * (N1 + 1);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[i][n1] = src[n1];
      }
    }
    if (STORE_SMEM) fft_step_sync<LOCAL>();
#pragma unroll
    for (int i = 0; i < It::I2; ++i) {
      int b, k2;
      if (It::step2(i, b, k2)) {
        fft_reg<N1, S>(v[i]);
        if constexpr (BATCH_STORE) {
          store.batch(b, k2, v[i]);  // outputs k = k2 + N2 k1, k1 < N1, in one call
        } else {
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) store(b, k2 + N2 * k1, v[i][k1]);
        }
      }
    }
  }
  if (STORE_SMEM) __syncthreads();
}

// 16-byte vector of T (4 floats or 2 doubles) for the streaming loops.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using t = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using t = double2; static constexpr int n = 2; };
template <typename T> __device__ __forceinline__ void vload(T* d, const T* s) {
  const typename Vec16<T>::t w = *reinterpret_cast<const typename Vec16<T>::t*>(s);
  const T* a = reinterpret_cast<const T*>(&w);
#pragma unroll
  for (int i = 0; i < Vec16<T>::n; ++i) d[i] = a[i];
}
// Bulk prefetch into L2 by the TMA unit (no data reaches the SM): `bytes` a
// multiple of 16 starting at a 16-byte aligned global address.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Prefetch `rows` contiguous rows of NX values, `rows_per_comp` per component
// (components comp_stride apart): one bulk request per row.
template <typename T, int NX>
__device__ __forceinline__ void prefetch_rows_l2(const T* base, int comps, int rows_per_comp, int64_t comp_stride) {
  static_assert((NX * sizeof(T)) % 16 == 0, "bulk prefetch sizes are multiples of 16 bytes");
  for (int i = threadIdx.x; i < comps * rows_per_comp; i += blockDim.x) {
    const int j = i / rows_per_comp, row = i % rows_per_comp;
    prefetch_l2_bulk(base + j * comp_stride + (int64_t)row * NX, (unsigned)(NX * sizeof(T)));
  }
}

// Two consecutive complex values (16 bytes for float, two 16-byte halves for double)
template <typename T> __device__ __forceinline__ void cload2(cplx<T>* d, const cplx<T>* s) {
  if constexpr (sizeof(T) == 4) {
    const float4 w = *reinterpret_cast<const float4*>(s);
    d[0] = mkc<T>(w.x, w.y); d[1] = mkc<T>(w.z, w.w);
  } else {
    d[0] = s[0]; d[1] = s[1];
  }
}
template <typename T> __device__ __forceinline__ void cstore2(cplx<T>* d, cplx<T> a, cplx<T> b) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(d) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    d[0] = a; d[1] = b;
  }
}
// VL consecutive values (VL = 2 or the 16-byte width), vectorised
template <typename T, int VL> __device__ __forceinline__ void vloadn(T* d, const T* s) {
  if constexpr (VL == Vec16<T>::n) {
    vload(d, s);
  } else if constexpr (sizeof(T) == 4 && VL == 2) {
    const float2 w = *reinterpret_cast<const float2*>(s);
    d[0] = w.x; d[1] = w.y;
  } else {
#pragma unroll
    for (int i = 0; i < VL; ++i) d[i] = s[i];
  }
}
template <typename T> __device__ __forceinline__ void vstore(T* d, const T* s) {
  typename Vec16<T>::t w;
  T* a = reinterpret_cast<T*>(&w);
#pragma unroll
  for (int i = 0; i < Vec16<T>::n; ++i) a[i] = s[i];
  *reinterpret_cast<typename Vec16<T>::t*>(d) = w;
}
template <typename T, int VL> __device__ __forceinline__ void vstoren(T* d, const T* s) {
  if constexpr (VL == Vec16<T>::n) {
    vstore(d, s);
  } else if constexpr (sizeof(T) == 4 && VL == 2) {
    *reinterpret_cast<float2*>(d) = make_float2(s[0], s[1]);
  } else {
#pragma unroll
    for (int i = 0; i < VL; ++i) d[i] = s[i];
  }
}

// Dynamic shared memory limit and the largest shared-memory carveout for a
// kernel (so that as many blocks as the shared memory allows can be resident).
template <typename K> inline void set_smem_attrs(K kernel, size_t smem) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// The calling thread's current device, or -1 if it cannot be read (then a
// DeviceOnce set-up runs on every call).
inline int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return d;
}
// Streaming multiprocessors of the current device (queried once per device).
inline int device_sm_count() {
  static DeviceOnce once;
  static int sms[kMaxDevices] = {0};
  const int dev = current_device();
  once.run(dev, [&] {
    if (dev >= 0 && dev < kMaxDevices) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  });
  return (dev >= 0 && dev < kMaxDevices && sms[dev] > 0) ? sms[dev] : 152;
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
