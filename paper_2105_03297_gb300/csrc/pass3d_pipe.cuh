// Pipelined first pass of the 3D projected-CG iteration (FP32, CG mode).
//
// The same arithmetic as pass_a_3d in A_CG mode (direction update
// p = r + beta p_old, the deferred x += alpha_prev p_old, the material
// sigma = E_v Cbar : p, the forward real FFT along x and <p, C p>), organised
// so that the memory system never waits for the SM: a persistent grid of
// blocks takes tiles (TY rows of one z plane, the six components of one
// tetrahedron group, one load case) in turn, and while a block transforms and
// stores its current tile, the TMA unit brings the raw rows of its next tile
// (r, p_old and x of the six components and the moduli; every one a contiguous
// run of TY * n_x values) into shared memory with bulk copies that complete on
// an mbarrier.  Waits on the mbarrier are bounded: a block whose copies do not
// arrive within about two seconds marks every load case as failed with a
// timeout mark, waits (bounded again) for its copies, and returns; the host
// reports RVE_ERR_TIMEOUT.
#pragma once
#include <algorithm>

#include "pass2d.cuh"

namespace rve {

constexpr int kPipeMaxL = 64;                  // load-case slots the per-slot partials hold
constexpr long long kMbarWaitCycles = 4000000000LL;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// One bulk copy global -> shared memory of this block (16-byte aligned
// addresses, size a multiple of 16), completing `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase with the given parity to complete; false after the cycle limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kMbarWaitCycles) return false;
  return true;
}

template <int NX, int TY> constexpr size_t pipe_a_smem() {
  // raw rows [3 streams][6 components][TY][NX] and the moduli [TY][NX] (FP32),
  // then the transform buffer [6][TY/2][ae_ld]
  return sizeof(float) * (3 * 6 + 1) * TY * NX + sizeof(float2) * 6 * (TY / 2) * ae_ld<NX>();
}

// grid: a multiple of the SM count (persistent), NT threads = the load units of
// a tile (2 rows x 4 values x 3 components each).
template <int NX, int TY, int NT>
__global__ void __launch_bounds__(NT, 2) pass_a_3d_pipe(PassArgs<float> a) {
  using T = float;
  using C = float2;
  constexpr int NP = TY / 2;
  constexpr int GS = 6;
  constexpr int KX = NX / 2 + 1;
  constexpr int LD = ae_ld<NX>();
  constexpr int ROW = TY * NX;                         // values of one component's tile rows
  constexpr int XV = NX / 4;                           // float4 vectors per row
  static_assert(NT == 2 * NP * XV, "one load unit per thread");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* stage = reinterpret_cast<T*>(smem_raw);           // [3][GS][ROW], then the moduli [ROW]
  C* buf = reinterpret_cast<C*>(smem_raw + sizeof(T) * (3 * GS + 1) * ROW);
  __shared__ uint64_t bar;
  __shared__ double red[NT / 32];
  __shared__ double accl[kPipeMaxL];
  __shared__ int flag;

  const int ny = a.n[1], nz = a.n[2], G = a.nq, L = a.L;
  const int nyt = ny / TY;
  const int64_t per_l = (int64_t)nyt * nz * G;
  const int64_t total = per_l * L;
  const int64_t N = a.N;
  const int tid = threadIdx.x;

  auto runs = [&](int l) -> bool {
    const CgState* cg = a.cg + l;
    return cg->active && (!a.cgphase || cg->status == ST_RUN);
  };
  auto next_tile = [&](int64_t t) -> int64_t {
    for (; t < total; t += gridDim.x)
      if (runs((int)(t / per_l))) return t;
    return total;
  };
  // tile t -> load case, group, z plane, first row
  auto decode = [&](int64_t t, int& l, int& grp, int& z, int& y0) {
    l = (int)(t / per_l);
    int64_t rem = t % per_l;
    grp = (int)(rem / ((int64_t)nyt * nz));
    rem %= (int64_t)nyt * nz;
    z = (int)(rem / nyt);
    y0 = (int)(rem % nyt) * TY;
  };
  // thread 0: the bulk copies of tile t into the stage
  auto issue = [&](int64_t t) {
    int l, grp, z, y0;
    decode(t, l, grp, z, y0);
    const bool use_old = a.cg[l].it > 0;
    const int streams = use_old ? 3 : 1;
    const unsigned bytes = (unsigned)(ROW * sizeof(T));
    const int64_t v0 = ((int64_t)z * ny + y0) * NX;
    mbar_arrive_expect_tx(&bar, (unsigned)(streams * GS + 1) * bytes);
    for (int s = 0; s < streams; ++s) {
      const T* base = s == 0 ? a.r : s == 1 ? a.p : a.x;
      for (int j = 0; j < GS; ++j)
        bulk_copy_g2s(stage + (s * GS + j) * ROW, base + ((int64_t)l * a.m + grp * GS + j) * N + v0, bytes, &bar);
    }
    bulk_copy_g2s(stage + 3 * GS * ROW, a.E + (int64_t)(l / a.lcs) * N + v0, bytes, &bar);
  };

  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  for (int l = tid; l < L; l += NT) accl[l] = 0.0;
  __syncthreads();

  int64_t t = next_tile(blockIdx.x);
  if (tid == 0 && t < total) issue(t);
  unsigned parity = 0;
  bool timed_out = false;
  // this thread's load unit: half (normal / shear components), row pair, vector
  const int half = tid / (NP * XV), pr = (tid / XV) % NP, xq = tid % XV;
  const int j0 = half * 3;
  while (t < total) {
    int l, grp, z, y0;
    decode(t, l, grp, z, y0);
    const CgState* cg = a.cg + l;
    const bool use_old = cg->it > 0;
    const T beta = (T)cg->beta, alpha_prev = (T)cg->alpha;
    const bool ok = mbar_wait_bounded(&bar, parity);
    if (__syncthreads_or(!ok)) {   // block-uniform decision
      timed_out = true;
      break;
    }
    parity ^= 1u;
    // direction update, deferred x update, material: rows (2 pr, 2 pr + 1), 4 values, 3 components
    const int64_t v0 = ((int64_t)z * ny + y0) * NX;
    T acc = 0;
    {
      T sv[2][3][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int off = (2 * pr + h) * NX + 4 * xq;
        T ev[4];
        vload(ev, stage + 3 * GS * ROW + off);
        T pv[3][4];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int c = j0 + j;
          vload(pv[j], stage + c * ROW + off);
          const int64_t idx = ((int64_t)l * a.m + grp * GS + c) * N + v0 + off;
          if (use_old) {
            T po[4], xo[4];
            vload(po, stage + (GS + c) * ROW + off);
            vload(xo, stage + (2 * GS + c) * ROW + off);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              pv[j][q] += beta * po[q];
              xo[q] += alpha_prev * po[q];
            }
            vstore(a.x + idx, xo);
          }
          vstore(a.p + idx, pv[j]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T e = ev[q];
          if (half == 0) {
            const T tr = a.lam * (pv[0][q] + pv[1][q] + pv[2][q]);
#pragma unroll
            for (int j = 0; j < 3; ++j) sv[h][j][q] = e * (tr + a.mu2 * pv[j][q]);
          } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) sv[h][j][q] = e * (a.mu2 * pv[j][q]);
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) acc += pv[j][q] * sv[h][j][q];
        }
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C* dst = buf + ((j0 + j) * NP + pr) * LD + 4 * xq;
#pragma unroll
        for (int q = 0; q < 4; q += 2)
          cstore2<T>(dst + q, mkc<T>(sv[0][j][q], sv[1][j][q]), mkc<T>(sv[0][j][q + 1], sv[1][j][q + 1]));
      }
    }
    __syncthreads();  // the stage is free and the transform buffer complete
    const int64_t tn = next_tile(t + gridDim.x);
    if (tid == 0 && tn < total) issue(tn);
    smem_fft<T, NX, GS * NP, LD, NT, -1>(buf, a.tw[0]);
    pass_a_store<T, NX, TY, NT, LD>(buf, GS, a.spec + ((((int64_t)l * a.m + grp * GS) * KX) * nz + z) * ny + y0,
                                    (int64_t)KX * nz * ny, (int64_t)nz * ny);
    const double s = block_sum<NT>((double)acc, red);   // its first barrier also ends the buffer reads
    if (tid == 0) accl[l] += s;
    t = tn;
  }
  if (timed_out) {
    // mark every load case, give the copies in flight a bounded time, return
    if (tid == 0) {
      for (int l = 0; l < L; ++l) {
        a.cg[l].status = ST_BAD;
        a.cg[l].pad = kTimeoutMark;
      }
      __threadfence();
    }
    mbar_wait_bounded(&bar, parity);
    return;
  }
  __syncthreads();
  // per load case: this block's partial of <p, C p>; the last block sums them
  for (int l = 0; l < L; ++l) {
    if (!runs(l)) continue;
    CgState* cg = a.cg + l;
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(accl[l], part, &cg->cnt_a, blockIdx.x, gridDim.x, &flag)) {
      const double pq = sum_partials<NT>(part, gridDim.x, red);
      if (tid == 0) finish_alpha(cg, pq);
    }
    __syncthreads();
  }
}

// Launch over min(tiles, 2 blocks per SM).
template <int NX>
cudaError_t launch_a_3d_pipe(const PassArgs<float>& a, cudaStream_t s) {
  constexpr int TY = 4;
  constexpr int NT = 2 * (TY / 2) * (NX / 4);
  constexpr size_t sm = pipe_a_smem<NX, TY>();
  auto k = pass_a_3d_pipe<NX, TY, NT>;
  static DeviceOnce attr;
  static int sms[kMaxDevices] = {0};
  const int dev = current_device();
  attr.run(dev, [&] {
    set_smem_attrs(k, sm);
    if (dev >= 0 && dev < kMaxDevices) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  });
  const int nsm = (dev >= 0 && dev < kMaxDevices && sms[dev] > 0) ? sms[dev] : 152;
  const int64_t tiles = (int64_t)(a.n[1] / TY) * a.n[2] * a.nq * a.L;
  const int blocks = (int)std::min<int64_t>(tiles, 2 * (int64_t)nsm);
  k<<<blocks, NT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rve
