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
#include <cuda.h>   // CUtensorMap (the type only; the encoder comes from the driver entry point)

#include <algorithm>

#include "pass2d.cuh"

namespace rve {

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
// Orders this thread's earlier shared-memory accesses before its later
// async-proxy (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

// Dynamic shared memory is only guaranteed 16-byte alignment: the pipelined
// passes round their base up to 128 bytes (TMA tensor copies need a 128-byte
// aligned destination) and ask for kSmemAlignPad bytes more.
constexpr int kSmemAlignPad = 128;
__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

template <int NX, int TY> constexpr size_t pipe_a_smem() {
  // raw rows [3 streams][6 components][TY][NX] and the moduli [TY][NX] (FP32),
  // then the transform buffer [6][TY/2][ae_ld]
  return kSmemAlignPad + sizeof(float) * (3 * 6 + 1) * TY * NX + sizeof(float2) * 6 * (TY / 2) * ae_ld<NX>();
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
  unsigned char* smem = align128(smem_raw);
  T* stage = reinterpret_cast<T*>(smem);               // [3][GS][ROW], then the moduli [ROW]
  C* buf = reinterpret_cast<C*>(smem + sizeof(T) * (3 * GS + 1) * ROW);
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
    if (a.stall_copies) return;   // test hook: the phase never completes
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
    if (tid == 0 && tn < total) {
      fence_proxy_async();
      issue(tn);
    }
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

namespace rve {

// ---------------------------------------------------------------- pass E
// Pipelined last pass (3D, FP32, CG mode): the same arithmetic as pass_e_3d
// in E_CG mode (inverse real FFT along x of the six components of a
// tetrahedron group, r -= alpha q, <r, r>).  Each tile's spectrum (k_x = 0..n_x/2
// of TY rows of one z plane: 6 x KX runs of TY complex values) arrives in one
// TMA tensor copy (cp.async.bulk.tensor.4d over the spectrum's [comp][k_x][z][y]
// layout), and its r rows in six bulk copies; the next tile's spectrum copy is
// issued as soon as the current one is unpacked, its r rows as soon as the
// current update has read them.  Bounded mbarrier waits as in the first pass.

template <int NX, int TY> constexpr size_t pipe_e_smem() {
  return kSmemAlignPad + sizeof(float2) * 6 * (NX / 2 + 1) * TY + sizeof(float) * 6 * TY * NX +
         sizeof(float2) * 6 * (TY / 2) * ae_ld<NX>();
}

// One tensor copy of a 4D box at coordinates (c0 innermost .. c3) into shared memory.
__device__ __forceinline__ void tensor_copy_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                               uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// r update of pass E from the staged rows: outputs x = k2 + N2 k1 of rows
// (2 pr, 2 pr + 1) of component j; r rows read from shared memory, written to HBM.
template <int NX, int TY>
struct PipeEStore {
  const float* rS;      // [6][TY][NX]
  float* r;             // first component's r rows of the tile in HBM: r + j * N + row * NX + x
  int64_t N;
  float alpha;
  float* acc;
  __device__ __forceinline__ void batch(int b, int k2, const float2* q) const {
    constexpr int NP = TY / 2;
    constexpr int N1 = FftSplit<NX>::N1, N2 = FftSplit<NX>::N2;
    const int j = b / NP, pr = b % NP;
    const float* s0 = rS + (j * TY + 2 * pr) * NX + k2;
    float* g0 = r + (int64_t)j * N + (int64_t)(2 * pr) * NX + k2;
    float s = 0.f;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      const float a0 = s0[N2 * k1] - alpha * q[k1].x;
      const float a1 = s0[NX + N2 * k1] - alpha * q[k1].y;
      g0[N2 * k1] = a0;
      g0[NX + N2 * k1] = a1;
      s += a0 * a0 + a1 * a1;
    }
    *acc += s;
  }
  __device__ __forceinline__ void operator()(int, int, float2) const {}
};

template <int NX, int TY, int NT>
__global__ void __launch_bounds__(NT, 2) pass_e_3d_pipe(PassArgs<float> a, const __grid_constant__ CUtensorMap tm) {
  using T = float;
  using C = float2;
  constexpr int NP = TY / 2;
  constexpr int GE = 6;
  constexpr int KX = NX / 2 + 1;
  constexpr int LD = ae_ld<NX>();
  constexpr int ROW = TY * NX;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = align128(smem_raw);
  C* specS = reinterpret_cast<C*>(smem);                                            // [GE][KX][TY]
  T* rS = reinterpret_cast<T*>(smem + sizeof(C) * GE * KX * TY);                    // [GE][TY][NX]
  C* buf = reinterpret_cast<C*>(smem + sizeof(C) * GE * KX * TY + sizeof(T) * GE * ROW);   // [GE][NP][LD]
  __shared__ uint64_t barS, barR;
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
  auto decode = [&](int64_t t, int& l, int& grp, int& z, int& y0) {
    l = (int)(t / per_l);
    int64_t rem = t % per_l;
    grp = (int)(rem / ((int64_t)nyt * nz));
    rem %= (int64_t)nyt * nz;
    z = (int)(rem / nyt);
    y0 = (int)(rem % nyt) * TY;
  };
  auto issue_spec = [&](int64_t t) {
    int l, grp, z, y0;
    decode(t, l, grp, z, y0);
    mbar_arrive_expect_tx(&barS, (unsigned)(sizeof(C) * GE * KX * TY));
    // checked before the copy: a 128-byte aligned destination and a box inside
    // the tensor (y0 a multiple of TY, the last component within the slots);
    // otherwise the copy is skipped and the bounded wait reports the failure
    const bool box_ok = (smem_u32(specS) & 127u) == 0 && (y0 % TY) == 0 && y0 + TY <= ny && z < nz &&
                        l * a.m + grp * GE + GE <= a.L * a.m;
    if (box_ok && !a.stall_copies) tensor_copy_4d(specS, &tm, y0, z, 0, l * a.m + grp * GE, &barS);
  };
  auto issue_r = [&](int64_t t) {
    int l, grp, z, y0;
    decode(t, l, grp, z, y0);
    const unsigned bytes = (unsigned)(ROW * sizeof(T));
    const int64_t v0 = ((int64_t)z * ny + y0) * NX;
    mbar_arrive_expect_tx(&barR, GE * bytes);
    if (a.stall_copies) return;
    for (int j = 0; j < GE; ++j)
      bulk_copy_g2s(rS + j * ROW, a.r + ((int64_t)l * a.m + grp * GE + j) * N + v0, bytes, &barR);
  };

  if (tid == 0) {
    mbar_init(&barS, 1);
    mbar_init(&barR, 1);
    mbar_init_fence();
  }
  for (int l = tid; l < L; l += NT) accl[l] = 0.0;
  __syncthreads();
  int64_t t = next_tile(blockIdx.x);
  if (tid == 0 && t < total) {
    issue_spec(t);
    issue_r(t);
  }
  unsigned parS = 0, parR = 0;
  bool timed_out = false;
  while (t < total) {
    int l, grp, z, y0;
    decode(t, l, grp, z, y0);
    const T alpha = (T)a.cg[l].alpha;
    const bool okS = mbar_wait_bounded(&barS, parS);
    if (__syncthreads_or(!okS)) { timed_out = true; break; }
    parS ^= 1u;
    // two-for-one unpack of the staged spectrum into packed rows
    for (int i = tid; i < GE * KX * NP; i += NT) {
      const int pr = i % NP, k = (i / NP) % KX, j = i / (NP * KX);
      const C* src = specS + (j * KX + k) * TY + 2 * pr;
      C xa = src[0], xb = src[1];
      if (k == 0 || k == NX / 2) { xa.y = 0; xb.y = 0; }  // C2R ignores these imaginary parts
      C* row = buf + (j * NP + pr) * LD;
      row[k] = mkc<T>(xa.x - xb.y, xa.y + xb.x);
      if (k > 0 && k < NX / 2) row[NX - k] = mkc<T>(xa.x + xb.y, xb.x - xa.y);
    }
    __syncthreads();   // the spectrum stage is free, the rows are packed
    const int64_t tn = next_tile(t + gridDim.x);
    if (tid == 0 && tn < total) {
      fence_proxy_async();
      issue_spec(tn);
    }
    const bool okR = mbar_wait_bounded(&barR, parR);
    if (__syncthreads_or(!okR)) { timed_out = true; break; }
    parR ^= 1u;
    T acc = 0;
    const int64_t v0 = ((int64_t)z * ny + y0) * NX;
    auto ld_s = [&](int b, int x) -> C { return buf[b * LD + x]; };
    PipeEStore<NX, TY> st{rS, a.r + ((int64_t)l * a.m + grp * GE) * N + v0, N, alpha, &acc};
    fft4<T, NX, GE * NP, LD, NT, +1, true, false, false, false, 0, decltype(ld_s), decltype(st), true>(buf, a.tw[0],
                                                                                                     ld_s, st);
    const double s = block_sum<NT>((double)acc, red);   // its barrier also ends the reads of the r stage
    if (tid == 0) {
      accl[l] += s;
      if (tn < total) {
        fence_proxy_async();
        issue_r(tn);
      }
    }
    t = tn;
  }
  if (timed_out) {
    if (tid == 0) {
      for (int l = 0; l < L; ++l) {
        a.cg[l].status = ST_BAD;
        a.cg[l].pad = kTimeoutMark;
      }
      __threadfence();
    }
    mbar_wait_bounded(&barS, parS);
    mbar_wait_bounded(&barR, parR);
    return;
  }
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    if (!runs(l)) continue;
    CgState* cg = a.cg + l;
    double* part = a.part + (int64_t)l * a.part_stride;
    if (publish_partial(accl[l], part, &cg->cnt_e, blockIdx.x, gridDim.x, &flag)) {
      const double rr = sum_partials<NT>(part, gridDim.x, red);
      if (tid == 0) finish_rr(cg, rr, false);
    }
    __syncthreads();
  }
}

template <int NX>
cudaError_t launch_e_3d_pipe(const PassArgs<float>& a, cudaStream_t s) {
  constexpr int TY = kPipeETY;
  constexpr int NT = 256;
  constexpr size_t sm = pipe_e_smem<NX, TY>();
  auto k = pass_e_3d_pipe<NX, TY, NT>;
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
  k<<<blocks, NT, sm, s>>>(a, *static_cast<const CUtensorMap*>(a.tm_spec));
  return cudaGetLastError();
}

}  // namespace rve
