// C ABI of the projected-CG homogenization solver: handle lifetime, device
// memory, host-side tables, and the solve driver.
//
// Solve structure (both precisions):
//   state: FP64 nodal fluctuation displacement u (D per node), so that the
//   strain E + B u is compatible by construction;
//   outer step: FP64 real-space residual f = B^T C (E + B u) (no FFT);
//     inner right-hand side r0 = -G C (E + B u) = -F^-1[B (B^H B)^-1 F[f]];
//     projected CG on the strain correction delta (Sec. 2.1; iterates stay
//     compatible because every search direction lies in the range of G);
//     delta -> u update through u^ = (B^H B)^-1 B^H delta^  (accumulated in FP64).
//   RVE_FP64 runs the inner solve in FP64 (normally one outer step);
//   RVE_MIXED runs it in FP32 and refines until the FP64 residual meets the
//   tolerance.
#include <cuda.h>   // CUtensorMap and its encoder's signature (looked up through the runtime)

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <new>
#include <vector>

#include "../../include/rve.h"
#include "rve_internal.h"

using namespace rve;

struct rve_s {
  // TMA tensor map of the first spectrum (3D, FP32), for the pipelined last pass
  CUtensorMap tm_spec;
  bool tm_ok = false;
  int stall_copies = 0;  // test hook (rve_test_stall_copies)
  int dim = 0, n[3] = {1, 1, 1};
  int64_t N = 0;
  double len[3] = {1, 1, 1};
  int precision = RVE_FP64;
  cudaStream_t stream = nullptr;       // internal stream all work runs on
  cudaStream_t user_stream = nullptr;  // caller's stream (ordered before every call's work)
  cudaEvent_t join_ev = nullptr;
  int device = 0;
  int ns = 0, nq = 0, m = 0, D = 0, kx = 0;
  double nu = 0.0, lam = 0.0, mu2 = 0.0;
  bool has_material = false;
  int lcs = 0;          // > 0: a batch group, slot l uses material l / lcs (rve_batch_*)
  int n_mat = 1;        // materials held in E64 / Ein
  size_t tsize = 8;  // bytes of the inner precision
  // device memory
  double* E64 = nullptr;
  void* Ein = nullptr;  // E in the inner precision (aliases E64 for FP64)
  void* x = nullptr; void* r = nullptr; void* p = nullptr;
  void* p2 = nullptr;   // second direction buffer (factored operator form only)
  void* fbuf = nullptr;
  void* spec = nullptr; void* spec2 = nullptr;
  double* u = nullptr;
  double* uadj = nullptr;
  double* part = nullptr;
  int part_stride = 0;
  CgState* cg = nullptr;
  CgState* cg_h = nullptr;  // pinned
  double* emac_d = nullptr;
  double* emac_adj_d = nullptr;
  double* hpart = nullptr;
  int hpart_cap = 0;
  void* ph[3] = {nullptr, nullptr, nullptr};
  void* tw[3] = {nullptr, nullptr, nullptr};
  int Lcap = 0;
  // results of the last solve
  int L_solved = 0;
  bool solved = false;
  std::vector<double> emac_h;  // [L][ns]
  std::vector<double> S_h;     // [L][ns]
  // kernel timing (measurement hook)
  bool timing = false;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  double t_ms[RVE_NKINDS] = {0};
  int64_t t_cnt[RVE_NKINDS] = {0};
  std::vector<Rec>* capturing = nullptr;  // event pairs recorded while capturing a graph
  CgState* cg_h2 = nullptr;               // second pinned copy of the CG state (run-ahead)
  // schedule: variants of pass A (tile rows / threads), pass E (tile rows), the
  // FFT split of pass C's axis and of passes B / D (3D); -1 = autotune at the
  // first solve
  int var[RVE_SCHED_PASSES] = {-1, -1, -1, -1};
  float tune_ms[RVE_SCHED_PASSES][RVE_SCHED_VARIANTS] = {{0}};  // candidate times of the last tuning
  int op_form = RVE_FORM_STRESS;          // order of the operator inside projected CG
  int deriv = D_FE;                       // discrete derivative of the projection (RVE_DERIV_*)
  int finite = 0;                         // RVE_FINITE_STRAIN: fields are deformation gradients
  double* Fs = nullptr;                   // [Lcap][m][N] deformation gradient (finite strain)
  double* fmac_d = nullptr;               // [64][D*D] macroscopic deformation gradients
  std::vector<double> P_h;                // [L][D*D] mean first Piola-Kirchhoff stress
};

namespace {

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return map_err(e_);    \
  } while (0)

int map_err(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return RVE_ERR_OOM; }
  return RVE_ERR_CUDA;
}

enum { K_A = 0, K_B = 1, K_C = 2, K_D = 3, K_E = 4, K_RES = 5, K_OTHER = 6, K_FS = 7, K_SU = 8 };

// Launch fn() on the handle's stream; with timing on, bracket it with events.
template <typename F> cudaError_t timed(rve_s* h, int kind, F fn) {
  if (!h->timing) return fn();
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!h->ev_pool.empty()) { ev = h->ev_pool.back(); h->ev_pool.pop_back(); }
  else {
    cudaEventCreate(&ev.first);
    cudaEventCreate(&ev.second);
  }
  // inside a graph capture the events must become event-record nodes
  const unsigned flags = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaError_t e = cudaEventRecordWithFlags(ev.first, h->stream, flags);
  if (e == cudaSuccess) e = fn();
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev.second, h->stream, flags);
  if (h->capturing) h->capturing->push_back({kind, ev.first, ev.second});
  else h->pending.push_back({kind, ev.first, ev.second});
  return e;
}

// Order the handle's stream after everything already queued on the caller's stream.
int join_user(rve_s* h) {
  if (h->user_stream == h->stream) return RVE_OK;
  if (cudaEventRecord(h->join_ev, h->user_stream) != cudaSuccess ||
      cudaStreamWaitEvent(h->stream, h->join_ev, 0) != cudaSuccess) {
    cudaGetLastError();
    return RVE_ERR_CUDA;
  }
  return RVE_OK;
}

// Accumulate the elapsed times of the launches that have completed; the
// others stay pending.
void flush_timing(rve_s* h) {
  std::vector<rve_s::Rec> keep;
  for (auto& r : h->pending) {
    if (cudaEventQuery(r.b) != cudaSuccess) {
      cudaGetLastError();
      keep.push_back(r);
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      h->t_ms[r.kind] += ms;
      h->t_cnt[r.kind] += 1;
    } else {
      cudaGetLastError();
    }
    h->ev_pool.push_back({r.a, r.b});
  }
  h->pending.swap(keep);
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Makes `device` current for the lifetime of the object (an API call, a batch
// group's host thread) and restores the thread's previous device afterwards;
// a negative index leaves the current device alone.
struct DeviceScope {
  int prev = -1;
  bool changed = false;
  explicit DeviceScope(int device) {
    if (device < 0) return;
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
    if (prev != device) {
      changed = (cudaSetDevice(device) == cudaSuccess);
      if (!changed) cudaGetLastError();
    }
  }
  ~DeviceScope() {
    if (changed && prev >= 0) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

void free_dev(void*& p) { if (p) { cudaFree(p); p = nullptr; } }
template <typename P> void free_devp(P*& p) { if (p) { cudaFree(p); p = nullptr; } }

int dev_alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) { *p = nullptr; return map_err(e); }
  return RVE_OK;
}

// exp(s * 2 pi i j / n) for j < n, FP64 libm, stored as T pairs
template <typename T> std::vector<T> phase_table(int n, int sgn) {
  std::vector<T> t(2 * (size_t)n);
  for (int j = 0; j < n; ++j) {
    const double a = 2.0 * M_PI * (double)j / (double)n;
    t[2 * j] = (T)std::cos(a);
    t[2 * j + 1] = (T)(sgn * std::sin(a));
  }
  return t;
}

// Copies and fills go on the handle's stream, which is non-blocking: a call on
// the legacy default stream would not be ordered with the kernels launched on
// it (a fill could still be running when the first kernel writes the buffer).
int copy_sync(rve_s* h, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  CK(cudaMemcpyAsync(dst, src, bytes, kind, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

template <typename T> int upload_tables(rve_s* h) {
  for (int a = 0; a < h->dim; ++a) {
    const int n = h->n[a];
    std::vector<T> ph = phase_table<T>(n, +1), tw = phase_table<T>(n, -1);
    int rc = dev_alloc(&h->ph[a], ph.size() * sizeof(T));
    if (rc) return rc;
    rc = dev_alloc(&h->tw[a], tw.size() * sizeof(T));
    if (rc) return rc;
    if ((rc = copy_sync(h, h->ph[a], ph.data(), ph.size() * sizeof(T), cudaMemcpyHostToDevice))) return rc;
    if ((rc = copy_sync(h, h->tw[a], tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice))) return rc;
  }
  return RVE_OK;
}

int64_t spec_elems(const rve_s* h) {
  return (int64_t)h->kx * h->n[1] * h->n[2];
}

void free_L(rve_s* h) {
  free_dev(h->x); free_dev(h->r); free_dev(h->p); free_dev(h->p2); free_dev(h->fbuf);
  free_devp(h->Fs); free_devp(h->fmac_d);
  free_dev(h->spec); free_dev(h->spec2);
  free_devp(h->u); free_devp(h->uadj); free_devp(h->part); free_devp(h->cg);
  free_devp(h->emac_d); free_devp(h->emac_adj_d);
  if (h->cg_h) { cudaFreeHost(h->cg_h); h->cg_h = nullptr; }
  if (h->cg_h2) { cudaFreeHost(h->cg_h2); h->cg_h2 = nullptr; }
  h->Lcap = 0;
}

// The driver's tensor-map encoder, looked up once through the runtime (no link
// against the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of the first spectrum [slot][component][k_x][z][y] (complex FP32
// copied as 8-byte elements), box = the pipelined last pass's tile: kPipeETY
// values of y, one z, every k_x, the six components of a tetrahedron group.
void make_spec_tensor_map(rve_s* h) {
  h->tm_ok = false;
  if (h->dim != 3 || h->tsize != 4 || h->n[0] < 128 || h->n[1] < kPipeETY || !h->spec) return;
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return;
  const cuuint64_t ny = (cuuint64_t)h->n[1], nz = (cuuint64_t)h->n[2], kx = (cuuint64_t)h->kx;
  const cuuint64_t dims[4] = {ny, nz, kx, (cuuint64_t)h->Lcap * h->m};
  const cuuint64_t strides[3] = {ny * 8, nz * ny * 8, kx * nz * ny * 8};
  const cuuint32_t box[4] = {(cuuint32_t)kPipeETY, 1, (cuuint32_t)kx, 6};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(&h->tm_spec, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, h->spec, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  h->tm_ok = (r == CUDA_SUCCESS);
}

// Buffers for L load cases (grown, never shrunk).
int ensure_capacity(rve_s* h, int L) {
  if (L <= h->Lcap) return RVE_OK;
  // the adjoint needs the forward u kept, so copy it over
  double* old_u = h->u;
  h->u = nullptr;
  int oldL = h->Lcap;
  double* keep_u = nullptr;
  if (old_u && h->solved) {
    if (cudaMalloc((void**)&keep_u, (size_t)oldL * h->D * h->N * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      h->u = old_u;
      return RVE_ERR_OOM;
    }
    if (int rc = copy_sync(h, keep_u, old_u, (size_t)oldL * h->D * h->N * sizeof(double), cudaMemcpyDeviceToDevice)) {
      cudaFree(keep_u);
      h->u = old_u;
      return rc;
    }
  }
  if (old_u) cudaFree(old_u);
  free_L(h);
  const size_t fld = (size_t)L * h->m * h->N * h->tsize;
  const size_t sp = (size_t)L * h->m * spec_elems(h) * 2 * h->tsize;
  int rc = 0;
  if ((rc = dev_alloc(&h->x, fld)) || (rc = dev_alloc(&h->r, fld)) || (rc = dev_alloc(&h->p, fld)) ||
      (rc = dev_alloc(&h->fbuf, fld)) || (rc = dev_alloc(&h->spec, sp)))
    { free_L(h); if (keep_u) cudaFree(keep_u); return rc; }
  if (h->dim == 3 && (rc = dev_alloc(&h->spec2, sp))) { free_L(h); if (keep_u) cudaFree(keep_u); return rc; }
  if (h->op_form == RVE_FORM_FACTORED && (rc = dev_alloc(&h->p2, fld)))
    { free_L(h); if (keep_u) cudaFree(keep_u); return rc; }
  if ((rc = dev_alloc((void**)&h->u, (size_t)L * h->D * h->N * sizeof(double))) ||
      (rc = dev_alloc((void**)&h->uadj, (size_t)h->ns * h->D * h->N * sizeof(double))))
    { free_L(h); if (keep_u) cudaFree(keep_u); return rc; }
  h->part_stride = (int)(h->N / 128 + (int64_t)h->n[1] * h->n[2] * h->m / 2 + 64);
  const int Lp = L > h->ns ? L : h->ns;
  if ((rc = dev_alloc((void**)&h->part, (size_t)Lp * h->part_stride * sizeof(double))) ||
      (rc = dev_alloc((void**)&h->cg, (size_t)Lp * sizeof(CgState))) ||
      (rc = dev_alloc((void**)&h->emac_d, (size_t)Lp * h->ns * sizeof(double))) ||
      (rc = dev_alloc((void**)&h->emac_adj_d, (size_t)h->ns * h->ns * sizeof(double))))
    { free_L(h); if (keep_u) cudaFree(keep_u); return rc; }
  if (cudaMallocHost((void**)&h->cg_h, (size_t)Lp * sizeof(CgState)) != cudaSuccess ||
      cudaMallocHost((void**)&h->cg_h2, (size_t)Lp * sizeof(CgState)) != cudaSuccess) {
    cudaGetLastError(); free_L(h); if (keep_u) cudaFree(keep_u); return RVE_ERR_OOM;
  }
  cudaMemsetAsync(h->p, 0, fld, h->stream);
  if (h->p2) cudaMemsetAsync(h->p2, 0, fld, h->stream);
  cudaMemsetAsync(h->x, 0, fld, h->stream);
  cudaMemsetAsync(h->part, 0, (size_t)Lp * h->part_stride * sizeof(double), h->stream);
  if (keep_u)
    cudaMemcpyAsync(h->u, keep_u, (size_t)oldL * h->D * h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  const cudaError_t se = cudaStreamSynchronize(h->stream);
  if (keep_u) cudaFree(keep_u);
  CK(se);
  h->Lcap = L;
  make_spec_tensor_map(h);
  CK(cudaGetLastError());
  return RVE_OK;
}

template <typename T> PassArgs<T> pass_args(const rve_s* h, int L, double* u, const double* emac) {
  PassArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  for (int i = 0; i < 3; ++i) a.n[i] = h->n[i];
  a.dim = h->dim; a.L = L; a.m = h->m; a.ns = h->ns;
  // passes A and E work in groups of n_s components: n_q groups for strain
  // fields, m / n_s for finite-strain gradient fields
  a.nq = h->finite ? h->m / h->ns : h->nq;
  a.N = h->N; a.kx = h->kx;
  a.E = (const T*)h->Ein;
  a.lcs = h->lcs > 0 ? h->lcs : L;
  a.x = (T*)h->x; a.r = (T*)h->r; a.p = (T*)h->p;
  a.p2 = h->op_form == RVE_FORM_FACTORED ? (T*)h->p2 : nullptr;
  a.in = (const T*)h->fbuf; a.out = (T*)h->fbuf;
  a.u64 = u;
  a.spec = (cplx<T>*)h->spec; a.spec2 = (cplx<T>*)h->spec2;
  a.emac = emac;
  for (int i = 0; i < 3; ++i) {
    a.ph[i] = (const cplx<T>*)h->ph[i];
    a.tw[i] = (const cplx<T>*)h->tw[i];
    a.ih[i] = (T)((double)h->n[i] / h->len[i]);
  }
  a.lam = (T)h->lam; a.mu2 = (T)h->mu2;
  a.inv_n = (T)(1.0 / (double)h->N);
  a.deriv = h->deriv;
  a.cg = h->cg; a.part = h->part; a.part_stride = h->part_stride;
  a.var_a = h->var[0] < 0 ? 0 : h->var[0];
  a.var_e = h->var[1] < 0 ? 0 : h->var[1];
  a.var_c = h->var[2] < 0 ? 0 : h->var[2];
  a.var_y = h->var[3] < 0 ? 0 : h->var[3];
  a.tm_spec = h->tm_ok ? static_cast<const void*>(&h->tm_spec) : nullptr;
  a.stall_copies = h->stall_copies;
  return a;
}

Fp64Args fp64_args(const rve_s* h, int L, const double* u, const double* emac, CgState* cg) {
  Fp64Args f;
  std::memset(&f, 0, sizeof(f));
  for (int i = 0; i < 3; ++i) { f.n[i] = h->n[i]; f.ih[i] = (double)h->n[i] / h->len[i]; }
  f.dim = h->dim; f.L = L; f.ns = h->ns; f.nq = h->nq; f.N = h->N;
  f.E = h->E64; f.u = u; f.emac = emac;
  f.lcs = h->lcs > 0 ? h->lcs : L;
  f.lam = h->lam; f.mu2 = h->mu2;
  f.cg = cg; f.part = h->part; f.part_stride = h->part_stride;
  f.fout = h->fbuf; f.fout_f32 = (h->tsize == 4);
  return f;
}

template <typename T> cudaError_t pass_a(rve_s* h, const PassArgs<T>& a) {
  return timed(h, a.cgphase ? K_A : K_OTHER, [&] {
    return h->dim == 2 ? launch_pass_a_2d<T>(a, h->stream) : launch_pass_a_3d<T>(a, h->stream);
  });
}
template <typename T> cudaError_t pass_mid(rve_s* h, const PassArgs<T>& a) {
  const int cg = a.cgphase;
  if (h->dim == 2) return timed(h, cg ? K_C : K_OTHER, [&] { return launch_pass_c_2d<T>(a, h->stream); });
  cudaError_t e = timed(h, cg ? K_B : K_OTHER, [&] { return launch_pass_b_3d<T>(a, h->stream); });
  if (e != cudaSuccess) return e;
  e = timed(h, cg ? K_C : K_OTHER, [&] { return launch_pass_c_3d<T>(a, h->stream); });
  if (e != cudaSuccess) return e;
  return timed(h, cg ? K_D : K_OTHER, [&] { return launch_pass_d_3d<T>(a, h->stream); });
}
template <typename T> cudaError_t pass_e(rve_s* h, const PassArgs<T>& a) {
  return timed(h, a.cgphase ? K_E : K_OTHER, [&] {
    return h->dim == 2 ? launch_pass_e_2d<T>(a, h->stream) : launch_pass_e_3d<T>(a, h->stream);
  });
}
// One full operator application with the modes set in a.
template <typename T> cudaError_t apply_passes(rve_s* h, const PassArgs<T>& a) {
  cudaError_t e = pass_a<T>(h, a);
  if (e == cudaSuccess) e = pass_mid<T>(h, a);
  if (e == cudaSuccess) e = pass_e<T>(h, a);
  return e;
}

// One projected-CG iteration in the factored nodal form:
//   force stencil (p update, material, f = B_r^T C p, alpha)
//   -> FFT passes on the D nodal components with w^ = (B^H B)^-1 f^
//   -> strain update (q = B_r w, r -= alpha q, beta).
// Iteration parity q writes the direction to {p, p2}[q] and reads the previous
// one from the other buffer.  f and w are carved out of fbuf (idle during CG).
template <typename T> cudaError_t apply_factored(rve_s* h, const PassArgs<T>& a, int parity) {
  T* P[2] = {(T*)h->p, (T*)h->p2};
  T* f = (T*)h->fbuf;
  T* w = f + (size_t)a.L * h->D * h->N;
  cudaError_t e = timed(h, K_FS, [&] { return launch_force_stencil<T>(a, P[parity ^ 1], P[parity], f, h->stream); });
  PassArgs<T> b = a;
  b.amode = A_NODAL; b.pmode = P_SOLVE; b.emode = E_NOUT;
  b.in = f; b.out = w;
  if (e == cudaSuccess) e = pass_a<T>(h, b);
  if (e == cudaSuccess) e = pass_mid<T>(h, b);
  if (e == cudaSuccess) e = pass_e<T>(h, b);
  if (e == cudaSuccess) e = timed(h, K_SU, [&] { return launch_strain_update<T>(a, w, h->stream); });
  return e;
}

// Nodal-state buffers: xi, rho[2], pi[2], f, w, each [L][D][N] of the inner
// precision, carved out of the strain-form fields (m >= 2 D components).
template <typename T> struct NodalBufs {
  T* xi; T* rho[2]; T* pi[2]; T* f; T* w;
  NodalBufs(const rve_s* h, int L) {
    const size_t nd = (size_t)L * h->D * h->N;
    xi = (T*)h->x;
    rho[0] = (T*)h->r; rho[1] = rho[0] + nd;
    pi[0] = (T*)h->p; pi[1] = pi[0] + nd;
    f = (T*)h->fbuf; w = f + nd;
  }
};

// One projected-CG iteration on the nodal state (parity q of the iteration):
// force kernel (pi, xi, f = B^T C B pi, alpha) -> FFT passes with
// w^ = (B^H B)^-1 f^ -> update kernel (rho -= alpha w, <B rho, B rho>, beta).
template <typename T> cudaError_t apply_nodal(rve_s* h, const PassArgs<T>& a, int q) {
  NodalBufs<T> nb(h, a.L);
  cudaError_t e = timed(h, K_FS, [&] {
    return launch_nodal_force<T>(a, nb.rho[q], nb.pi[q ^ 1], nb.pi[q], nb.xi, nb.f, h->stream);
  });
  PassArgs<T> b = a;
  b.amode = A_NODAL; b.pmode = P_SOLVE; b.emode = E_NOUT;
  b.in = nb.f; b.out = nb.w;
  if (e == cudaSuccess) e = pass_a<T>(h, b);
  if (e == cudaSuccess) e = pass_mid<T>(h, b);
  if (e == cudaSuccess) e = pass_e<T>(h, b);
  if (e == cudaSuccess)
    e = timed(h, K_SU, [&] { return launch_nodal_update<T>(a, nb.rho[q], nb.w, nb.rho[q ^ 1], nb.xi, 0, h->stream); });
  return e;
}

// The k-th CG iteration of a batch (k counts from 0 at the start of an inner
// solve; batches hold an even number of iterations, so k's parity is the
// parity of the CG iteration count of every slot still running).
// One Newton-CG iteration of the finite-strain solve: direction update and
// tangent t = K(F) : p (with <p, t>), then G t by the FFT passes with the
// r update of pass E.
inline cudaError_t apply_finite(rve_s* h, const PassArgs<double>& a) {
  cudaError_t e = timed(h, K_FS, [&] { return launch_fs_dir_tangent(a, h->Fs, (double*)h->fbuf, h->stream); });
  PassArgs<double> b = a;
  b.amode = A_BARE; b.pmode = P_FINITE; b.emode = E_CG;
  b.in = (const double*)h->fbuf;
  if (e == cudaSuccess) e = pass_a<double>(h, b);
  if (e == cudaSuccess) e = pass_mid<double>(h, b);
  if (e == cudaSuccess) e = pass_e<double>(h, b);
  return e;
}

template <typename T> cudaError_t cg_iteration(rve_s* h, const PassArgs<T>& a, int k) {
  if constexpr (std::is_same<T, double>::value) {
    if (h->finite) return apply_finite(h, a);
  }
  if (h->op_form == RVE_FORM_FACTORED) return apply_factored<T>(h, a, k & 1);
  if (h->op_form == RVE_FORM_NODAL) return apply_nodal<T>(h, a, k & 1);
  return apply_passes<T>(h, a);
}

int read_state(rve_s* h, int L) {
  CK(cudaMemcpyAsync(h->cg_h, h->cg, (size_t)L * sizeof(CgState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) flush_timing(h);
  return RVE_OK;
}
int write_state(rve_s* h, int L) {
  CK(cudaMemcpyAsync(h->cg, h->cg_h, (size_t)L * sizeof(CgState), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

// ---- autotuner: the schedule of the FFT passes --------------------------
// Candidates per pass (rve_sched_candidates): pass A rows per block (default,
// half, double) and one thread per load unit at the default and half rows;
// pass E rows per block (default, half, double); in 3D FP32 with n_x >= 128
// also the pipelined persistent passes and the default tiles with the L2
// prefetch of a later block's rows (A 5 and 6, E 3 and 4); in 2D FP32 with
// n_x = 512 or 1024 also pass A with the lane-pair x transform (A 5); the FFT split (radix
// schedule) of pass C's axis; in 3D the split of the y axis (passes B and D,
// timed together).  Each candidate is timed on the handle's own buffers
// (CG-iteration modes on zeroed fields of the solve's load cases, at most
// kTuneMaxL; 2 warm-up and 3 timed launches, CUDA events on the handle's
// stream), passes in the order A, E, C, B/D with the winners of the earlier
// ones, and the fastest is kept; choices are cached per (dimension, grid,
// precision, load cases timed) for the process.
struct TuneKey {
  int dim, n0, n1, n2, tsize, nl;
  bool operator<(const TuneKey& o) const {
    return std::tie(dim, n0, n1, n2, tsize, nl) < std::tie(o.dim, o.n0, o.n1, o.n2, o.tsize, o.nl);
  }
};
std::map<TuneKey, std::array<int, RVE_SCHED_PASSES>> g_tuned;
std::mutex g_tune_mutex;

int split_count(int n) {
  switch (n) {
    case 16: return fft_split_count<16>();
    case 32: return fft_split_count<32>();
    case 64: return fft_split_count<64>();
    case 128: return fft_split_count<128>();
    case 256: return fft_split_count<256>();
    case 512: return fft_split_count<512>();
    default: return fft_split_count<1024>();
  }
}

// Number of candidates of schedule entry `which` for a handle.
int rve_sched_candidates(const rve_s* h, int which) {
  switch (which) {
    case 0: return (h->dim == 3 && h->tsize == 4 && h->n[0] >= 128) ? 7
                 : (h->dim == 2 && h->tsize == 4 && h->n[0] >= 512) ? 6 : h->n[0] >= 64 ? 5 : 3;
    case 1: return (h->dim == 3 && h->tsize == 4 && h->n[0] >= 128 && h->tm_ok) ? 5 : 3;
    case 2: return split_count(h->n[h->dim - 1]);
    default: return h->dim == 3 ? split_count(h->n[1]) : 1;
  }
}

// Load cases the candidates are timed with: those of the solve that asks for
// the tuning (the grids of the passes scale with them, and with them how full
// the last wave of blocks is), at most kTuneMaxL.
constexpr int kTuneMaxL = 8;

template <typename T> int autotune(rve_s* h, int L) {
  const int Lt = L < 1 ? 1 : (L > kTuneMaxL ? kTuneMaxL : L);
  const TuneKey key{h->dim, h->n[0], h->n[1], h->n[2], (int)h->tsize, Lt};
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      for (int w = 0; w < RVE_SCHED_PASSES; ++w)
        if (h->var[w] < 0) h->var[w] = it->second[w];
      return RVE_OK;
    }
  }
  // passes A and E are timed in their CG-iteration modes (A: direction update,
  // deferred x update, material, x FFT, <p, C p>; E: inverse x FFT, r update,
  // <r, r>) on zeroed vectors of Lt load cases; the CG state they finalise is
  // reset by the solve that follows
  const size_t fld = (size_t)h->m * h->N * h->tsize;
  CK(cudaMemsetAsync(h->fbuf, 0, fld, h->stream));
  CK(cudaMemsetAsync(h->r, 0, fld * Lt, h->stream));
  CK(cudaMemsetAsync(h->p, 0, fld * Lt, h->stream));
  CK(cudaMemsetAsync(h->x, 0, fld * Lt, h->stream));
  std::memset(h->cg_h, 0, sizeof(CgState) * Lt);
  for (int l = 0; l < Lt; ++l) {
    h->cg_h[l].active = 1;
    h->cg_h[l].it = 1;
  }
  int rc = write_state(h, Lt);
  if (rc) return rc;
  PassArgs<T> a = pass_args<T>(h, Lt, h->u, h->emac_d);
  a.cgphase = 0; a.amode = A_CG; a.pmode = P_G; a.emode = E_CG;
  a.in = (const T*)h->fbuf; a.out = (T*)h->x;
  a.var_a = a.var_e = a.var_c = a.var_y = 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool d3 = (h->dim == 3);
  auto pass_a_l = [&]() { return d3 ? launch_pass_a_3d<T>(a, h->stream) : launch_pass_a_2d<T>(a, h->stream); };
  auto pass_b_l = [&]() { return d3 ? launch_pass_b_3d<T>(a, h->stream) : cudaSuccess; };
  auto pass_c_l = [&]() { return d3 ? launch_pass_c_3d<T>(a, h->stream) : launch_pass_c_2d<T>(a, h->stream); };
  auto pass_d_l = [&]() { return d3 ? launch_pass_d_3d<T>(a, h->stream) : cudaSuccess; };
  auto pass_e_l = [&]() { return d3 ? launch_pass_e_3d<T>(a, h->stream) : launch_pass_e_2d<T>(a, h->stream); };
  int best[RVE_SCHED_PASSES] = {0, 0, 0, 0};
  for (int w = 0; w < RVE_SCHED_PASSES; ++w)
    for (int v = 0; v < RVE_SCHED_VARIANTS; ++v) h->tune_ms[w][v] = 0.f;
  for (int which = 0; which < RVE_SCHED_PASSES; ++which) {
    const int nc = rve_sched_candidates(h, which);
    float best_ms = 1e30f;
    for (int v = 0; v < nc; ++v) {
      int* slot = which == 0 ? &a.var_a : which == 1 ? &a.var_e : which == 2 ? &a.var_c : &a.var_y;
      *slot = v;
      auto one = [&]() -> cudaError_t {
        if (which == 0) return pass_a_l();
        if (which == 1) return pass_e_l();
        if (which == 2) return pass_c_l();
        cudaError_t e = pass_b_l();
        return e == cudaSuccess ? pass_d_l() : e;
      };
      // the later passes read the spectra the earlier ones write: fill them once
      if (which >= 1) CK(pass_a_l());
      if (which >= 2) CK(pass_b_l());
      for (int k = 0; k < 2; ++k) CK(one());
      CK(cudaEventRecord(e0, h->stream));
      for (int k = 0; k < 3; ++k) CK(one());
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      h->tune_ms[which][v] = ms / 3.0f;
      if (ms < best_ms) { best_ms = ms; best[which] = v; }
    }
    *(which == 0 ? &a.var_a : which == 1 ? &a.var_e : which == 2 ? &a.var_c : &a.var_y) = best[which];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::array<int, RVE_SCHED_PASSES> chosen;
  for (int w = 0; w < RVE_SCHED_PASSES; ++w) {
    if (h->var[w] < 0) h->var[w] = best[w];
    chosen[w] = best[w];
  }
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tuned[key] = chosen;
  return RVE_OK;
}

// The projected-CG loop in batches of K iterations.  Each batch is a CUDA
// graph of K x (passes A, [B,] C, [D,] E); two copies (each with its own
// timing events) are launched alternately, and the host checks the CG state
// copied after batch i while batch i+1 already runs, so the GPU does not wait
// for the host.  A batch launched after every slot has stopped costs only the
// early exits of its kernels.  Without graphs (capture not possible, e.g. on
// the legacy default stream) the same launches are issued directly.
template <typename T> struct CgRunner {
  rve_s* h;
  int L, K;
  PassArgs<T> a;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<rve_s::Rec> recs[2];
  cudaEvent_t copied[2] = {nullptr, nullptr};
  CgState* host[2];

  CgRunner(rve_s* h_, int L_, const PassArgs<T>& a_, int K_) : h(h_), L(L_), K(K_), a(a_) {
    host[0] = h->cg_h;
    host[1] = h->cg_h2;
    for (int b = 0; b < 2; ++b) cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
    for (int b = 0; b < 2; ++b) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      h->capturing = &recs[b];
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < K && e == cudaSuccess; ++k) e = cg_iteration<T>(h, a, k);
      h->capturing = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess || !g || cudaGraphInstantiate(&exec[b], g, 0) != cudaSuccess) {
        cudaGetLastError();
        exec[b] = nullptr;
      }
      if (g) cudaGraphDestroy(g);
      if (!exec[b]) break;
    }
    if (!exec[0] || !exec[1]) {
      for (int b = 0; b < 2; ++b) {
        if (exec[b]) cudaGraphExecDestroy(exec[b]);
        exec[b] = nullptr;
        for (auto& r : recs[b]) h->ev_pool.push_back({r.a, r.b});
        recs[b].clear();
      }
    }
  }
  ~CgRunner() {
    for (int b = 0; b < 2; ++b) {
      if (exec[b]) cudaGraphExecDestroy(exec[b]);
      if (copied[b]) cudaEventDestroy(copied[b]);
      for (auto& r : recs[b]) h->ev_pool.push_back({r.a, r.b});
    }
  }
  cudaError_t launch(int b) {
    cudaError_t e = cudaSuccess;
    if (exec[b]) {
      e = cudaGraphLaunch(exec[b], h->stream);
    } else {
      for (int k = 0; k < K && e == cudaSuccess; ++k) e = cg_iteration<T>(h, a, k);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host[b], h->cg, (size_t)L * sizeof(CgState), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(copied[b], h->stream);
    return e;
  }
  // Wait for batch b's state copy; account its kernel times.
  cudaError_t wait(int b) {
    cudaError_t e = cudaEventSynchronize(copied[b]);
    if (e == cudaSuccess && h->timing && exec[b]) {
      for (auto& r : recs[b]) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
          h->t_ms[r.kind] += ms;
          h->t_cnt[r.kind] += 1;
        }
      }
    }
    if (e == cudaSuccess && h->timing && !exec[b]) flush_timing(h);
    return e;
  }
  // Run batches until no active slot is still iterating (or max_batches).
  int run(const std::vector<int>& active, int max_batches) {
    int cur = 0;
    if (cudaError_t e = launch(cur)) return map_err(e);
    for (int n = 1;; ++n) {
      const bool ahead = n < max_batches;
      if (ahead) {
        if (cudaError_t e = launch(1 - cur)) return map_err(e);
      }
      if (cudaError_t e = wait(cur)) return map_err(e);
      bool running = false;
      for (int l = 0; l < L; ++l)
        if (active[l] && host[cur][l].status == ST_RUN) running = true;
      if (!running || !ahead) {
        if (ahead) {
          if (cudaError_t e = wait(1 - cur)) return map_err(e);
        }
        return RVE_OK;
      }
      cur = 1 - cur;
    }
  }
};

// The solve driver, in phases so that a batch can run several handles in
// lockstep (FeSolve::begin, then per refinement step outer() -> the inner
// projected CG -> after_inner(), then finish()).  u_out [L][D][N] receives the
// FP64 nodal fluctuation.
template <typename T> struct FeSolve {
  rve_s* h;
  int L;
  double rel_tol;
  int max_iter;
  double* u_out;
  double* emac_dev;
  bool mixed;
  double inner_tol;
  int max_outer;
  int step = 0;
  std::vector<double> f0, frel, cgrel;
  std::vector<int> iters, steps, bad, active, floor_hit, timeout;
  Fp64Args fa;
  PassArgs<T> a;

  FeSolve(rve_s* h_, int L_, double rel_tol_, int max_iter_, double* u_out_, double* emac_dev_)
      : h(h_), L(L_), rel_tol(rel_tol_), max_iter(max_iter_), u_out(u_out_), emac_dev(emac_dev_),
        mixed(h_->tsize == 4), inner_tol(mixed ? std::fmax(rel_tol_, 2e-5) : rel_tol_), max_outer(mixed ? 12 : 6),
        f0(L_, 0.0), frel(L_, 0.0), cgrel(L_, 0.0), iters(L_, 0), steps(L_, 0), bad(L_, 0), active(L_, 1),
        floor_hit(L_, 0), timeout(L_, 0) {}

  int begin(const double* emac_host) {
    CK(cudaMemcpyAsync(emac_dev, emac_host, (size_t)L * h->ns * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(u_out, 0, (size_t)L * h->D * h->N * sizeof(double), h->stream));
    std::memset(h->cg_h, 0, (size_t)L * sizeof(CgState));
    for (int l = 0; l < L; ++l) { h->cg_h[l].active = 1; h->cg_h[l].status = ST_RUN; }
    int rc = write_state(h, L);
    if (rc) return rc;
    fa = fp64_args(h, L, u_out, emac_dev, h->cg);
    a = pass_args<T>(h, L, u_out, emac_dev);
    return RVE_OK;
  }

  // FP64 residual of the current iterate; decide which load cases go on; for
  // those, the inner right-hand side and the CG state.  *need = false: done.
  // hold: the slots that go on are left held (ST_HOLD) for the caller to
  // release, instead of running.
  int outer(bool* need, bool hold = false) {
    *need = false;
    CK(timed(h, K_RES, [&] { return launch_residual(fa, h->stream); }));
    int rc = read_state(h, L);
    if (rc) return rc;
    bool any = false;
    for (int l = 0; l < L; ++l) {
      if (!active[l]) continue;
      const double fn2 = h->cg_h[l].fn2;
      if (step == 0) f0[l] = std::sqrt(fn2);
      if (!std::isfinite(fn2)) { bad[l] = 1; active[l] = 0; continue; }
      const double prev = frel[l];
      frel[l] = (f0[l] > 0.0) ? std::sqrt(fn2) / f0[l] : 0.0;
      // Round-off level of f: a bound on the rounding error of summing the
      // terms of every nodal force in FP64 (backward-error floor).  A load
      // case whose residual is below it is solved, even if f_0 itself is at
      // that level (the macroscopic strain is already an equilibrium state).
      const double floor_abs = 64.0 * 2.220446049250313e-16 * std::sqrt(h->cg_h[l].fa2);
      const bool at_floor = std::sqrt(fn2) <= floor_abs;
      if (at_floor) floor_hit[l] = 1;
      // stop: tolerance met, at the round-off floor, step or iteration budget
      // spent, or no progress
      const bool stalled = step >= 2 && frel[l] > 0.5 * prev;
      if (frel[l] <= rel_tol || at_floor || step >= max_outer || iters[l] >= max_iter || stalled) {
        active[l] = 0;
        continue;
      }
      any = true;
    }
    if (!any) return RVE_OK;
    for (int l = 0; l < L; ++l) {
      h->cg_h[l].active = active[l];
      h->cg_h[l].status = hold ? ST_HOLD : ST_RUN;
      h->cg_h[l].it = 0;
      h->cg_h[l].maxit = max_iter - iters[l];
      // do not solve further than the outer tolerance needs: after a first
      // step the residual has to fall by rel_tol / frel only (with a margin of
      // 10 for the different norms of the inner and outer residuals).  This
      // also keeps a later inner solve from chasing the rounding noise of its
      // right-hand side, which with zero-stiffness regions has parts the
      // semi-definite operator cannot reduce.
      double tl = inner_tol;
      if (step > 0 && frel[l] > 0.0) tl = std::fmax(tl, std::fmin(0.5, 0.1 * rel_tol / frel[l]));
      h->cg_h[l].tol2 = tl * tl;
      h->cg_h[l].cnt_a = h->cg_h[l].cnt_e = h->cg_h[l].cnt_r = 0;
    }
    if ((rc = write_state(h, L))) return rc;
    // inner right-hand side r0 = -G C (E + B u) from f (nodal state: rho0 = -K^-1 f)
    a.cgphase = 0;
    if (h->op_form == RVE_FORM_NODAL) {
      NodalBufs<T> nb(h, L);
      PassArgs<T> b = a;
      b.amode = A_NODAL; b.pmode = P_SOLVE; b.emode = E_NOUT;
      b.in = nb.f; b.out = nb.w;
      CK(apply_passes<T>(h, b));
      CK(timed(h, K_OTHER, [&] { return launch_nodal_update<T>(a, nullptr, nb.w, nb.rho[0], nb.xi, 1, h->stream); }));
    } else {
      a.amode = A_NODAL; a.pmode = P_NODAL_IN; a.emode = E_INIT;
      a.in = (const T*)h->fbuf;
      CK(apply_passes<T>(h, a));
    }
    // the arguments of the projected-CG iterations
    a.cgphase = 1; a.amode = A_CG; a.pmode = P_G; a.emode = E_CG;
    *need = true;
    return RVE_OK;
  }

  // After the inner CG: the deferred x update, statistics, u += the correction.
  int after_inner() {
    // apply the x update the last iteration deferred (nodal state: and u += xi)
    if (h->op_form == RVE_FORM_NODAL) {
      NodalBufs<T> nb(h, L);
      CK(timed(h, K_OTHER, [&] { return launch_nodal_finish<T>(a, nb.pi[0], nb.pi[1], nb.xi, h->stream); }));
    } else {
      CK(timed(h, K_OTHER, [&] { return launch_cg_finish_x<T>(a, h->stream); }));
    }
    int rc = read_state(h, L);
    if (rc) return rc;
    for (int l = 0; l < L; ++l) {
      if (!active[l]) continue;
      iters[l] += h->cg_h[l].it;
      steps[l] += 1;
      cgrel[l] = h->cg_h[l].rr0 > 0 ? std::sqrt(h->cg_h[l].rr / h->cg_h[l].rr0) : 0.0;
      if (h->cg_h[l].status == ST_BAD) bad[l] = 1;
      if (h->cg_h[l].pad == kTimeoutMark) timeout[l] = 1;
    }
    // u += (B^H B)^-1 B^H delta  (delta = CG iterate x; the nodal state added xi above)
    if (h->op_form != RVE_FORM_NODAL) {
      a.cgphase = 0; a.amode = A_BARE; a.pmode = P_NODAL_OUT; a.emode = E_NODAL;
      a.in = (const T*)h->x;
      CK(apply_passes<T>(h, a));
    }
    for (int l = 0; l < L; ++l)
      if (bad[l]) { active[l] = 0; h->cg_h[l].active = 0; }
    if ((rc = write_state(h, L))) return rc;
    ++step;
    return RVE_OK;
  }

  // Take every slot out of the CG kernels (a finished handle whose kernels
  // still run in a lockstep batch graph then exits at once).
  int deactivate() {
    for (int l = 0; l < L; ++l) h->cg_h[l].active = 0;
    return write_state(h, L);
  }

  int finish(rve_info* info) const {
    int worst = RVE_OK;
    for (int l = 0; l < L; ++l) {
      int st = RVE_OK;
      if (timeout[l]) st = RVE_ERR_TIMEOUT;
      else if (bad[l]) st = RVE_ERR_NONFINITE;
      else if (frel[l] > rel_tol && !floor_hit[l]) st = RVE_ERR_NOT_CONVERGED;
      if (info) {
        info[l].iterations = iters[l];
        info[l].refine_steps = steps[l];
        info[l].status = st;
        info[l].reserved = 0;
        info[l].rel_residual = frel[l];
        info[l].cg_rel_residual = cgrel[l];
      }
      if (st == RVE_ERR_TIMEOUT || (st == RVE_ERR_NONFINITE && worst != RVE_ERR_TIMEOUT) ||
          (st != RVE_OK && worst == RVE_OK))
        worst = st;
    }
    return worst;
  }
};

constexpr int kCheckEvery = 8;  // CG iterations per graph; even: the factored form alternates its buffers

template <typename T>
int solve_impl(rve_s* h, const double* emac_host, int L, double rel_tol, int max_iter, rve_info* info,
               double* u_out, double* emac_dev) {
  FeSolve<T> sv(h, L, rel_tol, max_iter, u_out, emac_dev);
  int rc = sv.begin(emac_host);
  if (rc) return rc;
  std::unique_ptr<CgRunner<T>> runner;  // built at the first inner solve, reused by later ones
  for (;;) {
    bool need = false;
    if ((rc = sv.outer(&need))) return rc;
    if (!need) break;
    if (!runner) runner.reset(new CgRunner<T>(h, L, sv.a, kCheckEvery));
    if ((rc = runner->run(sv.active, (max_iter + kCheckEvery - 1) / kCheckEvery + 1))) return rc;
    if ((rc = sv.after_inner())) return rc;
  }
  return sv.finish(info);
}

// Release held slots of a handle: ST_HOLD -> ST_RUN (one block).
__global__ void release_held(CgState* cg, int L) {
  for (int l = threadIdx.x; l < L; l += blockDim.x)
    if (cg[l].status == ST_HOLD) cg[l].status = ST_RUN;
}

// The projected-CG iterations of several handles (the size groups of a
// batch) as ONE CUDA graph per batch of K iterations: a fork from the batch's
// stream to every handle's stream, K iterations of every handle on its own
// stream (parallel branches of the graph), each branch's copy of its CG states
// to its pinned host buffer, and a join back.  Two copies of the graph are
// launched alternately as in CgRunner, so the host checks batch i while batch
// i+1 runs.  Every kernel skips the slots whose CG stopped or that are not
// active (per-RVE, per-load-case masks): a handle that has finished costs
// only the early exits of its kernels.
template <typename T> struct MultiRunner {
  cudaStream_t root;
  std::vector<rve_s*> hs;
  std::vector<int> Ls;
  std::vector<PassArgs<T>> as;
  int K;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, copied[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> join;
  // pinned host copies of every handle's CG states, one per graph copy (the
  // handles' own buffers stay free for their refinement steps)
  std::vector<CgState*> hbuf[2];

  CgState* host(int b, size_t i) { return hbuf[b][i]; }

  // Fork, K iterations of every handle, state copies, join (captured or direct).
  cudaError_t issue(int b) {
    cudaError_t e = cudaEventRecord(fork, root);
    for (size_t i = 0; i < hs.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(hs[i]->stream, fork, 0);
    for (size_t i = 0; i < hs.size() && e == cudaSuccess; ++i) {
      for (int k = 0; k < K && e == cudaSuccess; ++k) e = cg_iteration<T>(hs[i], as[i], k);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(host(b, i), hs[i]->cg, (size_t)Ls[i] * sizeof(CgState), cudaMemcpyDeviceToHost,
                            hs[i]->stream);
      if (e == cudaSuccess) e = cudaEventRecord(join[i], hs[i]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(root, join[i], 0);
    }
    return e;
  }

  MultiRunner(cudaStream_t root_, const std::vector<rve_s*>& hs_, const std::vector<int>& Ls_,
              const std::vector<PassArgs<T>>& as_, int K_)
      : root(root_), hs(hs_), Ls(Ls_), as(as_), K(K_), join(hs_.size(), nullptr) {
    for (int b = 0; b < 2; ++b) {
      hbuf[b].assign(hs.size(), nullptr);
      for (size_t i = 0; i < hs.size(); ++i)
        if (cudaMallocHost((void**)&hbuf[b][i], (size_t)Ls[i] * sizeof(CgState)) != cudaSuccess) {
          cudaGetLastError();
          hbuf[b][i] = nullptr;
        }
    }
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (auto& ev : join) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (int b = 0; b < 2; ++b) cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
    for (int b = 0; b < 2; ++b) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      const cudaError_t e = issue(b);
      const cudaError_t e2 = cudaStreamEndCapture(root, &g);
      if (e != cudaSuccess || e2 != cudaSuccess || !g || cudaGraphInstantiate(&exec[b], g, 0) != cudaSuccess) {
        cudaGetLastError();
        exec[b] = nullptr;
      }
      if (g) cudaGraphDestroy(g);
      if (!exec[b]) break;
    }
    if (!exec[0] || !exec[1])
      for (int b = 0; b < 2; ++b) {
        if (exec[b]) cudaGraphExecDestroy(exec[b]);
        exec[b] = nullptr;
      }
  }
  ~MultiRunner() {
    for (int b = 0; b < 2; ++b) {
      if (exec[b]) cudaGraphExecDestroy(exec[b]);
      if (copied[b]) cudaEventDestroy(copied[b]);
    }
    if (fork) cudaEventDestroy(fork);
    for (auto& ev : join)
      if (ev) cudaEventDestroy(ev);
    for (int b = 0; b < 2; ++b)
      for (auto* p : hbuf[b])
        if (p) cudaFreeHost(p);
  }
  bool ok() const {
    for (int b = 0; b < 2; ++b)
      for (auto* p : hbuf[b])
        if (!p) return false;
    return true;
  }
  cudaError_t launch(int b) {
    cudaError_t e = exec[b] ? cudaGraphLaunch(exec[b], root) : issue(b);
    if (e == cudaSuccess) e = cudaEventRecord(copied[b], root);
    return e;
  }
  // Order the batch stream after the work queued on the given handles' streams.
  int sync_in(const std::vector<size_t>& which) {
    for (size_t i : which)
      if (cudaEventRecord(join[i], hs[i]->stream) != cudaSuccess || cudaStreamWaitEvent(root, join[i], 0) != cudaSuccess) {
        cudaGetLastError();
        return RVE_ERR_CUDA;
      }
    return RVE_OK;
  }
  // ... and every handle's stream after the batch stream.
  int sync_out() {
    if (cudaEventRecord(fork, root) != cudaSuccess) { cudaGetLastError(); return RVE_ERR_CUDA; }
    for (auto* h : hs)
      if (cudaStreamWaitEvent(h->stream, fork, 0) != cudaSuccess) { cudaGetLastError(); return RVE_ERR_CUDA; }
    return RVE_OK;
  }
  // No active slot of handle i is still iterating in the state copy of batch b.
  bool idle(int b, size_t i, const std::vector<int>& active) {
    for (int l = 0; l < Ls[i]; ++l)
      if (active[l] && host(b, i)[l].status == ST_RUN) return false;
    return true;
  }
  // Launch batches until every handle is done.  A handle whose inner solve has
  // finished (no active slot still iterating) is handed to transition(i) at
  // once, while the graph launched after that state copy is still in flight:
  // the handle's slots are not running, so that graph's branch for it only
  // exits early, and transition() prepares the next refinement step with the
  // slots held (ST_HOLD).  The held slots are released by a kernel on the
  // handle's stream that waits for the in-flight graph, and the next graph
  // waits for the release, so a branch never sees a handle's state change in
  // the middle of a graph.  A handle's state copies count again from the first
  // graph launched after its release.  max_batches bounds the launches.
  template <class Transition>
  int drive(const std::vector<const std::vector<int>*>& active, std::vector<char>& done, Transition transition,
            long max_batches) {
    const size_t G = hs.size();
    std::vector<size_t> all(G);
    for (size_t i = 0; i < G; ++i) all[i] = i;
    if (int rc = sync_in(all)) return rc;
    std::vector<long> valid_from(G, 0);   // first graph whose copy of the handle's state counts
    long idx[2] = {-1, -1};               // graph last launched into each copy
    long launched = 0;
    int cur = 0;
    if (cudaError_t e = launch(cur)) return map_err(e);
    idx[cur] = launched++;
    bool other = false;                   // the other copy is in flight
    for (;;) {
      if (launched < max_batches) {
        if (cudaError_t e = launch(1 - cur)) return map_err(e);
        idx[1 - cur] = launched++;
        other = true;
      }
      if (cudaError_t e = cudaEventSynchronize(copied[cur])) return map_err(e);
      std::vector<size_t> ready;
      for (size_t i = 0; i < G; ++i)
        if (!done[i] && idx[cur] >= valid_from[i] && idle(cur, i, *active[i])) ready.push_back(i);
      for (size_t i : ready) {
        if (int rc = transition(i)) return rc;
        if (done[i]) continue;
        // release after the graph in flight (if any), before the next one
        if (other && cudaStreamWaitEvent(hs[i]->stream, copied[1 - cur], 0) != cudaSuccess) {
          cudaGetLastError();
          return RVE_ERR_CUDA;
        }
        release_held<<<1, 64, 0, hs[i]->stream>>>(hs[i]->cg, Ls[i]);
        if (cudaGetLastError() != cudaSuccess) return RVE_ERR_CUDA;
        if (int rc = sync_in({i})) return rc;
        valid_from[i] = launched;
      }
      bool all_done = true;
      for (size_t i = 0; i < G; ++i) all_done = all_done && done[i];
      if (all_done || !other) {
        if (other) {
          if (cudaError_t e = cudaEventSynchronize(copied[1 - cur])) return map_err(e);
        }
        if (int rc = sync_out()) return rc;
        if (all_done || launched >= max_batches) return RVE_OK;
        // nothing in flight and budget left (cannot happen with run-ahead on); restart
        cur = 0;
        if (cudaError_t e = launch(cur)) return map_err(e);
        idx[cur] = launched++;
        continue;
      }
      cur = 1 - cur;
      other = false;
    }
  }
};

// A batch solve from one host thread: every size group runs the refinement
// phases of FeSolve, and the inner projected CG of all groups runs as one
// graph per K iterations (MultiRunner); a group moves to its next refinement
// step as soon as its own inner solve has finished.  emacs[g] are the
// macroscopic strains of group g's slots; infos[g] receives their statistics
// and codes[g] their status (the return value is an error of the whole call).
template <typename T>
int batch_lockstep(cudaStream_t root, const std::vector<rve_s*>& hs, const std::vector<std::vector<double>>& emacs,
                   double rel_tol, int max_iter, std::vector<std::vector<rve_info>>& infos, std::vector<int>& codes) {
  const size_t G = hs.size();
  std::vector<std::unique_ptr<FeSolve<T>>> sv(G);
  std::vector<int> Ls(G);
  std::vector<char> done(G, 0);
  bool any = false;
  for (size_t g = 0; g < G; ++g) {
    Ls[g] = (int)(emacs[g].size() / hs[g]->ns);
    sv[g].reset(new FeSolve<T>(hs[g], Ls[g], rel_tol, max_iter, hs[g]->u, hs[g]->emac_d));
    if (int rc = sv[g]->begin(emacs[g].data())) return rc;
    bool need = false;
    if (int rc = sv[g]->outer(&need)) return rc;
    if (!need) {
      done[g] = 1;
      if (int rc = sv[g]->deactivate()) return rc;
    }
    any = any || need;
  }
  if (any) {
    std::vector<PassArgs<T>> as(G);
    std::vector<const std::vector<int>*> act(G);
    for (size_t g = 0; g < G; ++g) {
      as[g] = sv[g]->a;  // the CG-iteration arguments (outer() leaves them so for a group that iterates)
      as[g].cgphase = 1; as[g].amode = A_CG; as[g].pmode = P_G; as[g].emode = E_CG;
      act[g] = &sv[g]->active;
    }
    MultiRunner<T> runner(root, hs, Ls, as, kCheckEvery);
    if (!runner.ok()) return RVE_ERR_OOM;
    auto transition = [&](size_t g) -> int {
      if (int rc = sv[g]->after_inner()) return rc;
      bool need = false;
      if (int rc = sv[g]->outer(&need, true)) return rc;
      if (!need) {
        done[g] = 1;
        return sv[g]->deactivate();
      }
      return RVE_OK;
    };
    const long per_solve = (max_iter + kCheckEvery - 1) / kCheckEvery + 1;
    const long max_batches = 1 + (long)G * 13 * per_solve;   // every group's refinement steps in turn
    if (int rc = runner.drive(act, done, transition, max_batches)) return rc;
    for (size_t g = 0; g < G; ++g)
      if (!done[g])
        if (int rc = sv[g]->after_inner()) return rc;
  }
  for (size_t g = 0; g < G; ++g) {
    infos[g].resize(Ls[g]);
    codes[g] = sv[g]->finish(infos[g].data());
  }
  return RVE_OK;
}

// Plain projected CG on the strain fluctuation (the scheme of Sec. 2.1 as the
// oracle runs it), for derivatives without a finite-element stencil: no nodal
// state and no real-space residual, FP64 throughout.  r0 = -G C E (pass A
// broadcasts E), stop on ||r|| <= rel_tol ||r0||; x holds the fluctuation.
int solve_strain_state(rve_s* h, const double* emac_host, int L, double rel_tol, int max_iter, rve_info* info) {
  using T = double;
  CK(cudaMemcpyAsync(h->emac_d, emac_host, (size_t)L * h->ns * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  std::memset(h->cg_h, 0, (size_t)L * sizeof(CgState));
  for (int l = 0; l < L; ++l) {
    h->cg_h[l].active = 1;
    h->cg_h[l].status = ST_RUN;
    h->cg_h[l].maxit = max_iter;
    h->cg_h[l].tol2 = rel_tol * rel_tol;
  }
  int rc = write_state(h, L);
  if (rc) return rc;
  PassArgs<T> a = pass_args<T>(h, L, h->u, h->emac_d);
  a.cgphase = 0; a.amode = A_MACRO; a.pmode = P_G; a.emode = E_INIT;
  CK(apply_passes<T>(h, a));
  a.cgphase = 1; a.amode = A_CG; a.pmode = P_G; a.emode = E_CG;
  {
    CgRunner<T> runner(h, L, a, 8);
    std::vector<int> active(L, 1);
    if ((rc = runner.run(active, (max_iter + 7) / 8 + 1))) return rc;
  }
  CK(timed(h, K_OTHER, [&] { return launch_cg_finish_x<T>(a, h->stream); }));
  if ((rc = read_state(h, L))) return rc;
  int worst = RVE_OK;
  for (int l = 0; l < L; ++l) {
    const CgState& c = h->cg_h[l];
    int st = RVE_OK;
    if (c.status == ST_BAD) st = RVE_ERR_NONFINITE;
    else if (c.status != ST_CONV) st = RVE_ERR_NOT_CONVERGED;
    const double rel = c.rr0 > 0 ? std::sqrt(c.rr / c.rr0) : 0.0;
    if (info) {
      info[l].iterations = c.it;
      info[l].refine_steps = 1;
      info[l].status = st;
      info[l].reserved = 0;
      info[l].rel_residual = rel;
      info[l].cg_rel_residual = rel;
    }
    if (st == RVE_ERR_NONFINITE || (st != RVE_OK && worst == RVE_OK)) worst = st;
  }
  return worst;
}

// Finite strain (St. Venant-Kirchhoff), FP64: Newton on G P(F) = 0 with each
// correction from projected CG on G K(F) dH = -G P(F) (Eq.
// stat-mech-equi-FFT-homogenization with the gradient projection of Eq.
// original-G).  Newton stops when ||G P(F)|| <= rel_tol ||G P(F_macro)|| or
// at the round-off level of |P|; the CG of step k stops at a relative
// residual of max(min(1e-2, frel_k), 0.1 rel_tol / frel_k), capped at 0.5.
int solve_finite(rve_s* h, const double* Fmac_host, int L, double rel_tol, int max_newton, int max_iter,
                 rve_info* info) {
  const int D = h->dim, DD = D * D;
  if (!h->Fs && dev_alloc((void**)&h->Fs, (size_t)h->Lcap * h->m * h->N * sizeof(double))) return RVE_ERR_OOM;
  if (!h->fmac_d && dev_alloc((void**)&h->fmac_d, (size_t)64 * 9 * sizeof(double))) return RVE_ERR_OOM;
  CK(cudaMemcpyAsync(h->fmac_d, Fmac_host, (size_t)L * DD * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  std::memset(h->cg_h, 0, (size_t)L * sizeof(CgState));
  for (int l = 0; l < L; ++l) { h->cg_h[l].active = 1; h->cg_h[l].status = ST_RUN; }
  int rc = write_state(h, L);
  if (rc) return rc;
  PassArgs<double> a = pass_args<double>(h, L, h->u, h->emac_d);
  CK(timed(h, K_OTHER, [&] { return launch_fs_init(a, h->Fs, h->fmac_d, h->stream); }));
  std::vector<double> r0(L, 0.0), frel(L, 1.0), cgrel(L, 0.0);
  std::vector<int> iters(L, 0), steps(L, 0), active(L, 1), bad(L, 0), done(L, 0);
  std::unique_ptr<CgRunner<double>> runner;
  for (int newton = 0;; ++newton) {
    // residual r = -G P(F) (pass E in init mode also zeroes x and sets rr0)
    a.cgphase = 0;
    CK(timed(h, K_RES, [&] { return launch_fs_stress(a, h->Fs, (double*)h->fbuf, h->stream); }));
    PassArgs<double> b = a;
    b.amode = A_BARE; b.pmode = P_FINITE; b.emode = E_INIT;
    b.in = (const double*)h->fbuf;
    CK(apply_passes<double>(h, b));
    if ((rc = read_state(h, L))) return rc;
    bool any = false;
    for (int l = 0; l < L; ++l) {
      if (!active[l]) continue;
      const double rn = std::sqrt(h->cg_h[l].rr0);
      if (!std::isfinite(rn)) { bad[l] = 1; active[l] = 0; continue; }
      if (newton == 0) r0[l] = rn;
      frel[l] = r0[l] > 0.0 ? rn / r0[l] : 0.0;
      const bool at_floor = rn <= 1e-13 * std::sqrt(h->cg_h[l].fa2);
      if (at_floor || frel[l] <= rel_tol) { done[l] = 1; active[l] = 0; continue; }
      if (newton >= max_newton || iters[l] >= max_iter) { active[l] = 0; continue; }
      any = true;
    }
    if (!any) break;
    for (int l = 0; l < L; ++l) {
      double tau = std::fmax(std::fmin(1e-2, frel[l]), 0.1 * rel_tol / std::fmax(frel[l], 1e-300));
      tau = std::fmin(tau, 0.5);
      h->cg_h[l].active = active[l];
      h->cg_h[l].status = ST_RUN;
      h->cg_h[l].it = 0;
      h->cg_h[l].maxit = max_iter - iters[l];
      h->cg_h[l].tol2 = tau * tau;
      h->cg_h[l].cnt_a = h->cg_h[l].cnt_e = h->cg_h[l].cnt_r = 0;
    }
    if ((rc = write_state(h, L))) return rc;
    a.cgphase = 1; a.amode = A_BARE; a.pmode = P_FINITE; a.emode = E_CG;
    if (!runner) runner.reset(new CgRunner<double>(h, L, a, 8));
    if ((rc = runner->run(active, (max_iter + 7) / 8 + 1))) return rc;
    CK(timed(h, K_OTHER, [&] { return launch_cg_finish_x<double>(a, h->stream); }));
    if ((rc = read_state(h, L))) return rc;
    for (int l = 0; l < L; ++l) {
      if (!active[l]) continue;
      iters[l] += h->cg_h[l].it;
      steps[l] += 1;
      cgrel[l] = h->cg_h[l].rr0 > 0 ? std::sqrt(h->cg_h[l].rr / h->cg_h[l].rr0) : 0.0;
      if (h->cg_h[l].status == ST_BAD) bad[l] = 1;
    }
    CK(timed(h, K_OTHER, [&] { return launch_fs_add(a, h->Fs, h->stream); }));
    for (int l = 0; l < L; ++l)
      if (bad[l]) { active[l] = 0; h->cg_h[l].active = 0; }
    for (int l = 0; l < L; ++l) h->cg_h[l].active = active[l];
    if ((rc = write_state(h, L))) return rc;
  }
  // mean first Piola-Kirchhoff stress over all elements
  for (int l = 0; l < L; ++l) h->cg_h[l].active = 1;
  if ((rc = write_state(h, L))) return rc;
  const int nb = fs_mean_blocks(a);
  const size_t need = (size_t)L * DD * nb;
  if ((int)need > h->hpart_cap) {
    free_devp(h->hpart);
    if ((rc = dev_alloc((void**)&h->hpart, need * sizeof(double)))) return rc;
    h->hpart_cap = (int)need;
  }
  CK(timed(h, K_OTHER, [&] { return launch_fs_mean(a, h->Fs, h->hpart, h->stream); }));
  std::vector<double> hp(need);
  CK(cudaMemcpyAsync(hp.data(), h->hpart, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) flush_timing(h);
  h->P_h.assign((size_t)L * DD, 0.0);
  const double scale = 1.0 / ((double)h->N * (D == 2 ? 2 : 6));
  for (int l = 0; l < L; ++l)
    for (int c = 0; c < DD; ++c) {
      double t = 0.0;
      const double* src = hp.data() + ((size_t)l * DD + c) * nb;
      for (int q = 0; q < nb; ++q) t += src[q];
      h->P_h[(size_t)l * DD + c] = t * scale;
    }
  int worst = RVE_OK;
  for (int l = 0; l < L; ++l) {
    int st = bad[l] ? RVE_ERR_NONFINITE : (done[l] ? RVE_OK : RVE_ERR_NOT_CONVERGED);
    if (info) {
      info[l].iterations = iters[l];
      info[l].refine_steps = steps[l];
      info[l].status = st;
      info[l].reserved = 0;
      info[l].rel_residual = frel[l];
      info[l].cg_rel_residual = cgrel[l];
    }
    if (st == RVE_ERR_NONFINITE || (st != RVE_OK && worst == RVE_OK)) worst = st;
  }
  return worst;
}

int compute_mean_stress(rve_s* h, int L) {
  // reuse cg[] slots with active = 1 (homogenise does not read them)
  Fp64Args fa = fp64_args(h, L, h->u, h->emac_d, h->cg);
  const int nblk = homogenise_blocks(fa);
  const size_t need = (size_t)L * h->ns * nblk;
  if ((int)need > h->hpart_cap) {
    free_devp(h->hpart);
    int rc = dev_alloc((void**)&h->hpart, need * sizeof(double));
    if (rc) return rc;
    h->hpart_cap = (int)need;
  }
  int nb = 0;
  if (h->deriv == D_FE) {
    CK(timed(h, K_OTHER, [&] { return launch_homogenise(fa, h->hpart, &nb, h->stream); }));
  } else {
    CK(timed(h, K_OTHER, [&] { return launch_homogenise_strain(fa, (const double*)h->x, h->hpart, &nb, h->stream); }));
  }
  std::vector<double> hp(need);
  CK(cudaMemcpyAsync(hp.data(), h->hpart, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) flush_timing(h);
  h->S_h.assign((size_t)L * h->ns, 0.0);
  const double scale = 1.0 / ((double)h->N * h->nq);
  for (int l = 0; l < L; ++l)
    for (int s = 0; s < h->ns; ++s) {
      double t = 0.0;
      const double* src = hp.data() + ((size_t)l * h->ns + s) * nb;
      for (int b = 0; b < nb; ++b) t += src[b];
      h->S_h[(size_t)l * h->ns + s] = t * scale;
    }
  return RVE_OK;
}

// Gauss-Jordan inverse of a small row-major matrix; false if singular.
bool invert(int n, const double* A, double* Ainv) {
  std::vector<double> M((size_t)n * 2 * n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) M[i * 2 * n + j] = A[i * n + j];
    M[i * 2 * n + n + i] = 1.0;
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i) if (std::fabs(M[i * 2 * n + c]) > std::fabs(M[piv * 2 * n + c])) piv = i;
    if (std::fabs(M[piv * 2 * n + c]) < 1e-300) return false;
    if (piv != c) for (int j = 0; j < 2 * n; ++j) std::swap(M[c * 2 * n + j], M[piv * 2 * n + j]);
    const double d = M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = M[i * 2 * n + c];
      if (f != 0.0) for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] -= f * M[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
  return true;
}

__global__ void f32_from_f64(const double* in, float* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// (Re)allocate the material buffers of a handle for n_mat fields.
int alloc_materials(rve_s* h, int n_mat) {
  if (h->Ein && h->Ein != (void*)h->E64) cudaFree(h->Ein);
  h->Ein = nullptr;
  free_devp(h->E64);
  int rc = dev_alloc((void**)&h->E64, (size_t)n_mat * h->N * sizeof(double));
  if (rc) return rc;
  if (h->precision == RVE_MIXED) {
    rc = dev_alloc(&h->Ein, (size_t)n_mat * h->N * sizeof(float));
    if (rc) return rc;
  } else {
    h->Ein = h->E64;
  }
  h->n_mat = n_mat;
  return RVE_OK;
}

// Moduli must be finite and >= 0 (zero-stiffness voxels model vacuum, which
// the linear-FE projection decouples, Sec. 3.2), with at least one > 0.
int check_moduli(const std::vector<double>& e64) {
  bool any = false;
  for (double v : e64) {
    if (!(v >= 0.0) || !std::isfinite(v)) return RVE_ERR_ARG;
    any = any || v > 0.0;
  }
  return any ? RVE_OK : RVE_ERR_ARG;
}

// Validated FP64 copy of a modulus field on the host.
int read_moduli(int64_t N, const void* E, int E_dtype, int ptr_flags, std::vector<double>& e64) {
  e64.resize((size_t)N);
  if (ptr_flags & RVE_PTR_DEVICE) {
    if (E_dtype == RVE_F64) {
      CK(cudaMemcpy(e64.data(), E, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> e32((size_t)N);
      CK(cudaMemcpy(e32.data(), E, (size_t)N * sizeof(float), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < N; ++i) e64[i] = e32[i];
    }
  } else {
    if (E_dtype == RVE_F64) std::memcpy(e64.data(), E, (size_t)N * sizeof(double));
    else for (int64_t i = 0; i < N; ++i) e64[i] = ((const float*)E)[i];
  }
  return check_moduli(e64);
}

// Upload field `slot` (FP64 host copy) and its inner-precision copy.
int upload_material(rve_s* h, int slot, const std::vector<double>& e64) {
  double* dst = h->E64 + (size_t)slot * h->N;
  if (int rc = copy_sync(h, dst, e64.data(), (size_t)h->N * sizeof(double), cudaMemcpyHostToDevice)) return rc;
  if (h->precision == RVE_MIXED) {
    f32_from_f64<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(dst, (float*)h->Ein + (size_t)slot * h->N,
                                                                          h->N);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
  }
  return RVE_OK;
}

void set_nu(rve_s* h, double nu) {
  h->nu = nu;
  h->lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));  // unit Young's modulus
  h->mu2 = 1.0 / (1.0 + nu);
}

// C = S^T M^-T for the L = n_s load cases of one RVE (rows S[l][:]).
int tangent_from_stress(int ns, const double* S, const double* emac, double* C) {
  std::vector<double> Minv((size_t)ns * ns);
  if (!invert(ns, emac, Minv.data())) return RVE_ERR_ARG;
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < ns; ++t) {
      double v = 0.0;
      for (int l = 0; l < ns; ++l) v += S[(size_t)l * ns + s] * Minv[(size_t)t * ns + l];
      C[s * ns + t] = v;
    }
  return RVE_OK;
}

}  // namespace

struct rve_batch_s {
  int dim = 0, count = 0, precision = RVE_FP64;
  int device = -1;              // the device current at rve_batch_create
  double nu = 0.3;
  struct Group {
    int n[3] = {1, 1, 1};
    std::vector<int> members;   // RVE indices
    std::vector<char> has_mat;
    rve_s* h = nullptr;
    cudaStream_t stream = nullptr;
  };
  std::vector<Group> groups;
  cudaStream_t root = nullptr;  // the stream the batch's CG graphs are launched on
  std::vector<int> group_of, slot_of;
  int L = 0;
  bool solved = false;
  std::vector<double> emac;     // [L][ns]
};

// ====================================================================
extern "C" {

const char* rve_error_string(int code) {
  switch (code) {
    case RVE_OK: return "ok";
    case RVE_ERR_ARG: return "invalid argument or call order";
    case RVE_ERR_UNSUPPORTED_SIZE: return "grid size not supported by the GPU FFT (powers of two, 16..1024 in 2D, 16..256 in 3D)";
    case RVE_ERR_CUDA: return "CUDA runtime error";
    case RVE_ERR_OOM: return "device memory allocation failed";
    case RVE_ERR_NOT_CONVERGED: return "iteration limit reached before the tolerance";
    case RVE_ERR_NONFINITE: return "non-finite value or CG breakdown";
    case RVE_ERR_TIMEOUT: return "device-side wait exceeded its limit";
    case RVE_ERR_SCRATCH_LIMIT: return "grid exceeds the static scratch of the allocation-free entry point (n <= 256 per axis)";
    default: return "unknown status";
  }
}

int rve_create(rve_t* out, int dim, const int64_t* n, const double* length, int precision, void* cuda_stream) {
  if (!out || !n || (dim != 2 && dim != 3) || (precision != RVE_FP64 && precision != RVE_MIXED)) return RVE_ERR_ARG;
  *out = nullptr;
  const int64_t maxn = (dim == 2) ? 1024 : 256;
  for (int a = 0; a < dim; ++a) {
    if (!is_pow2(n[a]) || n[a] < 16 || n[a] > maxn) return RVE_ERR_UNSUPPORTED_SIZE;
    if (length && !(length[a] > 0.0 && std::isfinite(length[a]))) return RVE_ERR_ARG;
  }
  rve_s* h = new (std::nothrow) rve_s();
  if (!h) return RVE_ERR_OOM;
  h->dim = dim;
  h->N = 1;
  for (int a = 0; a < dim; ++a) { h->n[a] = (int)n[a]; h->N *= n[a]; h->len[a] = length ? length[a] : 1.0; }
  h->precision = precision;
  h->user_stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return RVE_ERR_CUDA;
  }
  h->ns = dim == 2 ? 3 : 6;
  h->nq = dim == 2 ? 2 : 6;
  h->m = h->ns * h->nq;
  h->D = dim;
  h->kx = h->n[0] / 2 + 1;
  h->tsize = precision == RVE_MIXED ? 4 : 8;
  if (cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); delete h; return RVE_ERR_CUDA; }
  int rc = precision == RVE_MIXED ? upload_tables<float>(h) : upload_tables<double>(h);
  if (!rc) rc = dev_alloc((void**)&h->E64, (size_t)h->N * sizeof(double));
  if (!rc && precision == RVE_MIXED) rc = dev_alloc(&h->Ein, (size_t)h->N * sizeof(float));
  if (!rc) rc = ensure_capacity(h, 1);
  if (rc) { rve_destroy(h); return rc; }
  if (precision == RVE_FP64) h->Ein = h->E64;
  *out = h;
  return RVE_OK;
}

int rve_destroy(rve_t h) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h) return RVE_OK;
  cudaStreamSynchronize(h->stream);
  flush_timing(h);
  for (auto& ev : h->ev_pool) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  h->ev_pool.clear();
  free_L(h);
  if (h->Ein && h->Ein != (void*)h->E64) cudaFree(h->Ein);
  h->Ein = nullptr;
  free_devp(h->E64);
  free_devp(h->hpart);
  for (int a = 0; a < 3; ++a) { free_dev(h->ph[a]); free_dev(h->tw[a]); }
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return RVE_OK;
}

int rve_test_stall_copies(rve_t h, int on) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h) return RVE_ERR_ARG;
  h->stall_copies = on ? 1 : 0;
  return RVE_OK;
}

int rve_sizes(rve_t h, int64_t* n_voxels, int* m, int* n_s, int* dim) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h) return RVE_ERR_ARG;
  if (n_voxels) *n_voxels = h->N;
  if (m) *m = h->m;
  if (n_s) *n_s = h->ns;
  if (dim) *dim = h->dim;
  return RVE_OK;
}

int rve_set_material(rve_t h, const void* E, int E_dtype, double nu, int ptr_flags) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !E || (E_dtype != RVE_F32 && E_dtype != RVE_F64)) return RVE_ERR_ARG;
  if (!(nu > -1.0 && nu < 0.5)) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  if (ptr_flags & RVE_PTR_DEVICE) CK(cudaStreamSynchronize(h->stream));
  std::vector<double> e64((size_t)h->N);
  if (ptr_flags & RVE_PTR_DEVICE) {
    if (E_dtype == RVE_F64) {
      CK(cudaMemcpy(e64.data(), E, (size_t)h->N * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> e32((size_t)h->N);
      CK(cudaMemcpy(e32.data(), E, (size_t)h->N * sizeof(float), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < h->N; ++i) e64[i] = e32[i];
    }
  } else {
    if (E_dtype == RVE_F64) std::memcpy(e64.data(), E, (size_t)h->N * sizeof(double));
    else for (int64_t i = 0; i < h->N; ++i) e64[i] = ((const float*)E)[i];
  }
  if (int rc = check_moduli(e64)) return rc;
  if (int rc = copy_sync(h, h->E64, e64.data(), (size_t)h->N * sizeof(double), cudaMemcpyHostToDevice)) return rc;
  if (h->precision == RVE_MIXED) {
    f32_from_f64<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(h->E64, (float*)h->Ein, h->N);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
  }
  h->nu = nu;
  h->lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));  // unit Young's modulus
  h->mu2 = 1.0 / (1.0 + nu);
  h->has_material = true;
  h->solved = false;
  return RVE_OK;
}

int rve_solve(rve_t h, const double* E_macro, int L, double rel_tol, int max_iter, rve_info* info) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !E_macro || L < 1 || L > 64 || !(rel_tol > 0.0) || max_iter < 1) return RVE_ERR_ARG;
  if (!h->has_material || h->finite) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  for (int i = 0; i < L * h->ns; ++i) if (!std::isfinite(E_macro[i])) return RVE_ERR_ARG;
  h->solved = false;
  int rc = ensure_capacity(h, L);
  if (rc) return rc;
  if (h->var[0] < 0 || h->var[1] < 0 || h->var[2] < 0 || h->var[3] < 0) {
    rc = (h->precision == RVE_MIXED) ? autotune<float>(h, L) : autotune<double>(h, L);
    if (rc) return rc;
  }
  const int st = (h->deriv != D_FE)
                     ? solve_strain_state(h, E_macro, L, rel_tol, max_iter, info)
                     : (h->precision == RVE_MIXED)
                     ? solve_impl<float>(h, E_macro, L, rel_tol, max_iter, info, h->u, h->emac_d)
                     : solve_impl<double>(h, E_macro, L, rel_tol, max_iter, info, h->u, h->emac_d);
  if (st != RVE_OK && st != RVE_ERR_NOT_CONVERGED && st != RVE_ERR_NONFINITE) return st;
  h->emac_h.assign(E_macro, E_macro + (size_t)L * h->ns);
  h->L_solved = L;
  rc = compute_mean_stress(h, L);
  if (rc) return rc;
  h->solved = true;
  return st;
}

int rve_mean_stress(rve_t h, double* S) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !S || !h->solved) return RVE_ERR_ARG;
  std::memcpy(S, h->S_h.data(), h->S_h.size() * sizeof(double));
  return RVE_OK;
}

int rve_effective_tangent(rve_t h, double* C) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !C || !h->solved || h->L_solved != h->ns) return RVE_ERR_ARG;
  const int ns = h->ns;
  std::vector<double> Minv((size_t)ns * ns);
  if (!invert(ns, h->emac_h.data(), Minv.data())) return RVE_ERR_ARG;
  // C[s][t] = sum_l S[l][s] Minv[t][l]   (C = S^T M^-T)
  for (int s = 0; s < ns; ++s)
    for (int t = 0; t < ns; ++t) {
      double v = 0.0;
      for (int l = 0; l < ns; ++l) v += h->S_h[(size_t)l * ns + s] * Minv[(size_t)t * ns + l];
      C[s * ns + t] = v;
    }
  return RVE_OK;
}

int rve_energy_tangent(rve_t h, double* Ce) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !Ce || !h->solved) return RVE_ERR_ARG;
  if (h->deriv != D_FE) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  const int L = h->L_solved;
  const int npair = L * (L + 1) / 2;
  Fp64Args fa = fp64_args(h, L, h->u, h->emac_d, h->cg);
  const int nblk = homogenise_blocks(fa);
  const size_t need = (size_t)npair * nblk;
  if ((int64_t)need > h->hpart_cap) {
    free_devp(h->hpart);
    int rc = dev_alloc((void**)&h->hpart, need * sizeof(double));
    if (rc) return rc;
    h->hpart_cap = (int)need;
  }
  int nb = 0;
  CK(timed(h, K_OTHER, [&] { return launch_energy(fa, h->hpart, &nb, h->stream); }));
  std::vector<double> hp(need);
  CK(cudaMemcpyAsync(hp.data(), h->hpart, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->timing) flush_timing(h);
  const double scale = 1.0 / ((double)h->N * h->nq);
  int p = 0;
  for (int b = 0; b < L; ++b)
    for (int a = 0; a <= b; ++a, ++p) {
      double t = 0.0;
      for (int k = 0; k < nb; ++k) t += hp[(size_t)p * nb + k];
      Ce[a * L + b] = Ce[b * L + a] = t * scale;
    }
  return RVE_OK;
}

int rve_get_strain(rve_t h, int load_case, void* eps, int ptr_flags) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !eps || !h->solved || load_case < 0 || load_case >= h->L_solved) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  Fp64Args fa = fp64_args(h, h->L_solved, h->u, h->emac_d, h->cg);
  const size_t bytes = (size_t)h->m * h->N * sizeof(double);
  double* dst = (double*)eps;
  double* tmp = nullptr;
  if (!(ptr_flags & RVE_PTR_DEVICE)) {
    int rc = dev_alloc((void**)&tmp, bytes);
    if (rc) return rc;
    dst = tmp;
  }
  cudaError_t e = (h->deriv == D_FE) ? launch_strain_field(fa, load_case, dst, h->stream)
                                      : launch_strain_total(fa, (const double*)h->x, load_case, dst, h->stream);
  if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(eps, tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (tmp) cudaFree(tmp);
  return e == cudaSuccess ? RVE_OK : map_err(e);
}

int rve_adjoint(rve_t h, const double* W, double rel_tol, int max_iter, void* grad_E, int ptr_flags) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !W || !grad_E || !h->solved || h->L_solved != h->ns || !(rel_tol > 0.0) || max_iter < 1)
    return RVE_ERR_ARG;
  if (h->deriv != D_FE) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  const int ns = h->ns, L = h->L_solved;
  std::vector<double> Minv((size_t)ns * ns), Wp((size_t)ns * L, 0.0);
  if (!invert(ns, h->emac_h.data(), Minv.data())) return RVE_ERR_ARG;
  for (int a = 0; a < ns; ++a)
    for (int l = 0; l < L; ++l) {
      double v = 0.0;
      for (int b = 0; b < ns; ++b) v += W[a * ns + b] * Minv[(size_t)b * ns + l];
      Wp[(size_t)a * L + l] = v;
    }
  // adjoint solves for the rows of W' that are not zero, macroscopic strain e_a
  std::vector<int> rows;
  std::vector<int> has(ns, 0);
  for (int a = 0; a < ns; ++a)
    for (int l = 0; l < L; ++l)
      if (Wp[(size_t)a * L + l] != 0.0) { has[a] = 1; }
  for (int a = 0; a < ns; ++a) if (has[a]) rows.push_back(a);
  std::vector<double> ea((size_t)rows.size() * ns, 0.0);
  for (size_t i = 0; i < rows.size(); ++i) ea[i * ns + rows[i]] = 1.0;
  int rc = ensure_capacity(h, (int)rows.size());
  if (rc) return rc;
  int st = RVE_OK;
  if (!rows.empty()) {
    // solve into a temporary [rows][D][N], then scatter to uadj[a]
    st = (h->precision == RVE_MIXED)
             ? solve_impl<float>(h, ea.data(), (int)rows.size(), rel_tol, max_iter, nullptr, h->uadj, h->emac_adj_d)
             : solve_impl<double>(h, ea.data(), (int)rows.size(), rel_tol, max_iter, nullptr, h->uadj, h->emac_adj_d);
    if (st != RVE_OK && st != RVE_ERR_NOT_CONVERGED) return st;
    // uadj holds the rows compactly in solve order; expand to index a (from the back)
    for (int i = (int)rows.size() - 1; i >= 0; --i) {
      if (rows[i] == i) continue;
      CK(cudaMemcpyAsync(h->uadj + (size_t)rows[i] * h->D * h->N, h->uadj + (size_t)i * h->D * h->N,
                         (size_t)h->D * h->N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  double* Wd = nullptr; int* hasd = nullptr; double* gd = nullptr;
  if ((rc = dev_alloc((void**)&Wd, Wp.size() * sizeof(double)))) return rc;
  if ((rc = dev_alloc((void**)&hasd, ns * sizeof(int)))) { cudaFree(Wd); return rc; }
  const size_t gbytes = (size_t)h->N * sizeof(double);
  if (!(ptr_flags & RVE_PTR_DEVICE)) {
    if ((rc = dev_alloc((void**)&gd, gbytes))) { cudaFree(Wd); cudaFree(hasd); return rc; }
  } else {
    gd = (double*)grad_E;
  }
  cudaError_t e = cudaMemcpyAsync(Wd, Wp.data(), Wp.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hasd, has.data(), ns * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  Fp64Args fa = fp64_args(h, L, h->u, h->emac_d, h->cg);
  if (e == cudaSuccess) e = launch_adjoint_grad(fa, h->uadj, Wd, hasd, 1.0 / ((double)h->N * h->nq), gd, h->stream);
  if (e == cudaSuccess && !(ptr_flags & RVE_PTR_DEVICE))
    e = cudaMemcpyAsync(grad_E, gd, gbytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(Wd); cudaFree(hasd);
  if (!(ptr_flags & RVE_PTR_DEVICE)) cudaFree(gd);
  if (e != cudaSuccess) return map_err(e);
  return st;
}

int rve_apply_operator(rve_t h, const void* p, void* q, int apply_material, int ptr_flags) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !p || !q) return RVE_ERR_ARG;
  if (apply_material && !h->has_material) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  if (int rc = ensure_capacity(h, 1)) return rc;
  const size_t bytes = (size_t)h->m * h->N * h->tsize;
  const cudaMemcpyKind kin = (ptr_flags & RVE_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = (ptr_flags & RVE_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(h->fbuf, p, bytes, kin, h->stream));
  std::memset(h->cg_h, 0, sizeof(CgState));
  h->cg_h[0].active = 1;
  int rc = write_state(h, 1);
  if (rc) return rc;
  h->solved = false;  // the operator shares the solve's buffers
  if (h->finite && apply_material) return RVE_ERR_ARG;
  if (h->tsize == 4) {
    PassArgs<float> a = pass_args<float>(h, 1, h->u, h->emac_d);
    a.amode = apply_material ? A_FIELD : A_BARE; a.pmode = P_G; a.emode = E_OUT;
    a.in = (const float*)h->fbuf; a.out = (float*)h->x;
    CK(apply_passes<float>(h, a));
  } else {
    PassArgs<double> a = pass_args<double>(h, 1, h->u, h->emac_d);
    a.amode = apply_material ? A_FIELD : A_BARE; a.pmode = h->finite ? P_FINITE : P_G; a.emode = E_OUT;
    a.in = (const double*)h->fbuf; a.out = (double*)h->x;
    CK(apply_passes<double>(h, a));
  }
  CK(cudaMemcpyAsync(q, h->x, bytes, kout, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

int rve_schedule(rve_t h, int* variants, float* candidate_ms) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !variants) return RVE_ERR_ARG;
  for (int w = 0; w < RVE_SCHED_PASSES; ++w) variants[w] = h->var[w];
  if (candidate_ms)
    for (int w = 0; w < RVE_SCHED_PASSES; ++w)
      for (int v = 0; v < RVE_SCHED_VARIANTS; ++v) candidate_ms[w * RVE_SCHED_VARIANTS + v] = h->tune_ms[w][v];
  return RVE_OK;
}

int rve_set_schedule(rve_t h, const int* variants) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !variants) return RVE_ERR_ARG;
  for (int w = 0; w < RVE_SCHED_PASSES; ++w)
    if (variants[w] < -1 || variants[w] >= rve_sched_candidates(h, w)) return RVE_ERR_ARG;
  for (int w = 0; w < RVE_SCHED_PASSES; ++w) h->var[w] = variants[w];
  return RVE_OK;
}

int rve_set_operator_form(rve_t h, int form) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || (form != RVE_FORM_STRESS && form != RVE_FORM_FACTORED && form != RVE_FORM_NODAL)) return RVE_ERR_ARG;
  if (form != RVE_FORM_STRESS && (h->deriv != D_FE || h->finite)) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  CK(cudaStreamSynchronize(h->stream));
  if (form == RVE_FORM_FACTORED && h->Lcap > 0 && !h->p2) {
    const size_t fld = (size_t)h->Lcap * h->m * h->N * h->tsize;
    if (int rc = dev_alloc(&h->p2, fld)) return rc;
    CK(cudaMemsetAsync(h->p2, 0, fld, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  h->op_form = form;
  return RVE_OK;
}

int rve_set_derivative(rve_t h, int derivative) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || derivative < RVE_DERIV_FE || derivative > RVE_DERIV_FOURIER2) return RVE_ERR_ARG;
  if (derivative != RVE_DERIV_FE && (h->precision != RVE_FP64 || h->op_form != RVE_FORM_STRESS)) return RVE_ERR_ARG;
  if (derivative == RVE_DERIV_FOURIER2 && h->dim != 2) return RVE_ERR_ARG;
  if (h->finite) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  CK(cudaStreamSynchronize(h->stream));
  static_assert((int)RVE_DERIV_FE == (int)D_FE && (int)RVE_DERIV_FOURIER2 == (int)D_FOURIER2, "derivative codes");
  const int nq = (derivative == RVE_DERIV_FE) ? (h->dim == 2 ? 2 : 6) : (derivative == RVE_DERIV_FOURIER2 ? 2 : 1);
  if (derivative != h->deriv) {
    // the field layout depends on n_q: drop the per-load-case buffers and any solution
    free_L(h);
    h->solved = false;
    h->L_solved = 0;
  }
  h->deriv = derivative;
  h->nq = nq;
  h->m = h->ns * nq;
  // keep one load case allocated, as after rve_create
  return ensure_capacity(h, 1);
}

int rve_derivative(rve_t h, int* derivative, int* nq) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !derivative) return RVE_ERR_ARG;
  *derivative = h->deriv;
  if (nq) *nq = h->nq;
  return RVE_OK;
}

int rve_set_kinematics(rve_t h, int kinematics) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || (kinematics != RVE_SMALL_STRAIN && kinematics != RVE_FINITE_STRAIN)) return RVE_ERR_ARG;
  const bool fin = kinematics == RVE_FINITE_STRAIN;
  if (fin && (h->precision != RVE_FP64 || h->op_form != RVE_FORM_STRESS || h->deriv != D_FE)) return RVE_ERR_ARG;
  if (fin && h->dim == 3 && h->n[2] > 128) return RVE_ERR_UNSUPPORTED_SIZE;   // 54 pencil rows in shared memory
  if (int jr = join_user(h)) return jr;
  CK(cudaStreamSynchronize(h->stream));
  if ((int)fin != h->finite) {
    free_L(h);
    h->solved = false;
    h->L_solved = 0;
  }
  h->finite = fin ? 1 : 0;
  h->m = fin ? (h->dim == 2 ? 9 : 54) : h->ns * h->nq;
  for (int w = 0; w < RVE_SCHED_PASSES; ++w)
    if (h->var[w] < 0) h->var[w] = 0;
  return ensure_capacity(h, 1);
}

int rve_solve_finite(rve_t h, const double* F_macro, int L, double rel_tol, int max_newton, int max_iter,
                     rve_info* info) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !F_macro || L < 1 || L > 64 || !(rel_tol > 0.0) || max_newton < 0 || max_iter < 1) return RVE_ERR_ARG;
  if (!h->has_material || !h->finite) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  for (int i = 0; i < L * h->dim * h->dim; ++i) if (!std::isfinite(F_macro[i])) return RVE_ERR_ARG;
  h->solved = false;
  const int Lold = h->Lcap;
  int rc = ensure_capacity(h, L);
  if (rc) return rc;
  if (h->Lcap != Lold) free_devp(h->Fs);   // buffers were regrown
  const int st = solve_finite(h, F_macro, L, rel_tol, max_newton, max_iter, info);
  if (st != RVE_OK && st != RVE_ERR_NOT_CONVERGED && st != RVE_ERR_NONFINITE) return st;
  h->L_solved = L;
  h->solved = true;
  return st;
}

int rve_mean_piola(rve_t h, double* P) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !P || !h->solved || !h->finite) return RVE_ERR_ARG;
  std::memcpy(P, h->P_h.data(), h->P_h.size() * sizeof(double));
  return RVE_OK;
}

int rve_get_deformation(rve_t h, int load_case, void* F, int ptr_flags) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !F || !h->solved || !h->finite || load_case < 0 || load_case >= h->L_solved) return RVE_ERR_ARG;
  if (int jr = join_user(h)) return jr;
  const int nq = h->dim == 2 ? 2 : 6;
  const size_t bytes = (size_t)nq * h->dim * h->dim * h->N * sizeof(double);
  const cudaMemcpyKind k = (ptr_flags & RVE_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(F, h->Fs + (size_t)load_case * h->m * h->N, bytes, k, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

int rve_operator_form(rve_t h, int* form) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !form) return RVE_ERR_ARG;
  *form = h->op_form;
  return RVE_OK;
}

int rve_timing_enable(rve_t h, int enable) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h) return RVE_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  flush_timing(h);
  h->timing = enable != 0;
  return RVE_OK;
}

int rve_timing_read(rve_t h, double* ms, int64_t* launches) {
  DeviceScope dev_scope(h ? h->device : -1);
  if (!h || !ms || !launches) return RVE_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  flush_timing(h);
  for (int k = 0; k < RVE_NKINDS; ++k) {
    ms[k] = h->t_ms[k];
    launches[k] = h->t_cnt[k];
    h->t_ms[k] = 0.0;
    h->t_cnt[k] = 0;
  }
  return RVE_OK;
}

int rve_batch_destroy(rve_batch_t b) {
  DeviceScope dev_scope(b ? b->device : -1);
  if (!b) return RVE_OK;
  if (b->root) cudaStreamSynchronize(b->root);
  for (auto& g : b->groups) {
    if (g.h) rve_destroy(g.h);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  if (b->root) cudaStreamDestroy(b->root);
  delete b;
  return RVE_OK;
}

int rve_batch_create(rve_batch_t* out, int dim, int count, const int64_t* n, int precision, double nu) {
  if (!out || !n || count < 1 || (dim != 2 && dim != 3)) return RVE_ERR_ARG;
  if (!(nu > -1.0 && nu < 0.5)) return RVE_ERR_ARG;
  *out = nullptr;
  rve_batch_s* b = new (std::nothrow) rve_batch_s();
  if (!b) return RVE_ERR_OOM;
  b->dim = dim; b->count = count; b->precision = precision; b->nu = nu;
  if (cudaGetDevice(&b->device) != cudaSuccess) { cudaGetLastError(); delete b; return RVE_ERR_CUDA; }
  b->group_of.assign(count, -1);
  b->slot_of.assign(count, -1);
  std::map<std::vector<int64_t>, int> index;
  for (int i = 0; i < count; ++i) {
    std::vector<int64_t> key(n + (size_t)i * dim, n + (size_t)(i + 1) * dim);
    auto it = index.find(key);
    int gi;
    if (it == index.end()) {
      gi = (int)b->groups.size();
      index[key] = gi;
      b->groups.emplace_back();
      for (int a = 0; a < dim; ++a) b->groups[gi].n[a] = (int)key[a];
    } else {
      gi = it->second;
    }
    b->group_of[i] = gi;
    b->slot_of[i] = (int)b->groups[gi].members.size();
    b->groups[gi].members.push_back(i);
  }
  if (cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError(); rve_batch_destroy(b); return RVE_ERR_CUDA;
  }
  for (auto& g : b->groups) {
    g.has_mat.assign(g.members.size(), 0);
    if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError(); rve_batch_destroy(b); return RVE_ERR_CUDA;
    }
    int64_t nn[3] = {g.n[0], g.n[1], g.n[2]};
    int rc = rve_create(&g.h, dim, nn, nullptr, precision, g.stream);
    if (!rc) rc = alloc_materials(g.h, (int)g.members.size());
    if (rc) { rve_batch_destroy(b); return rc; }
    set_nu(g.h, nu);
  }
  *out = b;
  return RVE_OK;
}

int rve_batch_set_material(rve_batch_t b, int index, const void* E, int E_dtype, int ptr_flags) {
  DeviceScope dev_scope(b ? b->device : -1);
  if (!b || !E || index < 0 || index >= b->count || (E_dtype != RVE_F32 && E_dtype != RVE_F64)) return RVE_ERR_ARG;
  auto& g = b->groups[b->group_of[index]];
  std::vector<double> e64;
  int rc = read_moduli(g.h->N, E, E_dtype, ptr_flags, e64);
  if (rc) return rc;
  rc = upload_material(g.h, b->slot_of[index], e64);
  if (rc) return rc;
  g.has_mat[b->slot_of[index]] = 1;
  b->solved = false;
  return RVE_OK;
}

int rve_batch_solve(rve_batch_t b, const double* E_macro, int L, double rel_tol, int max_iter, rve_info* info) {
  DeviceScope dev_scope(b ? b->device : -1);
  if (!b || !E_macro || L < 1 || L > 64 || !(rel_tol > 0.0) || max_iter < 1) return RVE_ERR_ARG;
  const int ns = b->dim == 2 ? 3 : 6;
  for (int i = 0; i < L * ns; ++i) if (!std::isfinite(E_macro[i])) return RVE_ERR_ARG;
  for (auto& g : b->groups)
    for (char c : g.has_mat) if (!c) return RVE_ERR_ARG;
  b->solved = false;
  const int G = (int)b->groups.size();
  std::vector<int> codes(G, RVE_OK);
  std::vector<std::vector<rve_info>> infos(G);
  std::vector<std::vector<double>> emacs(G);
  std::vector<rve_s*> hs(G);
  for (int gi = 0; gi < G; ++gi) {
    auto& g = b->groups[gi];
    rve_s* h = g.h;
    hs[gi] = h;
    const int Lg = (int)g.members.size() * L;
    emacs[gi].resize((size_t)Lg * ns);
    for (int s = 0; s < Lg; ++s)
      for (int c = 0; c < ns; ++c) emacs[gi][(size_t)s * ns + c] = E_macro[(size_t)(s % L) * ns + c];
    h->lcs = L;
    h->has_material = true;
    h->solved = false;
    int rc = ensure_capacity(h, Lg);
    if (rc) return rc;
    if (h->var[0] < 0 || h->var[1] < 0 || h->var[2] < 0 || h->var[3] < 0) {
      rc = (h->precision == RVE_MIXED) ? autotune<float>(h, Lg) : autotune<double>(h, Lg);
      if (rc) return rc;
    }
  }
  // every group's refinement in lockstep, the CG iterations of all groups in one graph
  const int rcl = (b->precision == RVE_MIXED) ? batch_lockstep<float>(b->root, hs, emacs, rel_tol, max_iter, infos, codes)
                                              : batch_lockstep<double>(b->root, hs, emacs, rel_tol, max_iter, infos, codes);
  if (rcl) return rcl;
  for (int gi = 0; gi < G; ++gi) {
    rve_s* h = hs[gi];
    const int st = codes[gi];
    if (st != RVE_OK && st != RVE_ERR_NOT_CONVERGED && st != RVE_ERR_NONFINITE) return st;
    h->emac_h = emacs[gi];
    h->L_solved = (int)infos[gi].size();
    int rc = compute_mean_stress(h, h->L_solved);
    if (rc) return rc;
    h->solved = true;
  }
  int worst = RVE_OK;
  for (int gi = 0; gi < G; ++gi) {
    const int c = codes[gi];
    if (c != RVE_OK && c != RVE_ERR_NOT_CONVERGED && c != RVE_ERR_NONFINITE) return c;
    if (c == RVE_ERR_NONFINITE || (c != RVE_OK && worst == RVE_OK)) worst = c;
  }
  if (info)
    for (int i = 0; i < b->count; ++i) {
      const auto& ig = infos[b->group_of[i]];
      for (int l = 0; l < L; ++l) info[(size_t)i * L + l] = ig[(size_t)b->slot_of[i] * L + l];
    }
  b->L = L;
  b->emac.assign(E_macro, E_macro + (size_t)L * ns);
  b->solved = true;
  return worst;
}

int rve_batch_mean_stress(rve_batch_t b, int index, double* S) {
  DeviceScope dev_scope(b ? b->device : -1);
  if (!b || !S || !b->solved || index < 0 || index >= b->count) return RVE_ERR_ARG;
  const int ns = b->dim == 2 ? 3 : 6;
  const auto& g = b->groups[b->group_of[index]];
  std::memcpy(S, g.h->S_h.data() + (size_t)b->slot_of[index] * b->L * ns, (size_t)b->L * ns * sizeof(double));
  return RVE_OK;
}

int rve_batch_effective_tangent(rve_batch_t b, int index, double* C) {
  DeviceScope dev_scope(b ? b->device : -1);
  const int ns = b ? (b->dim == 2 ? 3 : 6) : 0;
  if (!b || !C || !b->solved || b->L != ns) return RVE_ERR_ARG;
  std::vector<double> S((size_t)ns * ns);
  int rc = rve_batch_mean_stress(b, index, S.data());
  if (rc) return rc;
  return tangent_from_stress(ns, S.data(), b->emac.data(), C);
}

}  // extern "C"
