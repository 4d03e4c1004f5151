// Allocation-free variant of one operator application (2D, FP32).
//
// Some callers cannot call cudaMalloc: code running inside a host that owns
// the whole device memory pool (a custom allocator or a framework that has
// reserved everything up front), code on paths where an allocation could
// block or fail at an unpredictable moment (latency-critical or real-time
// loops), and code that must not touch the device heap at all.  For them this
// file offers rve_apply_operator_2d_static: it takes the caller's device
// buffers for E, p and q and keeps its scratch (the half spectrum, the phase
// and twiddle tables and one CG-state record) in a file-scope __device__
// array of fixed size.  It calls no cudaMalloc, cudaFree or other allocating
// routine.  The kernels are the same three 2D pass kernels that
// rve_apply_operator uses, so the results are the same.
//
// Device memory is still taken once per device, at the first use of the
// library's device code there: with lazy module loading (the CUDA default)
// the module that holds the scratch array is loaded into the device's context
// by the first call, so the first call should be made at set-up time.
#include <atomic>
#include <cmath>
#include <cstring>

#include "../../include/rve.h"
#include "rve_internal.h"

using namespace rve;

namespace {

// Largest grid side served from the static scratch, and the scratch size:
// the half spectrum (6 components x (n/2+1) x n complex floats), 2 phase and
// 2 twiddle tables of n complex floats, and one CgState.
constexpr int kStaticMaxN = 256;
constexpr size_t kSpecBytes = 6ull * (kStaticMaxN / 2 + 1) * kStaticMaxN * sizeof(float2);
constexpr size_t kTableBytes = 4ull * kStaticMaxN * sizeof(float2);
constexpr size_t kStaticScratchBytes = kSpecBytes + kTableBytes + 256;

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_rve_scratch[kStaticScratchBytes];

// Device address of g_rve_scratch, per device (nullptr = not set up yet).
std::atomic<void*> g_scratch_ptr[kMaxDevices];
DeviceOnce g_scratch_once;

// Phase tables exp(+2 pi i j / n) of both axes, twiddle tables exp(-2 pi i j / n),
// and a fresh CG-state record (active, everything else zero), written on the
// device so that a call copies nothing from the host.  sincospi is CUDA's own
// FP64 function; its results are rounded to FP32 like the host tables of the
// handle path.
__global__ void fill_static_tables(float2* tables, CgState* cg, int nx, int ny) {
  const int len[2] = {nx, ny};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * kStaticMaxN; i += gridDim.x * blockDim.x) {
    const int a = i / kStaticMaxN, j = i % kStaticMaxN;
    if (j < len[a]) {
      double sn, cs;
      sincospi(2.0 * (double)j / (double)len[a], &sn, &cs);
      tables[a * kStaticMaxN + j] = make_float2((float)cs, (float)sn);             // exp(+i ang)
      tables[(2 + a) * kStaticMaxN + j] = make_float2((float)cs, (float)-sn);      // exp(-i ang)
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    CgState st{};
    st.active = 1;
    *cg = st;
  }
}

bool pow2_in(int64_t v, int64_t lo, int64_t hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int rve_apply_operator_2d_static(const int64_t* n, const double* length, const float* E, double nu,
                                            const float* p, float* q, int apply_material, void* cuda_stream) {
  if (!n || !p || !q || (apply_material && !E)) return RVE_ERR_ARG;
  if (!(nu > -1.0 && nu < 0.5)) return RVE_ERR_ARG;
  for (int a = 0; a < 2; ++a) {
    if (!pow2_in(n[a], 16, 1 << 30)) return RVE_ERR_UNSUPPORTED_SIZE;
    if (n[a] > kStaticMaxN) return RVE_ERR_SCRATCH_LIMIT;
    if (length && !(length[a] > 0.0 && std::isfinite(length[a]))) return RVE_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) { cudaGetLastError(); return RVE_ERR_CUDA; }
  // Set-up, once per device, with that device current: the device address of
  // the static array (its name is only a host-side stand-in).  The kernel
  // attributes of the pass kernels are likewise set once per device by their
  // launchers.
  g_scratch_once.run(dev, [&] {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_rve_scratch) != cudaSuccess || !ptr) { cudaGetLastError(); ptr = nullptr; }
    g_scratch_ptr[dev].store(ptr);
  });
  unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev].load());
  if (!base) return RVE_ERR_CUDA;
  float2* spec = reinterpret_cast<float2*>(base);
  float2* tables = reinterpret_cast<float2*>(base + kSpecBytes);   // ph_x, ph_y, tw_x, tw_y
  CgState* cg = reinterpret_cast<CgState*>(base + kSpecBytes + kTableBytes);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  const int nx = (int)n[0], ny = (int)n[1];
  // Tables and CG state of this call, written on the device (the scratch keeps
  // the previous call's contents).
  fill_static_tables<<<4, 128, 0, s>>>(tables, cg, nx, ny);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return RVE_ERR_CUDA;

  PassArgs<float> a;
  std::memset(&a, 0, sizeof(a));
  a.n[0] = nx; a.n[1] = ny; a.n[2] = 1;
  a.dim = 2; a.L = 1; a.m = 6; a.ns = 3; a.nq = 2;
  a.N = (int64_t)nx * ny;
  a.kx = nx / 2 + 1;
  a.E = E;
  a.lcs = 1;
  a.in = p; a.out = q;
  a.spec = spec;
  a.ph[0] = tables; a.ph[1] = tables + kStaticMaxN;
  a.tw[0] = tables + 2 * kStaticMaxN; a.tw[1] = tables + 3 * kStaticMaxN;
  for (int i = 0; i < 2; ++i) a.ih[i] = (float)((double)n[i] / (length ? length[i] : 1.0));
  a.lam = (float)(nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
  a.mu2 = (float)(1.0 / (1.0 + nu));
  a.inv_n = (float)(1.0 / (double)a.N);
  a.cg = cg;
  a.amode = apply_material ? A_FIELD : A_BARE;
  a.pmode = P_G;
  a.emode = E_OUT;
  a.cgphase = 0;
  e = launch_pass_a_2d<float>(a, s);
  if (e == cudaSuccess) e = launch_pass_c_2d<float>(a, s);
  if (e == cudaSuccess) e = launch_pass_e_2d<float>(a, s);
  if (e != cudaSuccess) { cudaGetLastError(); return RVE_ERR_CUDA; }
  return RVE_OK;
}
