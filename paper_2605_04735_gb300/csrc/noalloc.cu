// Element sensitivities and element-form compliance for callers that cannot
// allocate device memory (see topo_sensitivity_noalloc in include/topo.h).
//
// The reduction scratch of this entry point is a fixed, file-scope device
// array instead of memory the library allocates per mesh.  Host code only
// ever passes the array's device address, which it obtains once per device
// with cudaGetSymbolAddress (the symbol itself is a host-side stand-in that
// must never reach a kernel).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/topo.h"
#include "common.cuh"
#include "kernels.h"

namespace topo {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaElemsPerThread = 8;
constexpr int kNaElemsPerBlock = kNaThreads * kNaElemsPerThread;  // 2048
// Scratch: one FP64 partial per block plus an arrival counter.  32 KiB of
// partials bound the problem size at kNaSlots * 2048 = 8,388,608 elements.
constexpr int kNaSlots = 4096;
constexpr long long kNaMaxElems = (long long)kNaSlots * kNaElemsPerBlock;

struct NaScratch {
  double partial[kNaSlots];
  unsigned counter;
};

static __device__ __align__(256) NaScratch g_na_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
// per device: the scratch address and the id of the context it belongs to
// (a context that was destroyed, e.g. by cudaDeviceReset, and re-created has
// another id, so its address is looked up again)
NaScratch* g_na_ptr[kMaxDevices] = {};
unsigned long long g_na_ctx[kMaxDevices] = {};

__host__ __device__ constexpr int na_lidx(int dx, int dy, int dz) {
  return 4 * dz + (dy ? (dx ? 2 : 3) : (dx ? 1 : 0));
}

// dc_e = -p rho_e^(p-1) (E0 - Emin) h u_e^T k0 u_e and c = sum_e E_e h u_e^T k0 u_e,
// with u in the ABI's DOF order and rho in element order (dense, no ghosts).
// Block b handles elements [2048 b, 2048 (b+1)); its partial goes to slot b.
__global__ void __launch_bounds__(kNaThreads)
    k_sensitivity_noalloc(const double* __restrict__ u, const float* __restrict__ rho,
                          double* __restrict__ dc, double* __restrict__ c_out, int nx, int ny,
                          int nz, const __grid_constant__ K0<double> k0, double E0, double Emin,
                          double penal, double h, NaScratch* __restrict__ scr) {
  const long long n = (long long)nx * ny * nz;
  const long long base = (long long)blockIdx.x * kNaElemsPerBlock;
  double part = 0.0;
  for (int t = 0; t < kNaElemsPerThread; ++t) {
    const long long e = base + (long long)t * kNaThreads + threadIdx.x;
    if (e >= n) break;
    const int i = (int)(e % nx);
    const int j = (int)((e / nx) % ny);
    const int k = (int)(e / ((long long)nx * ny));
    double ue[24];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const long long node =
              (i + dx) + (long long)(nx + 1) * ((j + dy) + (long long)(ny + 1) * (k + dz));
          const int a = na_lidx(dx, dy, dz);
#pragma unroll
          for (int q = 0; q < 3; ++q) ue[3 * a + q] = __ldg(u + 3 * node + q);
        }
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 24; ++a) {
      double tt = 0.5 * k0.v[a * 24 + a] * ue[a];
#pragma unroll
      for (int b = a + 1; b < 24; ++b) tt = fma(k0.v[a * 24 + b], ue[b], tt);
      s = fma(2.0 * ue[a], tt, s);
    }
    const double r = (double)rho[e];
    const double rp1 = (penal == 3.0) ? r * r : pow(r, penal - 1.0);
    const double rp = (penal == 3.0) ? r * r * r : pow(r, penal);
    dc[e] = -penal * rp1 * (E0 - Emin) * h * s;
    part = fma((Emin + rp * (E0 - Emin)) * h, s, part);
  }
  // block sum -> slot, last block sums the slots in order and writes c
  __shared__ double sh[kNaThreads / 32];
  __shared__ bool last;
  const double w = warp_sum(part);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int q = 0; q < kNaThreads / 32; ++q) acc += sh[q];
    scr->partial[blockIdx.x] = acc;
    __threadfence();
    last = (atomicAdd(&scr->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaThreads) acc += __ldcg(&scr->partial[b]);
  const double ws = warp_sum(acc);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < kNaThreads / 32; ++q) tot += sh[q];
    *c_out = tot;
    scr->counter = 0u;
  }
}

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

CtxGetCurrentFn g_get_cur = nullptr;
CtxGetIdFn g_get_id = nullptr;

// Whether the driver can name contexts (entry points resolved once).
bool ctx_ids_available() {
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_get_cur = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  return g_get_cur && g_get_id;
}

// Id of the current context, 0 if none is current.
unsigned long long current_ctx_id() {
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_get_cur(&ctx) != CUDA_SUCCESS || !ctx || g_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up on
// the first call per device, and again only if the device's context has been
// destroyed and re-created since (e.g. by cudaDeviceReset: the old address
// would be stale).  cudaGetSymbolAddress may load the module, which a stream
// capture in progress does not allow: the first call must come before any.
cudaError_t scratch_address(NaScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const bool ids = ctx_ids_available();
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev] || (ids && current_ctx_id() != g_na_ctx[dev])) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);  // also makes the device's context current
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<NaScratch*>(p);
    g_na_ctx[dev] = ids ? current_ctx_id() : 0;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace topo

extern "C" topo_status topo_sensitivity_noalloc(int nx, int ny, int nz, const topo_params* prm,
                                                const double* u, const float* rho, double* dc,
                                                double* c, void* stream) {
  using namespace topo;
  if (nx < 1 || ny < 1 || nz < 1 || !u || !rho || !dc || !c) return TOPO_ERR_INVALID;
  const long long n = (long long)nx * ny * nz;
  if (n > kNaMaxElems) return TOPO_ERR_INVALID;  // more blocks than scratch slots
  topo_params p;
  if (prm)
    p = *prm;
  else
    topo_default_params(&p);
  if (!(p.nu >= 0.0 && p.nu < 0.5) || !(p.penal >= 1.0) || !(p.h > 0.0)) return TOPO_ERR_INVALID;
  NaScratch* scr = nullptr;
  if (scratch_address(&scr) != cudaSuccess) return TOPO_ERR_CUDA;
  double k[576];
  build_k0(p.nu, k);
  K0<double> k0;
  for (int t = 0; t < 576; ++t) k0.v[t] = k[t];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the arrival counter must start at zero; a previous call leaves it at zero
  // unless it was cut short, so clear it every time
  if (cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned), s) != cudaSuccess) return TOPO_ERR_CUDA;
  const int blocks = (int)((n + kNaElemsPerBlock - 1) / kNaElemsPerBlock);
  k_sensitivity_noalloc<<<blocks, kNaThreads, 0, s>>>(u, rho, dc, c, nx, ny, nz, k0, p.E0, p.Emin,
                                                      p.penal, p.h, scr);
  return cudaGetLastError() == cudaSuccess ? TOPO_OK : TOPO_ERR_CUDA;
}
