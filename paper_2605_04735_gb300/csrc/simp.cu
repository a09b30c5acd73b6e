// The rest of a SIMP iteration on the device: the sensitivity filter of
// Sec. 2.1.3, Eq. (4), and the Optimality Criteria density update (named in
// Sec. 2.1.2 and Sec. 4.1; the paper prints no move limit or damping, so both
// are parameters).
//
// Filter (structured grid, uniform element volume):
//   dc~_e = sum_{i in N_e} rho_i H_ei dc_i / (max(rho_e, guard) sum_{i in N_e} H_ei),
//   H_ei = max(0, R - |x_e - x_i|) over in-domain elements; a gather over the
//   integer offsets of the R-ball, FP64.
// OC: rho_new = clip(rho (b / lambda)^eta, max(rho_min, rho - move),
//   min(1, rho + move)), b = max(-dc~, 0), with lambda chosen so that the mean
//   density equals the volume fraction.  The volume is monotone in lambda, so
//   lambda is bracketed on the device: each pass evaluates kOcCand candidate
//   values spread over the current log-bracket in one streaming pass over the
//   elements, and the last block keeps the sub-bracket that contains the
//   target; kOcPasses passes shrink the log-bracket by (kOcCand+1)^kOcPasses.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace topo {

namespace {

constexpr int kSimpThreads = 256;
constexpr int kOcCand = 32;

struct FilterTaps {
  int n;
  int di[125], dj[125], dk[125];
  double w[125];
};

__global__ void __launch_bounds__(kSimpThreads)
    k_filter(const double* __restrict__ dc, const float* __restrict__ rho_g, double* __restrict__ dcf,
             const Dims d, const __grid_constant__ FilterTaps taps, double guard) {
  const long long n = (long long)d.nx * d.ny * d.nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(e, d.nx, d.ny, i, j, k);
    double num = 0.0, den = 0.0;
    for (int t = 0; t < taps.n; ++t) {
      const int ii = i + taps.di[t], jj = j + taps.dj[t], kk = k + taps.dk[t];
      if (ii < 0 || ii >= d.nx || jj < 0 || jj >= d.ny || kk < 0 || kk >= d.nz) continue;
      const long long q = ii + (long long)d.nx * (jj + (long long)d.ny * kk);
      num = fma(taps.w[t] * (double)rho_g[d.elem(ii, jj, kk)], dc[q], num);
      den += taps.w[t];
    }
    dcf[e] = num / (fmax((double)rho_g[d.elem(i, j, k)], guard) * den);
  }
}

struct OcState {
  double log_lo, log_hi;  // bracket of log(lambda)
  double target;          // sum of densities to reach
  double sum, change;     // results of the final pass
  unsigned counter;
};

struct OcParams {
  double move, eta, rho_min;
};

__device__ __forceinline__ float oc_new(float r, float b, float s, float eta_is_half, double eta,
                                        double lam, float lo, float hi) {
  const float v = eta_is_half ? r * sqrtf(b) * s : (float)((double)r * pow((double)b / lam, eta));
  return fminf(fmaxf(v, lo), hi);
}

// one bracketing pass: kOcCand candidate lambdas, per-block partial volumes
__global__ void __launch_bounds__(kSimpThreads)
    k_oc_pass(const float* __restrict__ rho, const double* __restrict__ dcf, long long n,
              OcState* __restrict__ st, double* __restrict__ part, const OcParams p) {
  __shared__ double lam[kOcCand];
  __shared__ float sc[kOcCand];
  __shared__ double red[kSimpThreads / 32][kOcCand];
  __shared__ bool last;
  if (threadIdx.x < kOcCand) {
    const double a = st->log_lo, b = st->log_hi;
    const double l = a + (b - a) * (threadIdx.x + 1) / (double)(kOcCand + 1);
    lam[threadIdx.x] = exp(l);
    sc[threadIdx.x] = (float)exp(-0.5 * l);
  }
  __syncthreads();
  const bool half = (p.eta == 0.5);
  float acc[kOcCand];
#pragma unroll
  for (int c = 0; c < kOcCand; ++c) acc[c] = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float r = rho[e];
    const float b = (float)fmax(-dcf[e], 0.0);
    const float lo = fmaxf((float)p.rho_min, r - (float)p.move);
    const float hi = fminf(1.0f, r + (float)p.move);
#pragma unroll
    for (int c = 0; c < kOcCand; ++c) acc[c] += oc_new(r, b, sc[c], half, p.eta, lam[c], lo, hi);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kOcCand; ++c) {
    const double w = warp_sum((double)acc[c]);
    if (lane == 0) red[warp][c] = w;
  }
  __syncthreads();
  if (threadIdx.x < kOcCand) {
    double s = 0.0;
    for (int q = 0; q < kSimpThreads / 32; ++q) s += red[q][threadIdx.x];
    part[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double vol[kOcCand];
  if (threadIdx.x < kOcCand) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b)
      s += __ldcg(&part[(long long)threadIdx.x * gridDim.x + b]);
    vol[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the volume decreases with lambda: keep the sub-bracket holding the target
    const double a = st->log_lo, b = st->log_hi;
    int k = -1;
    for (int c = 0; c < kOcCand; ++c)
      if (vol[c] > st->target) k = c;
    const double step = (b - a) / (double)(kOcCand + 1);
    st->log_lo = a + step * (k + 1);
    st->log_hi = a + step * (k + 2);
    st->counter = 0u;
  }
}

// final update with lambda at the bracket's centre: rho_new (dense),
// reductions of sum(rho_new) and max |rho_new - rho|
__global__ void __launch_bounds__(kSimpThreads)
    k_oc_apply(const float* __restrict__ rho, const double* __restrict__ dcf, float* __restrict__ out,
               long long n, OcState* __restrict__ st, double* __restrict__ part, const OcParams p) {
  const double l = 0.5 * (st->log_lo + st->log_hi);
  const double lam = exp(l);
  const float s = (float)exp(-0.5 * l);
  const bool half = (p.eta == 0.5);
  double sum = 0.0;
  float chg = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float r = rho[e];
    const float b = (float)fmax(-dcf[e], 0.0);
    const float lo = fmaxf((float)p.rho_min, r - (float)p.move);
    const float hi = fminf(1.0f, r + (float)p.move);
    const float v = oc_new(r, b, s, half, p.eta, lam, lo, hi);
    out[e] = v;
    sum += v;
    chg = fmaxf(chg, fabsf(v - r));
  }
  __shared__ double rs[kSimpThreads / 32];
  __shared__ float rc[kSimpThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double w = warp_sum(sum);
  float c = chg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, o));
  if (lane == 0) {
    rs[warp] = w;
    rc[warp] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    float m = 0.f;
    for (int q = 0; q < kSimpThreads / 32; ++q) {
      a += rs[q];
      m = fmaxf(m, rc[q]);
    }
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = (double)m;
    __threadfence();
    last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double a = 0.0, m = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) {
    a += __ldcg(&part[b]);
    m = fmax(m, __ldcg(&part[gridDim.x + b]));
  }
  st->sum = a;
  st->change = m;
  st->counter = 0u;
}

__global__ void k_oc_init(OcState* st, double target) {
  st->log_lo = log(1e-40);
  st->log_hi = log(1e40);
  st->target = target;
  st->sum = 0.0;
  st->change = 0.0;
  st->counter = 0u;
}

int simp_blocks(long long n) {
  long long b = (n + kSimpThreads - 1) / kSimpThreads;
  if (b > 152 * 4) b = 152 * 4;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

size_t oc_state_bytes() { return sizeof(OcState); }
size_t oc_partials_count() { return (size_t)kOcCand * 152 * 4; }

cudaError_t launch_filter(const double* dc, const float* rho_g, double* dcf, const Dims& d,
                          double radius, double guard, cudaStream_t s) {
  FilterTaps taps{};
  const int reach = (int)std::ceil(radius);
  for (int k = -reach; k <= reach; ++k)
    for (int j = -reach; j <= reach; ++j)
      for (int i = -reach; i <= reach; ++i) {
        const double w = radius - std::sqrt((double)(i * i + j * j + k * k));
        if (w <= 0.0) continue;
        if (taps.n >= 125) return cudaErrorInvalidValue;
        taps.di[taps.n] = i;
        taps.dj[taps.n] = j;
        taps.dk[taps.n] = k;
        taps.w[taps.n] = w;
        ++taps.n;
      }
  const long long n = (long long)d.nx * d.ny * d.nz;
  k_filter<<<simp_blocks(n), kSimpThreads, 0, s>>>(dc, rho_g, dcf, d, taps, guard);
  return cudaGetLastError();
}

cudaError_t launch_oc(const float* rho, const double* dcf, float* out, long long n, double volfrac,
                      double move, double eta, double rho_min, int passes, void* state,
                      double* partials, cudaStream_t s) {
  OcState* st = static_cast<OcState*>(state);
  OcParams p{move, eta, rho_min};
  k_oc_init<<<1, 1, 0, s>>>(st, volfrac * (double)n);
  const int g = simp_blocks(n);
  for (int q = 0; q < passes; ++q) k_oc_pass<<<g, kSimpThreads, 0, s>>>(rho, dcf, n, st, partials, p);
  k_oc_apply<<<g, kSimpThreads, 0, s>>>(rho, dcf, out, n, st, partials, p);
  return cudaGetLastError();
}

void oc_results(const void* state_host, double* sum, double* change, double* lambda) {
  const OcState* st = static_cast<const OcState*>(state_host);
  if (sum) *sum = st->sum;
  if (change) *change = st->change;
  if (lambda) *lambda = std::exp(0.5 * (st->log_lo + st->log_hi));
}

}  // namespace topo
