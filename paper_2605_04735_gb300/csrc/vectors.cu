// Vector kernels of preconditioned CG and of the FP64 refinement loop.
//
// Dot products: the four products of one 16-byte group are summed in the
// operand precision and only then widened, so FP32 vectors cost one FP64
// add per four entries (GB300's FP64 rate is 1/64 of FP32; an FP64 FMA per
// entry would make these streaming kernels FP64-bound).
//
// All vectors are whole padded arrays (ghost and pitch padding included,
// always 0), 16-byte aligned with a length that is a multiple of 4, so the
// kernels stream them with 16-byte vector loads.  Dots are accumulated in
// FP64 per thread, reduced per block and finalised by the last block
// (deterministic order), which also takes the CG scalar decisions.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "dword.cuh"
#include "kernels.h"

namespace topo {

namespace {

constexpr int kThreads = 256;

// blocks per design: one float4 per thread up to 8 blocks per SM in all,
// shared among the nb designs of a batched launch (so each thread of a
// large batch streams several float4 and the reductions have fewer partials)
inline int reduce_blocks(long long n4, int nb = 1) {
  long long b = (n4 + kThreads - 1) / kThreads;
  const long long cap = std::max(4LL, 152LL * 8 * 2 / std::max(nb, 1));
  b = std::min(b, std::min(cap, 152LL * 8));
  if (b < 1) b = 1;
  return (int)b;
}

inline dim3 vgrid(long long n4, const Bat& bt) { return dim3(reduce_blocks(n4, bt.nb), bt.nb); }

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_32a;  // every vector starts on a 32-byte boundary
};

template <typename T>
__device__ __forceinline__ typename Vec4<T>::type ld4(const T* p, long long q) {
  return reinterpret_cast<const typename Vec4<T>::type*>(p)[q];
}
template <typename T>
__device__ __forceinline__ void st4(T* p, long long q, const typename Vec4<T>::type& v) {
  reinterpret_cast<typename Vec4<T>::type*>(p)[q] = v;
}

// r = b, x = 0, z = D^-1 r (or z = r when the preconditioner runs later),
// p = z; reduces r.z and r.r -> FIN_INIT
template <typename T, bool JAC>
__global__ void __launch_bounds__(kThreads)
    k_pcg_init(const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
               T* __restrict__ p, const T* __restrict__ dinv, long long n4, const Red red0,
               const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  b = bshift(b, off);
  x = bshift(x, off);
  r = bshift(r, off);
  z = bshift(z, off);
  p = bshift(p, off);
  dinv = bshift(dinv, off);
  const Red red = red0.shifted(off);
  double rz = 0.0, rr = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    auto bv = ld4(b, q);
    typename Vec4<T>::type zero = {T(0), T(0), T(0), T(0)};
    st4(x, q, zero);
    st4(r, q, bv);
    if (JAC) {
      auto dv = ld4(dinv, q);
      typename Vec4<T>::type zv;
      zv.x = dv.x * bv.x;
      zv.y = dv.y * bv.y;
      zv.z = dv.z * bv.z;
      zv.w = dv.w * bv.w;
      st4(z, q, zv);
      st4(p, q, zv);
      rz += (double)(bv.x * zv.x + bv.y * zv.y + bv.z * zv.z + bv.w * zv.w);
    } else {
      st4(p, q, zero);  // the first direction is set after z = M r
    }
    rr += (double)(bv.x * bv.x + bv.y * bv.y + bv.z * bv.z + bv.w * bv.w);
  }
  double v[2] = {rz, rr};
  reduce_finalize<2>(v, red, blockIdx.x, gridDim.x);
}

// x += alpha p, r -= alpha q; Jacobi: z = D^-1 r, reduce (r.z, r.r) -> FIN_UPDATE;
// otherwise reduce r.r -> FIN_RR_ONLY, and with dinv given also z = D^-1 r scale
// (the multigrid's first Chebyshev direction on the finest level)
template <typename T, bool JAC>
__global__ void __launch_bounds__(kThreads)
    k_pcg_update(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, const T* __restrict__ p,
                 const T* __restrict__ qv, const T* __restrict__ dinv, long long n4,
                 const T scale, const Red red0, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  x = bshift(x, off);
  r = bshift(r, off);
  z = bshift(z, off);
  p = bshift(p, off);
  qv = bshift(qv, off);
  dinv = bshift(dinv, off);
  const Red red = red0.shifted(off);
  const PcgScalars* sc = red.sc;
  if (sc->done) return;
  const T a = (T)sc->alpha;
  double rz = 0.0, rr = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    auto xv = ld4(x, q);
    auto rv = ld4(r, q);
    const auto pv = ld4(p, q);
    const auto Av = ld4(qv, q);
    xv.x = fma(a, pv.x, xv.x);
    xv.y = fma(a, pv.y, xv.y);
    xv.z = fma(a, pv.z, xv.z);
    xv.w = fma(a, pv.w, xv.w);
    rv.x = fma(-a, Av.x, rv.x);
    rv.y = fma(-a, Av.y, rv.y);
    rv.z = fma(-a, Av.z, rv.z);
    rv.w = fma(-a, Av.w, rv.w);
    st4(x, q, xv);
    st4(r, q, rv);
    if (JAC) {
      const auto dv = ld4(dinv, q);
      typename Vec4<T>::type zv;
      zv.x = dv.x * rv.x;
      zv.y = dv.y * rv.y;
      zv.z = dv.z * rv.z;
      zv.w = dv.w * rv.w;
      st4(z, q, zv);
      rz += (double)(rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w);
    } else if (dinv != nullptr) {
      const auto dv = ld4(dinv, q);
      typename Vec4<T>::type zv;
      zv.x = dv.x * rv.x * scale;
      zv.y = dv.y * rv.y * scale;
      zv.z = dv.z * rv.z * scale;
      zv.w = dv.w * rv.w * scale;
      st4(z, q, zv);
    }
    rr += (double)(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
  }
  if (JAC) {
    double v[2] = {rz, rr};
    reduce_finalize<2>(v, red, blockIdx.x, gridDim.x);
  } else {
    double v[1] = {rr};
    reduce_finalize<1>(v, red, blockIdx.x, gridDim.x);
  }
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_pcg_direction(T* __restrict__ p, const T* __restrict__ z, long long n4,
                    const PcgScalars* __restrict__ sc, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  p = bshift(p, off);
  z = bshift(z, off);
  sc = bshift(sc, off);
  if (sc->done) return;
  const T b = (T)sc->beta;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    auto pv = ld4(p, q);
    const auto zv = ld4(z, q);
    pv.x = fma(b, pv.x, zv.x);
    pv.y = fma(b, pv.y, zv.y);
    pv.z = fma(b, pv.z, zv.z);
    pv.w = fma(b, pv.w, zv.w);
    st4(p, q, pv);
  }
}

// reduce a.b (and, for dot2, a.c) -> red.op
template <typename T, bool TWO>
__global__ void __launch_bounds__(kThreads)
    k_dot(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ c, long long n4,
          const Red red0, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  a = bshift(a, off);
  b = bshift(b, off);
  c = bshift(c, off);
  const Red red = red0.shifted(off);
  // a finished inner solve (converged, or a design sitting out a batched
  // step) takes no further scalar decisions
  if ((red.op == FIN_RZ_BETA || red.op == FIN_SET_RZ) && red.sc->done) return;
  double s0 = 0.0, s1 = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const auto av = ld4(a, q);
    const auto bv = ld4(b, q);
    s0 += (double)(av.x * bv.x + av.y * bv.y + av.z * bv.z + av.w * bv.w);
    if (TWO) {
      const auto cv = ld4(c, q);
      s1 += (double)(av.x * cv.x + av.y * cv.y + av.z * cv.z + av.w * cv.w);
    }
  }
  double v[2] = {s0, s1};
  reduce_finalize<2>(v, red, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads)
    k_narrow_scaled(float* __restrict__ b32, const double* __restrict__ r64, long long n4,
                    const PcgScalars* __restrict__ sc, int skip, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  b32 = bshift(b32, off);
  r64 = bshift(r64, off);
  sc = bshift(sc, off);
  if (skip && sc->sat_out) return;
  const double nrm2 = sc->aux[0];
  const double s = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const double4_32a v = ld4(r64, q);
    float4 o;
    o.x = (float)(v.x * s);
    o.y = (float)(v.y * s);
    o.z = (float)(v.z * s);
    o.w = (float)(v.w * s);
    st4(b32, q, o);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_accumulate(double* __restrict__ u, const T* __restrict__ x, long long n4,
                 const PcgScalars* __restrict__ sc, int scaled, int skip, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  u = bshift(u, off);
  x = bshift(x, off);
  sc = bshift(sc, off);
  if (skip && sc->sat_out) return;
  const double s = scaled ? sqrt(sc->aux[0]) : 1.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    double4_32a uv = ld4(u, q);
    const auto xv = ld4(x, q);
    uv.x = fma(s, (double)xv.x, uv.x);
    uv.y = fma(s, (double)xv.y, uv.y);
    uv.z = fma(s, (double)xv.z, uv.z);
    uv.w = fma(s, (double)xv.w, uv.w);
    st4(u, q, uv);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_copy_cast(T* __restrict__ dst, const double* __restrict__ src, long long n4, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  dst = bshift(dst, off);
  src = bshift(src, off);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const double4_32a v = ld4(src, q);
    typename Vec4<T>::type o;
    o.x = (T)v.x;
    o.y = (T)v.y;
    o.z = (T)v.z;
    o.w = (T)v.w;
    st4(dst, q, o);
  }
}

__global__ void __launch_bounds__(kThreads)
    k_split_dw(const double* __restrict__ u, float* __restrict__ hi, float* __restrict__ lo,
               long long n4, const int* __restrict__ skip, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  skip = bshift(skip, off);
  if (skip && *skip) return;
  u = bshift(u, off);
  hi = bshift(hi, off);
  lo = bshift(lo, off);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const double4_32a v = ld4(u, q);
    const Dw a = dw_from(v.x), b = dw_from(v.y), c = dw_from(v.z), e = dw_from(v.w);
    st4(hi, q, make_float4(a.hi, b.hi, c.hi, e.hi));
    st4(lo, q, make_float4(a.lo, b.lo, c.lo, e.lo));
  }
}

// thread b: the design of slot b; max_iter < 0 takes each design's max_iter_next
__global__ void k_set_max_iter(PcgScalars* sc, int max_iter, int nb, const DSel S) {
  const int b = threadIdx.x + blockIdx.x * blockDim.x;
  if (b >= nb) return;
  PcgScalars* t = bshift(sc, S.off(b));
  t->max_iter = (max_iter >= 0) ? max_iter : t->max_iter_next;
  t->done = 0;
  t->status = 0;
}

}  // namespace

cudaError_t launch_set_max_iter(PcgScalars* sc, int max_iter, cudaStream_t s, const Bat& bt) {
  return launch_pdl(k_set_max_iter, dim3((bt.nb + 127) / 128), dim3(128), 0, s, sc, max_iter, bt.nb,
                    bt.sel());
}

template <typename T>
cudaError_t launch_pcg_init(const T* b, T* x, T* r, T* z, T* p, const T* dinv, long long n,
                            const Red& red, bool jacobi, cudaStream_t s, const Bat& bt) {
  const long long n4 = n / 4;
  const dim3 g = vgrid(n4, bt);
  if (jacobi)
    return launch_pdl(k_pcg_init<T, true>, g, dim3(kThreads), 0, s, b, x, r, z, p, dinv, n4, red,
                      bt.sel());
  return launch_pdl(k_pcg_init<T, false>, g, dim3(kThreads), 0, s, b, x, r, z, p, dinv, n4, red,
                    bt.sel());
}

template <typename T>
cudaError_t launch_pcg_update(T* x, T* r, T* z, const T* p, const T* q, const T* dinv, long long n,
                              const Red& red, bool jacobi, cudaStream_t s, const Bat& bt,
                              T scale) {
  const long long n4 = n / 4;
  const dim3 g = vgrid(n4, bt);
  if (jacobi)
    return launch_pdl(k_pcg_update<T, true>, g, dim3(kThreads), 0, s, x, r, z, p, q, dinv, n4,
                      scale, red, bt.sel());
  return launch_pdl(k_pcg_update<T, false>, g, dim3(kThreads), 0, s, x, r, z, p, q, dinv, n4,
                    scale, red, bt.sel());
}

template <typename T>
cudaError_t launch_pcg_direction(T* p, const T* z, long long n, const PcgScalars* sc,
                                 cudaStream_t s, const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_pcg_direction<T>, vgrid(n4, bt), dim3(kThreads), 0, s, p, z, n4, sc, bt.sel());
}

template <typename T>
cudaError_t launch_dot(const T* a, const T* b, long long n, const Red& red, cudaStream_t s,
                       const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_dot<T, false>, vgrid(n4, bt), dim3(kThreads), 0, s, a, b, nullptr, n4, red,
                    bt.sel());
}

template <typename T>
cudaError_t launch_dot2(const T* a, const T* b, const T* c, long long n, const Red& red,
                        cudaStream_t s, const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_dot<T, true>, vgrid(n4, bt), dim3(kThreads), 0, s, a, b, c, n4, red, bt.sel());
}

cudaError_t launch_narrow_scaled(float* b32, const double* r64, long long n, const PcgScalars* sc,
                                 cudaStream_t s, const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_narrow_scaled, vgrid(n4, bt), dim3(kThreads), 0, s, b32, r64, n4, sc,
                    bt.nb > 1 ? 1 : 0, bt.sel());
}

template <typename T>
cudaError_t launch_accumulate(double* u64, const T* x, long long n, const PcgScalars* sc,
                              bool scaled, cudaStream_t s, const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_accumulate<T>, vgrid(n4, bt), dim3(kThreads), 0, s, u64, x, n4, sc,
                    scaled ? 1 : 0, bt.nb > 1 ? 1 : 0, bt.sel());
}

cudaError_t launch_split_dw(const double* u, float* hi, float* lo, long long n, const int* skip,
                            cudaStream_t s, const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_split_dw, vgrid(n4, bt), dim3(kThreads), 0, s, u, hi, lo, n4, skip,
                    bt.sel());
}

template <typename T>
cudaError_t launch_copy_cast(T* dst, const double* src, long long n, cudaStream_t s,
                             const Bat& bt) {
  const long long n4 = n / 4;
  return launch_pdl(k_copy_cast<T>, vgrid(n4, bt), dim3(kThreads), 0, s, dst, src, n4, bt.sel());
}

#define TOPO_INST(T)                                                                           \
  template cudaError_t launch_pcg_init<T>(const T*, T*, T*, T*, T*, const T*, long long,       \
                                          const Red&, bool, cudaStream_t, const Bat&);         \
  template cudaError_t launch_pcg_update<T>(T*, T*, T*, const T*, const T*, const T*,          \
                                            long long, const Red&, bool, cudaStream_t,         \
                                            const Bat&, T);                                    \
  template cudaError_t launch_pcg_direction<T>(T*, const T*, long long, const PcgScalars*,     \
                                               cudaStream_t, const Bat&);                      \
  template cudaError_t launch_dot<T>(const T*, const T*, long long, const Red&, cudaStream_t,  \
                                     const Bat&);                                              \
  template cudaError_t launch_dot2<T>(const T*, const T*, const T*, long long, const Red&,     \
                                      cudaStream_t, const Bat&);                               \
  template cudaError_t launch_accumulate<T>(double*, const T*, long long, const PcgScalars*,   \
                                            bool, cudaStream_t, const Bat&);                   \
  template cudaError_t launch_copy_cast<T>(T*, const double*, long long, cudaStream_t,         \
                                           const Bat&);
TOPO_INST(float)
TOPO_INST(double)

}  // namespace topo
