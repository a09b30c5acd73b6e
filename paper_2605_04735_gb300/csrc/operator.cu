// The masked stiffness operator A = M K M + (I - M) (M: free-DOF mask) and
// its Jacobi diagonal, for CG: plain apply, apply fused with p . A p, and the
// FP64 residual r = f - K u fused with ||r||^2.  The gather core is in
// stencil.cuh; this file holds the epilogues.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "stencil.cuh"

namespace topo {

namespace {

// y = A x: (K x) on free DOFs, x itself on fixed DOFs (0 by the invariant)
template <typename T, bool DOT>
struct EpiApply {
  static constexpr bool kReduce = DOT;
  T* y;
  __device__ __forceinline__ double operator()(int i, int j, int k, long long o, const T (&acc)[3],
                                               const T (&ctr)[3], const Dims& d) const {
    double part = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T out = d.fixed(r, i, j, k) ? ctr[r] : acc[r];
      y[r * d.comp + o] = out;
      if (DOT) part += (double)ctr[r] * (double)out;
    }
    return part;
  }
};

// y = f - K x on free DOFs, 0 on fixed DOFs; reduces ||y||^2
template <typename T>
struct EpiResid {
  static constexpr bool kReduce = true;
  T* y;
  const T* f;
  __device__ __forceinline__ double operator()(int i, int j, int k, long long o, const T (&acc)[3],
                                               const T (&)[3], const Dims& d) const {
    double part = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T out = d.fixed(r, i, j, k) ? T(0) : (f[r * d.comp + o] - acc[r]);
      y[r * d.comp + o] = out;
      part += (double)out * (double)out;
    }
    return part;
  }
};

// D^-1 of the masked operator: 1 / sum_{e owns n} E_e k0[3 ln + c][3 ln + c],
// and 1 on fixed DOFs (and on nodes that touch no stiffness at all).
template <typename T>
__global__ void k_diag_inv(T* __restrict__ dinv, const T* __restrict__ E, const Dims d,
                           const __grid_constant__ K0<T> k0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > d.nx || j > d.ny) return;
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const T ee = E[d.elem(i - 1 + a, j - 1 + b, k - 1 + c)];
        const int ln = lidx(1 - a, 1 - b, 1 - c);
#pragma unroll
        for (int r = 0; r < 3; ++r) acc[r] += ee * k0.v[(3 * ln + r) * 24 + 3 * ln + r];
      }
  const long long o = d.node(i, j, k);
#pragma unroll
  for (int r = 0; r < 3; ++r)
    dinv[r * d.comp + o] = (d.fixed(r, i, j, k) || !(acc[r] > T(0))) ? T(1) : T(1) / acc[r];
}

}  // namespace

template <typename T>
cudaError_t launch_apply(const T* x, T* y, const T* E, const T* f, const Dims& d, const K0<T>& k0,
                         const Red& red, int mode, const int* done, int* errflag,
                         cudaStream_t s) {
  switch (mode) {
    case APPLY_PLAIN:
      return launch_stencil<T>(x, E, d, k0, EpiApply<T, false>{y}, red, done, errflag, s);
    case APPLY_DOT:
      return launch_stencil<T>(x, E, d, k0, EpiApply<T, true>{y}, red, done, errflag, s);
    default:
      return launch_stencil<T>(x, E, d, k0, EpiResid<T>{y, f}, red, done, errflag, s);
  }
}

template <typename T>
cudaError_t launch_diag_inv(T* dinv, const T* E, const Dims& d, const K0<T>& k0, cudaStream_t s) {
  dim3 block(32, 4, 1);
  dim3 grid((d.nx + 32) / 32, (d.ny + 4) / 4, d.nz + 1);
  k_diag_inv<T><<<grid, block, 0, s>>>(dinv, E, d, k0);
  return cudaGetLastError();
}

template cudaError_t launch_apply<float>(const float*, float*, const float*, const float*,
                                         const Dims&, const K0<float>&, const Red&, int,
                                         const int*, int*, cudaStream_t);
template cudaError_t launch_apply<double>(const double*, double*, const double*, const double*,
                                          const Dims&, const K0<double>&, const Red&, int,
                                          const int*, int*, cudaStream_t);
template cudaError_t launch_diag_inv<float>(float*, const float*, const Dims&, const K0<float>&,
                                            cudaStream_t);
template cudaError_t launch_diag_inv<double>(double*, const double*, const Dims&,
                                             const K0<double>&, cudaStream_t);

}  // namespace topo
