// The masked stiffness operator A = M K M + (I - M) (M: free-DOF mask) and
// its Jacobi diagonal, for CG: plain apply, apply fused with p . A p, and the
// FP64 residual r = f - K u fused with ||r||^2.  The gather core is in
// stencil.cuh; this file holds the epilogues.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "modal.cuh"
#include "modal2.cuh"
#include "modal_dw.cuh"
#include "modal_tc.cuh"
#include "stencil.cuh"

namespace topo {

namespace {

// y = A x: (K x) on free DOFs, x itself on fixed DOFs (0 by the invariant)
template <typename T, bool DOT>
struct EpiApply {
  static constexpr bool kReduce = DOT;
  static constexpr int kAux = 0;
  static constexpr int kDinvAux = -1;
  T* y;
  __device__ EpiApply shifted(long long off) const { return EpiApply{bshift(y, off)}; }
  __host__ __device__ const T* aux(int) const { return nullptr; }
  template <int N, class DD>
  __device__ __forceinline__ T finish(const int (&i)[N], int j, int k, const long long (&o)[N],
                                      const bool (&own)[N], const T (&acc)[N][3],
                                      const T (&ctr)[N][3], const T (&)[1][N][3],
                                      const DD& d) const {
    T part = T(0);
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n])
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const T out = d.fixed(r, i[n], j, k) ? ctr[n][r] : acc[n][r];
          y[r * d.comp + o[n]] = out;
          if (DOT) part = fma(ctr[n][r], out, part);
        }
    return part;
  }
};

// y = f - K x on free DOFs, 0 on fixed DOFs; reduces ||y||^2
template <typename T>
struct EpiResid {
  static constexpr bool kReduce = true;
  static constexpr int kAux = 1;  // f
  static constexpr int kDinvAux = -1;
  T* y;
  const T* f;
  __device__ EpiResid shifted(long long off) const {
    return EpiResid{bshift(y, off), bshift(f, off)};
  }
  __host__ __device__ const T* aux(int) const { return f; }
  template <int N, class DD>
  __device__ __forceinline__ T finish(const int (&i)[N], int j, int k, const long long (&o)[N],
                                      const bool (&own)[N], const T (&acc)[N][3],
                                      const T (&)[N][3], const T (&av)[1][N][3],
                                      const DD& d) const {
    T part = T(0);
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n])
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const T out = d.fixed(r, i[n], j, k) ? T(0) : (av[0][n][r] - acc[n][r]);
          y[r * d.comp + o[n]] = out;
          part = fma(out, out, part);
        }
    return part;
  }
};

// 1 / x of a diagonal entry: FP32 through the same reciprocal as the kernels
// that form D^-1 on the fly from the element moduli
__device__ __forceinline__ float inv_diag(float x) { return jacobi_rcp(x); }
__device__ __forceinline__ double inv_diag(double x) { return 1.0 / x; }

// D^-1 of the masked operator: 1 / sum_{e owns n} E_e k0[3 ln + c][3 ln + c],
// and 1 on fixed DOFs (and on nodes that touch no stiffness at all).
template <typename T>
__global__ void k_diag_inv(T* __restrict__ dinv, const T* __restrict__ E, const Dims d,
                           const __grid_constant__ K0<T> k0, const DSel S) {
  pdl_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int slot = blockIdx.z / (d.nz + 1);
  const int k = blockIdx.z - slot * (d.nz + 1);
  dinv = bshift(dinv, S.off(slot));
  E = bshift(E, S.off(slot));
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
    dinv[r * d.comp + o] = (d.fixed(r, i, j, k) || !(acc[r] > T(0))) ? T(1) : inv_diag(acc[r]);
}

}  // namespace

template <typename T>
cudaError_t launch_apply(const T* x, T* y, const T* E, const T* f, const Dims& d, const K0<T>& k0,
                         const ModalCoef<T>* mc, const Red& red, int mode, const int* done,
                         int* errflag, cudaStream_t s, const Bat& bt, T* energy) {
  if (mc) {
    switch (mode) {
      case APPLY_PLAIN:
        return launch_modal_any<3, T>(x, E, d, *mc, k0, EpiApply<T, false>{y}, red, done,
                                      errflag, s, bt);
      case APPLY_DOT:
        return launch_modal_any<3, T>(x, E, d, *mc, k0, EpiApply<T, true>{y}, red, done, errflag,
                                      s, bt);
      default:
        return launch_modal_any<3, T>(x, E, d, *mc, k0, EpiResid<T>{y, f}, red, done, errflag,
                                      s, bt, energy);
    }
  }
  if (energy) return cudaErrorInvalidValue;    // element energies: the modal kernels only
  if (bt.nb != 1) return cudaErrorInvalidValue;  // the gather kernels run one design
  switch (mode) {
    case APPLY_PLAIN:
      return launch_stencil<T>(x, E, d, k0, EpiApply<T, false>{y}, red, done, errflag, s);
    case APPLY_DOT:
      return launch_stencil<T>(x, E, d, k0, EpiApply<T, true>{y}, red, done, errflag, s);
    default:
      return launch_stencil<T>(x, E, d, k0, EpiResid<T>{y, f}, red, done, errflag, s);
  }
}

cudaError_t launch_apply_dw(const float* xh, const float* xl, double* y, const double* E,
                            const double* f, const Dims& d, const ModalCoef<double>& mc,
                            const Red& red, int mode, const int* done, cudaStream_t s,
                            const Bat& bt) {
  switch (mode) {
    case APPLY_PLAIN:
      return launch_modal_dw(xh, xl, E, d, mc, EpiApply<double, false>{y}, red, done, s, bt);
    case APPLY_DOT:
      return launch_modal_dw(xh, xl, E, d, mc, EpiApply<double, true>{y}, red, done, s, bt);
    default:
      return launch_modal_dw(xh, xl, E, d, mc, EpiResid<double>{y, f}, red, done, s, bt);
  }
}

template <typename T>
cudaError_t launch_diag_inv(T* dinv, const T* E, const Dims& d, const K0<T>& k0, cudaStream_t s,
                            const Bat& bt) {
  dim3 block(32, 4, 1);
  dim3 grid((d.nx + 32) / 32, (d.ny + 4) / 4, (d.nz + 1) * bt.nb);
  return launch_pdl(k_diag_inv<T>, grid, block, 0, s, dinv, E, d, k0, bt.sel());
}

template cudaError_t launch_apply<float>(const float*, float*, const float*, const float*,
                                         const Dims&, const K0<float>&, const ModalCoef<float>*,
                                         const Red&, int, const int*, int*, cudaStream_t,
                                         const Bat&, float*);
template cudaError_t launch_apply<double>(const double*, double*, const double*, const double*,
                                          const Dims&, const K0<double>&,
                                          const ModalCoef<double>*, const Red&, int, const int*,
                                          int*, cudaStream_t, const Bat&, double*);

bool build_modal_coef(const double* k0, ModalCoef<double>* out) {
  // corner a of the local numbering -> binary index b = ax + 2 ay + 4 az
  static const int bin[8] = {0, 1, 3, 2, 4, 5, 7, 6};
  auto H = [](int b, int m) { return (__builtin_popcount(b & m) & 1) ? -1.0 : 1.0; };
  double Kt[24][24];  // [(p,m)][(q,n)] = (1/64) sum_ab H[b(a)][m] k0[3a+p][3b+q] H[b(b)][n]
  for (int p = 0; p < 3; ++p)
    for (int m = 0; m < 8; ++m)
      for (int q = 0; q < 3; ++q)
        for (int n = 0; n < 8; ++n) {
          double acc = 0.0;
          for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b)
              acc += H(bin[a], m) * k0[(3 * a + p) * 24 + 3 * b + q] * H(bin[b], n);
          Kt[p * 8 + m][q * 8 + n] = acc / 64.0;
        }
  double scale = 0.0;
  for (int r = 0; r < 24; ++r)
    for (int c = 0; c < 24; ++c) scale = std::fmax(scale, std::fabs(Kt[r][c]));
  *out = ModalCoef<double>{};
  double used[24][24] = {};
  for (int p = 0; p < 3; ++p)
    for (int m = 1; m < 8; ++m) {
      out->D[p][m] = Kt[p * 8 + m][p * 8 + m];
      used[p * 8 + m][p * 8 + m] = 1;
      for (int q = 0; q < 3; ++q) {
        if (q == p || ((m >> p) & 1) == ((m >> q) & 1)) continue;
        const int n = m ^ (1 << p) ^ (1 << q);
        out->C[p][q][m] = Kt[p * 8 + m][q * 8 + n];
        used[p * 8 + m][q * 8 + n] = 1;
      }
    }
  for (int r = 0; r < 24; ++r)
    for (int c = 0; c < 24; ++c)
      if (!used[r][c] && std::fabs(Kt[r][c]) > 1e-12 * scale) return false;
  // the Jacobi diagonal is kdiag times the sum of the moduli around a node
  out->kdiag = k0[0];
  for (int a = 1; a < 24; ++a)
    if (std::fabs(k0[a * 24 + a] - out->kdiag) > 1e-12 * std::fabs(out->kdiag)) return false;
  return true;
}
template cudaError_t launch_diag_inv<float>(float*, const float*, const Dims&, const K0<float>&,
                                            cudaStream_t, const Bat&);
template cudaError_t launch_diag_inv<double>(double*, const double*, const Dims&,
                                             const K0<double>&, cudaStream_t, const Bat&);

}  // namespace topo
