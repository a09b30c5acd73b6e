// Matrix-free application of the SIMP stiffness operator (Sec. 2.1.1,
// Eq. (2): K(rho) = sum_e E_e k0 assembled over the structured grid, E_e from
// Eq. (1)), as a node-centric gather with no atomics.
//
// Each thread owns a column of nodes (i, j, k0..k1) and marches up in z,
// holding the 3x3x3 node neighbourhood (3 displacement components each) and
// the 2x2x2 surrounding elements' moduli in registers; per z step it loads
// only the next node plane (9 nodes) and element plane (4 elements).  For
// node n the result is
//     y_n = sum_{e owns n} E_e * (k0[row block of n in e] . u_e),
// 8 elements x 24 columns x 3 rows = 576 FMAs per node with k0 read as
// constant-bank operands (compile-time indices).  Fixed DOFs return y = x.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace topo {

namespace {

// local node number of the corner at offsets (dx, dy, dz) in {0,1}^3
__host__ __device__ constexpr int lidx(int dx, int dy, int dz) {
  return 4 * dz + (dy ? (dx ? 2 : 3) : (dx ? 1 : 0));
}

constexpr int kBX = 32;
constexpr int kBY = 8;

template <typename T, int MODE>
__global__ void __launch_bounds__(kBX* kBY)
    k_apply(const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ E,
            const T* __restrict__ f, const Dims d, const __grid_constant__ K0<T> k0, const Red red,
            const int zchunk, const int* __restrict__ done) {
  if (done != nullptr && *done) return;  // uniform over the grid
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool act = (i <= d.nx) && (j <= d.ny);
  double part = 0.0;
  if (act) {
    const long long ps = d.plane_stride();
    const long long eps = d.eplane();
    const long long cs = d.comp;
    // window w[z][y][x][c]: nodes (i-1+x, j-1+y, k-1+z)
    T w[3][3][3][3];
    T e[2][2][2];  // e[z][y][x]: element (i-1+x, j-1+y, k-1+z)
    const long long nb = d.node(i - 1, j - 1, kb - 1);
    const long long eb = d.elem(i - 1, j - 1, kb - 1);
#pragma unroll
    for (int zz = 0; zz < 2; ++zz)
#pragma unroll
      for (int yy = 0; yy < 3; ++yy)
#pragma unroll
        for (int xx = 0; xx < 3; ++xx) {
          const long long o = nb + zz * ps + yy * d.px + xx;
#pragma unroll
          for (int c = 0; c < 3; ++c) w[zz][yy][xx][c] = __ldg(x + c * cs + o);
        }
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int xx = 0; xx < 2; ++xx) e[0][yy][xx] = __ldg(E + eb + yy * d.ex + xx);

    for (int k = kb; k < ke; ++k) {
      const long long np = nb + (long long)(k - kb + 2) * ps;  // plane k+1
      const long long ep = eb + (long long)(k - kb + 1) * eps; // element plane k
#pragma unroll
      for (int yy = 0; yy < 3; ++yy)
#pragma unroll
        for (int xx = 0; xx < 3; ++xx) {
          const long long o = np + yy * d.px + xx;
#pragma unroll
          for (int c = 0; c < 3; ++c) w[2][yy][xx][c] = __ldg(x + c * cs + o);
        }
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
#pragma unroll
        for (int xx = 0; xx < 2; ++xx) e[1][yy][xx] = __ldg(E + ep + yy * d.ex + xx);

      T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            const int ln = lidx(1 - a, 1 - b, 1 - c);
            T s[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
              for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                  const int lm = lidx(dx, dy, dz);
#pragma unroll
                  for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                      s[r] = fma(k0.v[(3 * ln + r) * 24 + 3 * lm + q],
                                 w[c + dz][b + dy][a + dx][q], s[r]);
                }
            const T ee = e[c][b][a];
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[r] = fma(ee, s[r], acc[r]);
          }

      const long long o = d.node(i, j, k);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const bool fx = d.fixed(r, i, j, k);
        T out;
        if (MODE == APPLY_RESID) {
          out = fx ? T(0) : (f[r * cs + o] - acc[r]);
          part += (double)out * (double)out;
        } else {
          out = fx ? w[1][1][1][r] : acc[r];
          if (MODE == APPLY_DOT) part += (double)w[1][1][1][r] * (double)out;
        }
        y[r * cs + o] = out;
      }
      // slide the window up one plane
#pragma unroll
      for (int yy = 0; yy < 3; ++yy)
#pragma unroll
        for (int xx = 0; xx < 3; ++xx)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            w[0][yy][xx][c] = w[1][yy][xx][c];
            w[1][yy][xx][c] = w[2][yy][xx][c];
          }
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
#pragma unroll
        for (int xx = 0; xx < 2; ++xx) e[0][yy][xx] = e[1][yy][xx];
    }
  }
  if (MODE != APPLY_PLAIN) {
    double v[1] = {part};
    reduce_finalize<1>(v, red);
  }
}

// FP64 variant: one thread per node, no register window (an FP64 window of
// 81 values spills); the FP64 pipe, not the loads, bounds this kernel.
template <typename T, int MODE>
__global__ void __launch_bounds__(kBX* kBY)
    k_apply_direct(const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ E,
                   const T* __restrict__ f, const Dims d, const __grid_constant__ K0<T> k0,
                   const Red red, const int zchunk, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int i = blockIdx.x * kBX + threadIdx.x;
  const int j = blockIdx.y * kBY + threadIdx.y;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool act = (i <= d.nx) && (j <= d.ny);
  double part = 0.0;
  for (int k = kb; act && k < ke; ++k) {
    const long long cs = d.comp;
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int ln = lidx(1 - a, 1 - b, 1 - c);
          const long long ob = d.node(i - 1 + a, j - 1 + b, k - 1 + c);
          T s[3] = {T(0), T(0), T(0)};
#pragma unroll
          for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
              for (int dx = 0; dx < 2; ++dx) {
                const int lm = lidx(dx, dy, dz);
                const long long o = ob + dz * d.plane_stride() + dy * d.px + dx;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                  const T u = __ldg(x + q * cs + o);
#pragma unroll
                  for (int r = 0; r < 3; ++r)
                    s[r] = fma(k0.v[(3 * ln + r) * 24 + 3 * lm + q], u, s[r]);
                }
              }
          const T ee = __ldg(E + d.elem(i - 1 + a, j - 1 + b, k - 1 + c));
#pragma unroll
          for (int r = 0; r < 3; ++r) acc[r] = fma(ee, s[r], acc[r]);
        }
    const long long o = d.node(i, j, k);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const bool fx = d.fixed(r, i, j, k);
      const T xin = x[r * cs + o];
      T out;
      if (MODE == APPLY_RESID) {
        out = fx ? T(0) : (f[r * cs + o] - acc[r]);
        part += (double)out * (double)out;
      } else {
        out = fx ? xin : acc[r];
        if (MODE == APPLY_DOT) part += (double)xin * (double)out;
      }
      y[r * cs + o] = out;
    }
  }
  if (MODE != APPLY_PLAIN) {
    double v[1] = {part};
    reduce_finalize<1>(v, red);
  }
}

// D^-1 of the masked operator: 1 / sum_{e owns n} E_e k0[3 ln + c][3 ln + c],
// and 1 on fixed DOFs.
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
  for (int r = 0; r < 3; ++r) dinv[r * d.comp + o] = d.fixed(r, i, j, k) ? T(1) : T(1) / acc[r];
}

int pick_zchunk(const Dims& d) {
  // enough blocks for ~4 waves of 152 SMs at 2 resident blocks each, while
  // keeping the 2-plane halo reload below ~15% and within the partial buffer
  const long long xy = (long long)((d.nx + kBX) / kBX) * ((d.ny + kBY) / kBY);
  const int planes = d.nz + 1;
  int z = (int)((xy * planes) / (152 * 2 * 4));
  if (z < 2) z = 2;
  if (z > 32) z = 32;
  while (xy * ((planes + z - 1) / z) > kMaxPartials) ++z;
  return z;
}

}  // namespace

template <typename T>
cudaError_t launch_apply(const T* x, T* y, const T* E, const T* f, const Dims& d, const K0<T>& k0,
                         const Red& red, int mode, const int* done, cudaStream_t s) {
  dim3 block(kBX, kBY, 1);
  const int z = pick_zchunk(d);
  dim3 grid((d.nx + kBX) / kBX, (d.ny + kBY) / kBY, (d.nz + z) / z);
  if constexpr (sizeof(T) == 8) {
    switch (mode) {
      case APPLY_PLAIN:
        k_apply_direct<T, APPLY_PLAIN><<<grid, block, 0, s>>>(x, y, E, f, d, k0, red, z, done);
        break;
      case APPLY_DOT:
        k_apply_direct<T, APPLY_DOT><<<grid, block, 0, s>>>(x, y, E, f, d, k0, red, z, done);
        break;
      default:
        k_apply_direct<T, APPLY_RESID><<<grid, block, 0, s>>>(x, y, E, f, d, k0, red, z, done);
        break;
    }
  } else {
    switch (mode) {
      case APPLY_PLAIN:
        k_apply<T, APPLY_PLAIN><<<grid, block, 0, s>>>(x, y, E, f, d, k0, red, z, done);
        break;
      case APPLY_DOT:
        k_apply<T, APPLY_DOT><<<grid, block, 0, s>>>(x, y, E, f, d, k0, red, z, done);
        break;
      default:
        k_apply<T, APPLY_RESID><<<grid, block, 0, s>>>(x, y, E, f, d, k0, red, z, done);
        break;
    }
  }
  return cudaGetLastError();
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
                                         const int*, cudaStream_t);
template cudaError_t launch_apply<double>(const double*, double*, const double*, const double*,
                                          const Dims&, const K0<double>&, const Red&, int,
                                          const int*, cudaStream_t);
template cudaError_t launch_diag_inv<float>(float*, const float*, const Dims&, const K0<float>&,
                                            cudaStream_t);
template cudaError_t launch_diag_inv<double>(double*, const double*, const Dims&,
                                             const K0<double>&, cudaStream_t);

}  // namespace topo
