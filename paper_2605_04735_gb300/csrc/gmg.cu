// Geometric multigrid V-cycle (see gmg.h).  All grid transfers are gathers
// (no atomics); the Chebyshev smoother's vector updates are fused into the
// operator kernel's epilogue, so one smoothing step is one pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "gmg.h"
#include "gmg_tail.h"
#include "kernels.h"
#include "modal2.cuh"
#include "modal_tc.cuh"
#include "stencil.cuh"

namespace topo {

namespace {

constexpr int kCoarseMaxDof = 400;  // target size of the dense coarsest problem
// prolongation: four fine nodes of a row per thread (k_prolong_add4); 0 keeps
// one node per thread (k_prolong_add)
#ifndef TOPO_PROLONG4
#define TOPO_PROLONG4 1
#endif
constexpr int kPT = 256;

// blocks per design: one item per thread up to 16 blocks per SM in all,
// shared among the nb designs of a batched launch
inline int grid1d(long long n, int nb = 1) {
  long long b = (n + kPT - 1) / kPT;
  const long long cap = std::max(4LL, 152LL * 16 / std::max(nb, 1));
  return (int)std::max(1LL, std::min(b, cap));
}

// ---------------------------------------------------------------- smoother
// Chebyshev iteration for A x = b preconditioned by D^-1, on [lmin, lmax]
// (theta = centre, delta = half width): d_0 = D^-1 r_0 / theta,
// d_k = c1_k d_{k-1} + c2_k D^-1 r_k, r_k = r_{k-1} - A d_{k-1}, x += d_k.

// pre-smoothing start from x = 0: r = b, d0 = D^-1 b / theta, x = d0
// (all kernels below: blockIdx.y = design, buffers at design * S bytes)
__global__ void k_cheb_init(const float* __restrict__ b, float* __restrict__ r,
                            float* __restrict__ d0, float* __restrict__ x,
                            const float* __restrict__ dinv, long long n4, float inv_theta,
                            int d_only, const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  b = bshift(b, off);
  r = bshift(r, off);
  d0 = bshift(d0, off);
  x = bshift(x, off);
  dinv = bshift(dinv, off);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const float4 bv = reinterpret_cast<const float4*>(b)[q];
    const float4 dv = reinterpret_cast<const float4*>(dinv)[q];
    float4 o;
    o.x = dv.x * bv.x * inv_theta;
    o.y = dv.y * bv.y * inv_theta;
    o.z = dv.z * bv.z * inv_theta;
    o.w = dv.w * bv.w * inv_theta;
    reinterpret_cast<float4*>(d0)[q] = o;
    if (!d_only) {
      reinterpret_cast<float4*>(r)[q] = bv;
      reinterpret_cast<float4*>(x)[q] = o;
    }
  }
}

__global__ void k_axpy1(float* __restrict__ x, const float* __restrict__ d, long long n4,
                        const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  x = bshift(x, off);
  d = bshift(d, off);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    float4 xv = reinterpret_cast<float4*>(x)[q];
    const float4 dv = reinterpret_cast<const float4*>(d)[q];
    xv.x += dv.x;
    xv.y += dv.y;
    xv.z += dv.z;
    xv.w += dv.w;
    reinterpret_cast<float4*>(x)[q] = xv;
  }
}

// one Chebyshev step, fused: gathers d_{k-1}; r -= A d_{k-1};
// d_k = c1 d_{k-1} + c2 D^-1 r; x += d_k (+ d_{k-1} when it was not yet added)
struct EpiChebStep {
  static constexpr bool kReduce = false;
  static constexpr int kAux = 2;  // r (read from rin), D^-1
  static constexpr int kDinvAux = 1;
  // how the step's direction reaches x: x += d_q; x += d_{q-1} + d_q (the
  // previous step did not add its own); x = d_{q-1} + d_q (x not yet set)
  enum : int { kXAdd = 0, kXAddPrev = 1, kXStore = 2 };
  float* r;
  const float* rin;  // the residual before the step (r itself, or b on the first step)
  float* dn;
  float* x;
  const float* dinv;
  float c1, c2;
  int xmode;
  __device__ EpiChebStep shifted(long long off) const {
    return EpiChebStep{bshift(r, off), bshift(rin, off), bshift(dn, off), bshift(x, off),
                       bshift(dinv, off), c1, c2, xmode};
  }
  __host__ __device__ const float* aux(int q) const { return q == 0 ? rin : dinv; }
  template <int N, class DD>
  __device__ __forceinline__ float finish(const int (&i)[N], int j, int k,
                                          const long long (&o)[N], const bool (&own)[N],
                                          const float (&acc)[N][3], const float (&ctr)[N][3],
                                          const float (&av)[2][N][3], const DD& d) const {
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n])
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long oc = c * d.comp + o[n];
          const float Ad = d.fixed(c, i[n], j, k) ? 0.0f : acc[n][c];
          const float rn = av[0][n][c] - Ad;
          const float dd = fmaf(c1, ctr[n][c], c2 * av[1][n][c] * rn);
          r[oc] = rn;
          dn[oc] = dd;
          if (xmode == kXStore)
            x[oc] = dd + ctr[n][c];
          else
            red_add(x + oc, xmode == kXAddPrev ? (dd + ctr[n][c]) : dd);
        }
    return 0.0f;
  }
};

// The last post-smoothing step of the finest level with the CG's r.z fused:
// z = x + d_q (+ d_{q-1}) is stored (not added: x is read here, one owner
// per entry), neither r nor d is (nothing reads them after the V-cycle),
// and the per-thread partial of b . z (b: the V-cycle's right-hand side,
// the CG residual) goes to the launch's reduction.
struct EpiChebStepDot {
  static constexpr bool kReduce = true;
  static constexpr int kAux = 2;  // r, D^-1
  static constexpr int kDinvAux = 1;
  const float* r;
  float* x;
  const float* b;
  const float* dinv;
  float c1, c2;
  int add_prev;
  __device__ EpiChebStepDot shifted(long long off) const {
    return EpiChebStepDot{bshift(r, off), bshift(x, off), bshift(b, off), bshift(dinv, off), c1,
                          c2, add_prev};
  }
  __host__ __device__ const float* aux(int q) const { return q == 0 ? r : dinv; }
  template <int N, class DD>
  __device__ __forceinline__ float finish(const int (&i)[N], int j, int k,
                                          const long long (&o)[N], const bool (&own)[N],
                                          const float (&acc)[N][3], const float (&ctr)[N][3],
                                          const float (&av)[2][N][3], const DD& d) const {
    float part = 0.0f;
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n]) {
        float xo[3], bo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {  // both loads before the stores
          xo[c] = x[c * d.comp + o[n]];
          bo[c] = b[c * d.comp + o[n]];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long oc = c * d.comp + o[n];
          const float Ad = d.fixed(c, i[n], j, k) ? 0.0f : acc[n][c];
          const float rn = av[0][n][c] - Ad;
          const float dd = fmaf(c1, ctr[n][c], c2 * av[1][n][c] * rn);
          const float z = xo[c] + (add_prev ? (dd + ctr[n][c]) : dd);
          x[oc] = z;
          part = fmaf(bo[c], z, part);
        }
      }
    return part;
  }
};

// r -= A d (the residual after pre-smoothing)
struct EpiChebLast {
  static constexpr bool kReduce = false;
  static constexpr int kAux = 0;
  static constexpr int kDinvAux = -1;
  float* r;
  __device__ EpiChebLast shifted(long long off) const { return EpiChebLast{bshift(r, off)}; }
  __host__ __device__ const float* aux(int) const { return nullptr; }
  template <int N, class DD>
  __device__ __forceinline__ float finish(const int (&i)[N], int j, int k,
                                          const long long (&o)[N], const bool (&own)[N],
                                          const float (&acc)[N][3], const float (&)[N][3],
                                          const float (&)[1][N][3], const DD& d) const {
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n])
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (!d.fixed(c, i[n], j, k)) red_add(r + c * d.comp + o[n], -acc[n][c]);
    return 0.0f;
  }
};

// post-smoothing start: r = b - A x (gathering x), d0 = D^-1 r / theta
struct EpiChebResid {
  static constexpr bool kReduce = false;
  static constexpr int kAux = 2;  // b, D^-1
  static constexpr int kDinvAux = 1;
  const float* b;
  float* r;
  float* d0;
  const float* dinv;
  float inv_theta;
  __device__ EpiChebResid shifted(long long off) const {
    return EpiChebResid{bshift(b, off), bshift(r, off), bshift(d0, off), bshift(dinv, off),
                        inv_theta};
  }
  __host__ __device__ const float* aux(int q) const { return q == 0 ? b : dinv; }
  template <int N, class DD>
  __device__ __forceinline__ float finish(const int (&i)[N], int j, int k,
                                          const long long (&o)[N], const bool (&own)[N],
                                          const float (&acc)[N][3], const float (&)[N][3],
                                          const float (&av)[2][N][3], const DD& d) const {
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n])
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long oc = c * d.comp + o[n];
          const float rr = d.fixed(c, i[n], j, k) ? 0.0f : (av[0][n][c] - acc[n][c]);
          r[oc] = rr;
          d0[oc] = av[1][n][c] * rr * inv_theta;
        }
    return 0.0f;
  }
};

// ---------------------------------------------------------------- transfers
// coarse element modulus: mean of its (up to) 8 children, times 2 for the
// doubled edge (k0 of an element of edge 2h is 2h times the unit k0);
// children beyond an odd fine grid are ghosts with E = 0
__global__ void k_coarsen_E(const float* __restrict__ Ef, const Dims df, float* __restrict__ Ec,
                            const Dims dc, const DSel S) {
  pdl_start();
  Ef = bshift(Ef, S.off(blockIdx.y));
  Ec = bshift(Ec, S.off(blockIdx.y));
  const long long n = (long long)dc.nx * dc.ny * dc.nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int I, J, K;
    unflatten3(e, dc.nx, dc.ny, I, J, K);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
          if (i < df.nx && j < df.ny && k < df.nz) s += Ef[df.elem(i, j, k)];
        }
    Ec[dc.elem(I, J, K)] = 0.25f * s;
  }
}

// b_c = P^T r_f for trilinear P: coarse node (I,J,K) sits on fine node
// (2I,2J,2K) and collects fine neighbours with weights 1, 1/2 per axis offset
__global__ void k_restrict(const float* __restrict__ rf, const Dims df, float* __restrict__ bc,
                           const Dims dc, const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  rf = bshift(rf, off);
  bc = bshift(bc, off);
  const long long nn = (long long)(dc.nx + 1) * (dc.ny + 1) * (dc.nz + 1);
  // fine node (i, j, k) of component c at rc[c] + i + px j + pz k (one design's
  // vector holds < 2^31 entries)
  const float* rc[3] = {rf + df.node(0, 0, 0), rf + df.comp + df.node(0, 0, 0),
                        rf + 2 * df.comp + df.node(0, 0, 0)};
  const int px = (int)df.row_stride(), pz = (int)df.plane_stride();
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int I, J, K;
    unflatten3(n, dc.nx + 1, dc.ny + 1, I, J, K);
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
      const int k = 2 * K + dk;
      if (k < 0 || k > df.nz) continue;
      const float wk = dk ? 0.5f : 1.0f;
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
        const int j = 2 * J + dj;
        if (j < 0 || j > df.ny) continue;
        const float wjk = wk * (dj ? 0.5f : 1.0f);
        const int row = px * j + pz * k;
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const int i = 2 * I + di;
          if (i < 0 || i > df.nx) continue;
          const float wt = wjk * (di ? 0.5f : 1.0f);
#pragma unroll
          for (int c = 0; c < 3; ++c) s[c] = fmaf(wt, rc[c][row + i], s[c]);
        }
      }
    }
    const long long o = dc.node(I, J, K);
#pragma unroll
    for (int c = 0; c < 3; ++c) bc[c * dc.comp + o] = dc.fixed(c, I, J, K) ? 0.0f : s[c];
  }
}

// x_f += P x_c (trilinear interpolation from the coarse nodes around each
// fine node), fixed fine DOFs untouched
__global__ void k_prolong_add(const float* __restrict__ xc, const Dims dc, float* __restrict__ xf,
                              const Dims df, const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  xc = bshift(xc, off);
  xf = bshift(xf, off);
  const long long nn = (long long)(df.nx + 1) * (df.ny + 1) * (df.nz + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(n, df.nx + 1, df.ny + 1, i, j, k);
    // trilinear interpolation: an even index sits on coarse node i/2 (weight
    // 1), an odd one halfway between i/2 and i/2+1 (1/2 each; clamped to the
    // last coarse node where the coarse grid rounded up).  Rows are read only
    // where their weight is non-zero: the y-z parity is the same along a row.
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const bool oi = i & 1, oj = j & 1, ok = k & 1;
    const int di = min(i0 + 1, dc.nx) - i0;
    const long long dy = (long long)(min(j0 + 1, dc.ny) - j0) * dc.row_stride();
    const long long dz = (long long)(min(k0 + 1, dc.nz) - k0) * dc.plane_stride();
    const long long cb = dc.node(i0, j0, k0);
    const float wjk = (oj ? 0.5f : 1.0f) * (ok ? 0.5f : 1.0f);
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      if (c2 && !ok) break;
#pragma unroll
      for (int b2 = 0; b2 < 2; ++b2) {
        if (b2 && !oj) break;
        const long long o = cb + (b2 ? dy : 0) + (c2 ? dz : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* p = xc + c * dc.comp + o;
          const float v = oi ? 0.5f * (p[0] + p[di]) : p[0];
          s[c] = fmaf(wjk, v, s[c]);
        }
      }
    }
    const long long o = df.node(i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (!df.fixed(c, i, j, k)) xf[c * df.comp + o] += s[c];
  }
}

// The same update, four fine nodes of a row per thread: storage entries
// 4q .. 4q+3 of a node row (i = 4q-1 .. 4q+2; rows are 16-byte aligned) are
// read and written as one float4 per component, and the three coarse
// columns 2q-1 .. 2q+1 that interpolate them are read once per coarse row.
// Per node the arithmetic is k_prolong_add's, in its order (the clamp of
// the odd nodes' right neighbour never acts on a node of the grid: odd
// i <= nx - 1 has i/2 + 1 <= nx/2 <= the coarse nx).  Ghost entries keep 0.
__global__ void k_prolong_add4(const float* __restrict__ xc, const Dims dc,
                               float* __restrict__ xf, const Dims df,
                               const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  xc = bshift(xc, off);
  xf = bshift(xf, off);
  const int nq = (df.nx + 2 + 3) / 4;  // quads of a row holding i = -1 .. nx
  const int nrow = (df.ny + 1) * (df.nz + 1);
  const int total = nq * nrow;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int row = t / nq, q = t - row * nq;
    const int j = row % (df.ny + 1), k = row / (df.ny + 1);
    const int j0 = j >> 1, k0 = k >> 1;
    const bool oj = j & 1, ok = k & 1;
    const long long dy = (long long)(min(j0 + 1, dc.ny) - j0) * dc.row_stride();
    const long long dz = (long long)(min(k0 + 1, dc.nz) - k0) * dc.plane_stride();
    const long long cb = dc.node(2 * q - 1, j0, k0);  // coarse column 2q - 1 (a ghost for q = 0)
    const float wjk = (oj ? 0.5f : 1.0f) * (ok ? 0.5f : 1.0f);
    float s[3][4] = {};
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      if (c2 && !ok) break;
#pragma unroll
      for (int b2 = 0; b2 < 2; ++b2) {
        if (b2 && !oj) break;
        const long long o = cb + (b2 ? dy : 0) + (c2 ? dz : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* p = xc + c * dc.comp + o;
          const float a = p[0], b = p[1], e = p[2];
          s[c][0] = fmaf(wjk, 0.5f * (a + b), s[c][0]);  // i = 4q - 1 (odd)
          s[c][1] = fmaf(wjk, b, s[c][1]);                // i = 4q
          s[c][2] = fmaf(wjk, 0.5f * (b + e), s[c][2]);  // i = 4q + 1 (odd)
          s[c][3] = fmaf(wjk, e, s[c][3]);                // i = 4q + 2
        }
      }
    }
    const long long o = df.node(4 * q - 1, j, k);  // storage entry 4q: 16-byte aligned
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4* px = reinterpret_cast<float4*>(xf + c * df.comp + o);
      float4 v = *px;
      float* vv = reinterpret_cast<float*>(&v);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 4 * q - 1 + e;
        if (i >= 0 && i <= df.nx && !df.fixed(c, i, j, k)) vv[e] += s[c][e];
      }
      *px = v;
    }
  }
}

// ---------------------------------------------------------------- coarsest grid
// dense FP64 matrix of the masked operator on the coarsest grid, one entry
// per thread, summed over the elements shared by the two nodes (a gather:
// deterministic, no atomics)
__global__ void k_dense_assemble(double* __restrict__ A, const Dims d, const float* __restrict__ E,
                                 const __grid_constant__ K0<double> k0, const DSel S) {
  pdl_start();
  A = bshift(A, S.off(blockIdx.y));
  E = bshift(E, S.off(blockIdx.y));
  const int n = 3 * (d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / n), col = (int)(t % n);
    const int p = row / 3, r = row % 3, q = col / 3, s = col % 3;
    const int pi = p % (d.nx + 1), pj = (p / (d.nx + 1)) % (d.ny + 1),
              pk = p / ((d.nx + 1) * (d.ny + 1));
    const int qi = q % (d.nx + 1), qj = (q / (d.nx + 1)) % (d.ny + 1),
              qk = q / ((d.nx + 1) * (d.ny + 1));
    double v = 0.0;
    const bool fr = d.fixed(r, pi, pj, pk), fc = d.fixed(s, qi, qj, qk);
    if (fr || fc) {
      v = (row == col) ? 1.0 : 0.0;
    } else if (abs(pi - qi) <= 1 && abs(pj - qj) <= 1 && abs(pk - qk) <= 1) {
      for (int ek = max(max(pk, qk) - 1, 0); ek <= min(min(pk, qk), d.nz - 1); ++ek)
        for (int ej = max(max(pj, qj) - 1, 0); ej <= min(min(pj, qj), d.ny - 1); ++ej)
          for (int ei = max(max(pi, qi) - 1, 0); ei <= min(min(pi, qi), d.nx - 1); ++ei) {
            const int lp = 4 * (pk - ek) + ((pj - ej) ? ((pi - ei) ? 2 : 3) : ((pi - ei) ? 1 : 0));
            const int lq = 4 * (qk - ek) + ((qj - ej) ? ((qi - ei) ? 2 : 3) : ((qi - ei) ? 1 : 0));
            v += (double)E[d.elem(ei, ej, ek)] * k0.v[(3 * lp + r) * 24 + 3 * lq + s];
          }
    }
    A[t] = v;
  }
}

// In-place Gauss-Jordan inversion of the SPD coarsest matrix (no pivoting
// needed: every pivot is a Schur-complement diagonal, hence positive), one
// kernel per pivot k.  The pivot row and column as they were before step k
// are read from side buffers that step k-1 wrote (ping-pong), so no entry is
// read after being overwritten in the same step.  (Kernel boundaries are the
// barriers: a single cooperative kernel with grid-wide barriers is not safe
// when many meshes set up concurrently on their own streams.)  The chain of
// n launches is captured once per hierarchy as a CUDA graph.
__global__ void k_gj_seed(const double* __restrict__ A, int n, double* __restrict__ row,
                          double* __restrict__ col, const DSel S) {
  pdl_start();
  A = bshift(A, S.off(blockIdx.y));
  row = bshift(row, S.off(blockIdx.y));
  col = bshift(col, S.off(blockIdx.y));
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    row[t] = A[t];
    col[t] = A[(long long)t * n];
  }
}

__global__ void k_gj_step(double* __restrict__ A, int n, int k, const double* __restrict__ rowk,
                          const double* __restrict__ colk, double* __restrict__ rown,
                          double* __restrict__ coln, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  A = bshift(A, off);
  rowk = bshift(rowk, off);
  colk = bshift(colk, off);
  rown = bshift(rown, off);
  coln = bshift(coln, off);
  __shared__ double sp;  // the pivot's reciprocal, one division per block
  if (threadIdx.x == 0) sp = 1.0 / rowk[k];
  __syncthreads();
  const double p = sp;
  // block b: rows b, b + gridDim.x, ...; threads across the row
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    double* Ai = A + (long long)i * n;
    const double ci = colk[i];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double v;
      if (i == k && j == k)
        v = p;
      else if (i == k)
        v = rowk[j] * p;
      else if (j == k)
        v = -ci * p;
      else
        v = Ai[j] - ci * rowk[j] * p;
      Ai[j] = v;
      if (i == k + 1) rown[j] = v;
      if (j == k + 1) coln[i] = v;
    }
  }
}

// The coarsest inverse in one kernel per design, for batched setups (one
// design alone keeps the pivot chain below: a single SM's FP64 rate makes
// this kernel no faster than the chain for one design, but a batch fills the
// SMs with designs and saves the chain's n launches).  The symmetric sweep
// operator on the packed lower triangle in shared memory: sweeping pivot k
// maps a_kk -> -1/a_kk, a_ik -> a_ik/a_kk (i != k) and a_ij -> a_ij -
// a_ik a_kj / a_kk; after all n pivots the matrix holds -A^-1 (no pivoting:
// every pivot is a Schur-complement diagonal of the SPD A, as in
// Gauss-Jordan).  CTA barriers separate the pivots.  In: the dense n x n A
// at A; out: A^-1 (full, symmetric).
constexpr int kSweepThreads = 1024;
constexpr int kSweepMaxN = 222;  // n (n + 1) / 2 + 2 n doubles within 200 KB
constexpr int kSweepPer = (kSweepMaxN * (kSweepMaxN + 1) / 2 + kSweepThreads - 1) / kSweepThreads;

__global__ void __launch_bounds__(kSweepThreads)
    k_gj_sweep(double* __restrict__ A, int n, const DSel S) {
  pdl_start();
  A = bshift(A, S.off(blockIdx.y));
  extern __shared__ double sweep_smem[];
  double* P = sweep_smem;        // packed: (i, j), i >= j at i (i + 1) / 2 + j
  const int np = n * (n + 1) / 2;
  double* col = P + np;          // column k before pivot k
  double* cs = col + n;          // the same divided by the pivot
  // this thread's packed entries t = tid + q * blockDim.x as (i, j)
  int ij[kSweepPer];
#pragma unroll
  for (int q = 0; q < kSweepPer; ++q) {
    const int t = threadIdx.x + q * kSweepThreads;
    int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    if (i * (i + 1) / 2 > t) --i;
    if ((i + 1) * (i + 2) / 2 <= t) ++i;
    ij[q] = (i << 16) | (t - i * (i + 1) / 2);
    if (t < np) P[t] = A[(long long)i * n + (t - i * (i + 1) / 2)];
  }
  for (int k = 0; k < n; ++k) {
    __syncthreads();  // the previous pivot's updates are done
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      col[i] = i >= k ? P[i * (i + 1) / 2 + k] : P[k * (k + 1) / 2 + i];
    __syncthreads();
    const double inv = 1.0 / col[k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) cs[i] = col[i] * inv;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSweepPer; ++q) {
      const int t = threadIdx.x + q * kSweepThreads;
      if (t >= np) break;
      const int i = ij[q] >> 16, j = ij[q] & 0xffff;
      double v;
      if (i == k)
        v = (j == k) ? -inv : cs[j];
      else if (j == k)
        v = cs[i];
      else
        v = fma(-col[i], cs[j], P[t]);
      P[t] = v;
    }
  }
  __syncthreads();
  const long long nn = (long long)n * n;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / n), j = (int)(t - (long long)i * n);
    A[t] = -(i >= j ? P[i * (i + 1) / 2 + j] : P[j * (j + 1) / 2 + i]);
  }
}

__global__ void k_coarse_gather(const float* __restrict__ b, const Dims d, double* __restrict__ bd,
                                const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  b = bshift(b, off);
  bd = bshift(bd, off);
  const int nn = (d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
    const int i = n % (d.nx + 1), j = (n / (d.nx + 1)) % (d.ny + 1),
              k = n / ((d.nx + 1) * (d.ny + 1));
    const long long o = d.node(i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) bd[3 * n + c] = (double)b[c * d.comp + o];
  }
}

// x = A^-1 b, one warp per row (A^-1 symmetric, rows read coalesced), FP64
__global__ void k_coarse_apply(const double* __restrict__ Ainv, const double* __restrict__ bd,
                               int n, float* __restrict__ x, const Dims d,
                               const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;
  Ainv = bshift(Ainv, off);
  bd = bshift(bd, off);
  x = bshift(x, off);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* a = Ainv + (long long)warp * n;
  double s = 0.0;
  for (int t = lane; t < n; t += 32) s = fma(a[t], bd[t], s);
  s = warp_sum(s);
  if (lane == 0) {
    const int node = warp / 3, c = warp % 3;
    const int i = node % (d.nx + 1), j = (node / (d.nx + 1)) % (d.ny + 1),
              k = node / ((d.nx + 1) * (d.ny + 1));
    x[c * d.comp + d.node(i, j, k)] = d.fixed(c, i, j, k) ? 0.0f : (float)s;
  }
}

// Zero-filled allocation, ordered on the mesh's own stream (a plain
// cudaMemset would go to the legacy default stream, which does not order
// against the mesh's non-blocking stream).
template <typename T>
cudaError_t dmalloc(T** p, long long count, long long* bytes, cudaStream_t s,
                    const GmgAlloc* alloc) {
  cudaError_t e = alloc ? alloc->fn(alloc->ctx, reinterpret_cast<void**>(p),
                                    (size_t)count * sizeof(T))
                        : cudaMalloc(reinterpret_cast<void**>(p), (size_t)count * sizeof(T));
  if (e != cudaSuccess) return e;
  *bytes += count * (long long)sizeof(T);
  return cudaMemsetAsync(*p, 0, (size_t)count * sizeof(T), s);
}

#define GCK(call)                          \
  do {                                     \
    cudaError_t e__ = (call);              \
    if (e__ != cudaSuccess) return e__;    \
  } while (0)

struct ChebCoef {
  float inv_theta;
  std::vector<float> c1, c2;  // index k = 1..degree-1
};

ChebCoef cheb_coef(double lmax, double ratio, int degree) {
  const double lmin = lmax / ratio;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  ChebCoef c;
  c.inv_theta = (float)(1.0 / theta);
  c.c1.assign(degree, 0.f);
  c.c2.assign(degree, 0.f);
  double rho_prev = 1.0 / sigma;
  for (int k = 1; k < degree; ++k) {
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    c.c1[k] = (float)(rho * rho_prev);
    c.c2[k] = (float)(2.0 * rho / delta);
    rho_prev = rho;
  }
  return c;
}

}  // namespace

double k0_jacobi_bound(const double* k0) {
  // power iteration on S = D^-1/2 k0 D^-1/2 (symmetric positive semidefinite)
  double dis[24], v[24], w[24];
  for (int a = 0; a < 24; ++a) {
    dis[a] = 1.0 / std::sqrt(k0[a * 24 + a]);
    v[a] = 1.0 + 0.01 * a;
  }
  double lam = 0.0;
  for (int it = 0; it < 500; ++it) {
    double nrm = 0.0;
    for (int a = 0; a < 24; ++a) {
      double s = 0.0;
      for (int b = 0; b < 24; ++b) s += dis[a] * k0[a * 24 + b] * dis[b] * v[b];
      w[a] = s;
      nrm += s * s;
    }
    nrm = std::sqrt(nrm);
    double dot = 0.0;
    for (int a = 0; a < 24; ++a) dot += v[a] * w[a];
    double vn = 0.0;
    for (int a = 0; a < 24; ++a) vn += v[a] * v[a];
    lam = dot / vn;
    for (int a = 0; a < 24; ++a) v[a] = w[a] / nrm;
  }
  return lam;
}

std::vector<Dims> gmg_plan(const Dims& fine, int max_levels, int max_dof) {
  std::vector<Dims> out;
  Dims d = fine;
  for (;;) {
    out.push_back(d);
    const long long dof = 3LL * (d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    if (dof <= max_dof) break;
    if (max_levels > 0 && (int)out.size() >= max_levels) break;
    const int nx = (d.nx + 1) / 2, ny = (d.ny + 1) / 2, nz = (d.nz + 1) / 2;
    if (nx == d.nx && ny == d.ny && nz == d.nz) break;
    d = make_dims(nx, ny, nz, d.bc, d.pin_j / 2);
    if ((int)out.size() >= 16) break;
  }
  return out;
}

long long gmg_footprint(const Dims& fine, int max_levels) {
  const std::vector<Dims> lv = gmg_plan(fine, max_levels);
  long long b = 0;
  for (size_t l = 0; l < lv.size(); ++l) {
    const long long nvec = 3 * lv[l].comp;
    b += nvec * 4 * 3;                                  // r, two Chebyshev directions
    if (l > 0) b += lv[l].ecount * 4 + nvec * 4 * 3;    // E, dinv, b, x
  }
  const Dims& dc = lv.back();
  const long long nc = 3LL * (dc.nx + 1) * (dc.ny + 1) * (dc.nz + 1);
  b += (nc * nc + 5 * nc) * 8;
  return b;
}

cudaError_t gmg_create(Gmg& g, const Dims& fine, int max_levels, int degree, double lam_max,
                       cudaStream_t s, const GmgAlloc* alloc, bool throughput) {
  g.arena = (alloc != nullptr);
  g.degree = std::max(1, degree);
  g.lam_max = lam_max;
  g.throughput = throughput;
  g.lv.clear();
  for (const Dims& d : gmg_plan(fine, max_levels, throughput ? kSweepMaxN : kCoarseMaxDof)) {
    GmgLevel L;
    L.d = d;
    L.nvec = 3 * d.comp;
    g.lv.push_back(L);
  }
  const Dims& dc = g.lv.back().d;
  g.nc = 3 * (dc.nx + 1) * (dc.ny + 1) * (dc.nz + 1);
  if ((long long)g.nc * g.nc > (1LL << 27)) return cudaErrorInvalidValue;  // > 1 GB inverse
  for (size_t l = 0; l < g.lv.size(); ++l) {
    GmgLevel& L = g.lv[l];
    GCK(dmalloc(&L.r, L.nvec, &g.bytes, s, alloc));
    GCK(dmalloc(&L.dv[0], L.nvec, &g.bytes, s, alloc));
    GCK(dmalloc(&L.dv[1], L.nvec, &g.bytes, s, alloc));
    if (l > 0) {
      GCK(dmalloc(&L.E, L.d.ecount, &g.bytes, s, alloc));
      GCK(dmalloc(&L.dinv, L.nvec, &g.bytes, s, alloc));
      GCK(dmalloc(&L.b, L.nvec, &g.bytes, s, alloc));
      GCK(dmalloc(&L.x, L.nvec, &g.bytes, s, alloc));
    }
  }
  {
    std::vector<Dims> dims;
    for (const GmgLevel& L : g.lv) dims.push_back(L.d);
    g.tail_l0 = tail_first_level(dims, g.degree);
  }
  GCK(dmalloc(&g.Ainv, (long long)g.nc * g.nc, &g.bytes, s, alloc));
  GCK(dmalloc(&g.side, 4LL * g.nc, &g.bytes, s, alloc));
  GCK(dmalloc(&g.bd, (long long)g.nc, &g.bytes, s, alloc));
  g.ready = false;
  return cudaSuccess;
}

cudaError_t gmg_setup(Gmg& g, const float* E0, const float* dinv0, const K0<float>& k0f,
                      const K0<double>& k0d, cudaStream_t s, long long* launches, const Bat& bt) {
  if (bt.ids) return cudaErrorInvalidValue;  // the setup covers every design of a batch
  g.lv[0].E = const_cast<float*>(E0);
  g.lv[0].dinv = const_cast<float*>(dinv0);
  for (size_t l = 1; l < g.lv.size(); ++l) {
    const GmgLevel& F = g.lv[l - 1];
    GmgLevel& C = g.lv[l];
    const long long ne = (long long)C.d.nx * C.d.ny * C.d.nz;
    GCK(launch_pdl(k_coarsen_E, dim3(grid1d(ne, bt.nb), bt.nb), dim3(kPT), 0, s, F.E, F.d, C.E,
                   C.d, bt.sel()));
    GCK(launch_diag_inv<float>(C.dinv, C.E, C.d, k0f, s, bt));
    *launches += 2;
  }
  const GmgLevel& Lc = g.lv.back();
  const long long nn = (long long)g.nc * g.nc;
  GCK(launch_pdl(k_dense_assemble, dim3(grid1d(nn, bt.nb), bt.nb), dim3(kPT), 0, s, g.Ainv, Lc.d,
                 Lc.E, k0d, bt.sel()));
  // a batch, or the throughput form: the whole inverse in one kernel per design
  if ((bt.nb > 1 || g.throughput) && g.nc <= kSweepMaxN) {
    const size_t smem = sizeof(double) * ((size_t)g.nc * (g.nc + 1) / 2 + 2 * g.nc);
    static bool attr = false;
    if (!attr) {
      GCK(cudaFuncSetAttribute(k_gj_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(sizeof(double) * ((size_t)kSweepMaxN * (kSweepMaxN + 1) / 2 +
                                                       2 * kSweepMaxN))));
      attr = true;
    }
    GCK(launch_pdl(k_gj_sweep, dim3(1, bt.nb), dim3(kSweepThreads), smem, s, g.Ainv, g.nc,
                   bt.sel()));
    *launches += 2;  // the dense assembly and the sweep
    g.ready = true;
    return cudaSuccess;
  }
  // the pivot chain, captured once per batch shape as a graph and replayed per density
  if (g.gj_exec && (g.gj_nb != bt.nb || g.gj_S != bt.S)) {
    cudaGraphExecDestroy(g.gj_exec);
    g.gj_exec = nullptr;
  }
  if (!g.gj_exec) {
    cudaStream_t cs = nullptr;
    GCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      double* buf[2][2] = {{g.side, g.side + g.nc}, {g.side + 2 * g.nc, g.side + 3 * g.nc}};
      e = launch_pdl(k_gj_seed, dim3((g.nc + kPT - 1) / kPT, bt.nb), dim3(kPT), 0, cs, g.Ainv,
                     g.nc, buf[0][0], buf[0][1], bt.sel());
      for (int k = 0; k < g.nc && e == cudaSuccess; ++k) {
        double** cur = buf[k & 1];
        double** nxt = buf[(k + 1) & 1];
        e = launch_pdl(k_gj_step, dim3(std::min(g.nc, 1024), bt.nb), dim3(128), 0, cs, g.Ainv,
                       g.nc, k, cur[0], cur[1], nxt[0], nxt[1], bt.sel());
      }
      const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.gj_exec, graph, 0);
    g.gj_nb = bt.nb;
    g.gj_S = bt.S;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    GCK(e);
  }
  GCK(cudaGraphLaunch(g.gj_exec, s));
  *launches += 2 + g.nc;  // the dense assembly, the seed and the pivot steps
  g.ready = true;
  return cudaSuccess;
}

template <class Epi>
cudaError_t level_op(const float* x, const GmgLevel& L, const K0<float>& k0f,
                     const ModalCoef<float>* mcf, const Epi& ep, const int* done, int* errflag,
                     cudaStream_t s, const Bat& bt, const Red& red = Red{}) {
  // the smoother's operator: one TF32 pass on the tensor-core form (a fixed
  // approximation of the level operator is all a smoother needs)
  if (mcf)
    return launch_modal_any<TOPO_TC_SMOOTH_PASSES, float>(x, L.E, L.d, *mcf, k0f, ep, red, done,
                                                         errflag, s, bt);
  if (bt.nb != 1) return cudaErrorInvalidValue;  // the gather kernels run one design
  return launch_stencil<float>(x, L.E, L.d, k0f, ep, red, done, errflag, s);
}

float gmg_first_direction(const Gmg& g, float** d0) {
  if (g.lv.size() < 2 || g.degree < 2) return 0.0f;  // no finest-level smoothing step
  *d0 = g.lv[0].dv[0];
  return cheb_coef(g.lam_max, g.lam_ratio, g.degree).inv_theta;
}

cudaError_t gmg_vcycle(Gmg& g, const float* b0, float* x0, const K0<float>& k0f,
                       const ModalCoef<float>* mcf, const int* done, int* errflag,
                       cudaStream_t s, long long* launches, const Bat& bt, const Red* zdot,
                       bool d0_ready, GmgProf* prof) {
  // event pair around a finest-level Chebyshev step (prof given and room left)
  auto mark = [&](int l, bool after, bool store) -> cudaError_t {
    if (!prof || l != 0 || prof->n >= prof->cap) return cudaSuccess;
    const cudaError_t e =
        cudaEventRecordWithFlags(prof->ev[2 * prof->n + (after ? 1 : 0)], s, cudaEventRecordExternal);
    if (after) prof->store[prof->n++] = store ? 1 : 0;
    return e;
  };
  const ChebCoef cc = cheb_coef(g.lam_max, g.lam_ratio, g.degree);
  const int m = g.degree;
  const int nl = (int)g.lv.size();
  auto B = [&](int l) { return l == 0 ? b0 : g.lv[l].b; };
  auto X = [&](int l) { return l == 0 ? x0 : g.lv[l].x; };
  // Levels >= l_end run as one kernel per design (the tail) when several
  // designs share the launch: one SM per design is then the better use of the
  // GPU than a few-microsecond launch per coarse step.  A single design keeps
  // the per-level kernels, which spread each level over many SMs.
  const bool tail = g.tail_l0 > 0 && (bt.nb > 1 || g.throughput);
  const int l_end = tail ? g.tail_l0 : nl - 1;
  // down
  for (int l = 0; l < l_end; ++l) {
    GmgLevel& L = g.lv[l];
    const long long n4 = L.nvec / 4;
    // d0 = D^-1 b / theta; with further steps the first one reads b as its
    // residual and sets x = d0 + d1, so r = b and x = d0 are not written here
    // (on the finest level the CG update may have written d0 already)
    if (!(l == 0 && d0_ready && m > 1)) {
      GCK(launch_pdl(k_cheb_init, dim3(grid1d(n4, bt.nb), bt.nb), dim3(kPT), 0, s, B(l), L.r,
                     L.dv[0], X(l), L.dinv, n4, cc.inv_theta, m > 1 ? 1 : 0, done, bt.sel()));
      ++*launches;
    }
    for (int k = 1; k < m; ++k) {
      EpiChebStep ep{L.r, k == 1 ? B(l) : L.r, L.dv[k & 1], X(l), L.dinv, cc.c1[k], cc.c2[k],
                     k == 1 ? EpiChebStep::kXStore : EpiChebStep::kXAdd};
      GCK(mark(l, false, false));
      GCK(level_op(L.dv[(k - 1) & 1], L, k0f, mcf, ep, done, errflag, s, bt));
      GCK(mark(l, true, ep.xmode == EpiChebStep::kXStore));
      ++*launches;
    }
    GCK(level_op(L.dv[(m - 1) & 1], L, k0f, mcf, EpiChebLast{L.r}, done, errflag, s, bt));
    const GmgLevel& C = g.lv[l + 1];
    const long long nnc = (long long)(C.d.nx + 1) * (C.d.ny + 1) * (C.d.nz + 1);
    GCK(launch_pdl(k_restrict, dim3(grid1d(nnc, bt.nb), bt.nb), dim3(kPT), 0, s, L.r, L.d, C.b,
                   C.d, done, bt.sel()));
    *launches += 2;
  }
  if (tail) {  // levels l_end .. coarsest in one kernel per design
    TailPlan p{};
    p.nt = nl - 1 - l_end;
    p.degree = m;
    p.inv_theta = cc.inv_theta;
    for (int k = 1; k < m; ++k) {
      p.c1[k] = cc.c1[k];
      p.c2[k] = cc.c2[k];
    }
    p.kdiag = k0f.v[0];
    p.nc = g.nc;
    std::vector<Dims> dims;
    for (const GmgLevel& L : g.lv) dims.push_back(L.d);
    const size_t smem = tail_plan_smem(dims, l_end, p.off);
    for (int t = 0; t <= p.nt; ++t) p.d[t] = g.lv[l_end + t].d;
    for (int t = 0; t < p.nt; ++t) p.E[t] = g.lv[l_end + t].E;
    p.b = g.lv[l_end].b;
    p.x = g.lv[l_end].x;
    p.Ainv = g.Ainv;
    GCK(launch_vcycle_tail(p, smem, k0f, done, s, bt));
    ++*launches;
  } else {  // coarsest
    const GmgLevel& C = g.lv[nl - 1];
    const int nnc = (C.d.nx + 1) * (C.d.ny + 1) * (C.d.nz + 1);
    GCK(launch_pdl(k_coarse_gather, dim3((nnc + kPT - 1) / kPT, bt.nb), dim3(kPT), 0, s,
                   B(nl - 1), C.d, g.bd, done, bt.sel()));
    const long long thr = 32LL * g.nc;
    GCK(launch_pdl(k_coarse_apply, dim3((int)((thr + kPT - 1) / kPT), bt.nb), dim3(kPT), 0, s,
                   g.Ainv, g.bd, g.nc, X(nl - 1), C.d, done, bt.sel()));
    *launches += 2;
  }
  // up
  bool fused = false;  // b . x reduced by the last finest-level step
  for (int l = l_end - 1; l >= 0; --l) {
    GmgLevel& L = g.lv[l];
    const GmgLevel& C = g.lv[l + 1];
#if TOPO_PROLONG4
    {
      const long long nq4 = (long long)((L.d.nx + 5) / 4) * (L.d.ny + 1) * (L.d.nz + 1);
      GCK(launch_pdl(k_prolong_add4, dim3(grid1d(nq4, bt.nb), bt.nb), dim3(kPT), 0, s, X(l + 1),
                     C.d, X(l), L.d, done, bt.sel()));
    }
#else
    const long long nnf = (long long)(L.d.nx + 1) * (L.d.ny + 1) * (L.d.nz + 1);
    GCK(launch_pdl(k_prolong_add, dim3(grid1d(nnf, bt.nb), bt.nb), dim3(kPT), 0, s, X(l + 1), C.d,
                   X(l), L.d, done, bt.sel()));
#endif
    EpiChebResid er{B(l), L.r, L.dv[0], L.dinv, cc.inv_theta};
    GCK(level_op(X(l), L, k0f, mcf, er, done, errflag, s, bt));
    *launches += 2;
    for (int k = 1; k < m; ++k) {
      if (l == 0 && zdot && k == m - 1) {  // the V-cycle's last step, with b . z
        EpiChebStepDot ep{L.r, X(0), b0, L.dinv, cc.c1[k], cc.c2[k], k == 1 ? 1 : 0};
        GCK(level_op(L.dv[(k - 1) & 1], L, k0f, mcf, ep, done, errflag, s, bt, *zdot));
        fused = true;
      } else {
        EpiChebStep ep{L.r, L.r, L.dv[k & 1], X(l), L.dinv, cc.c1[k], cc.c2[k],
                       k == 1 ? EpiChebStep::kXAddPrev : EpiChebStep::kXAdd};
        GCK(mark(l, false, false));
        GCK(level_op(L.dv[(k - 1) & 1], L, k0f, mcf, ep, done, errflag, s, bt));
        GCK(mark(l, true, false));
      }
      ++*launches;
    }
    if (m == 1) {
      GCK(launch_pdl(k_axpy1, dim3(grid1d(L.nvec / 4, bt.nb), bt.nb), dim3(kPT), 0, s, X(l),
                     L.dv[0], L.nvec / 4, done, bt.sel()));
      ++*launches;
    }
  }
  if (zdot && !fused) {  // no finest-level smoothing step to fuse the product into
    GCK(launch_dot<float>(b0, x0, g.lv[0].nvec, *zdot, s, bt));
    ++*launches;
  }
  return cudaSuccess;
}

void gmg_free(Gmg& g) {
  if (g.gj_exec) cudaGraphExecDestroy(g.gj_exec);
  g.gj_exec = nullptr;
  if (g.arena) {  // the buffers belong to the mesh group's arena
    g.lv.clear();
    return;
  }
  for (size_t l = 0; l < g.lv.size(); ++l) {
    GmgLevel& L = g.lv[l];
    cudaFree(L.r);
    cudaFree(L.dv[0]);
    cudaFree(L.dv[1]);
    if (l > 0) {
      cudaFree(L.E);
      cudaFree(L.dinv);
      cudaFree(L.b);
      cudaFree(L.x);
    }
  }
  g.lv.clear();
  cudaFree(g.Ainv);
  cudaFree(g.side);
  cudaFree(g.bd);
  g.Ainv = g.side = g.bd = nullptr;
  g.ready = false;
}

}  // namespace topo
