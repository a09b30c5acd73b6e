// The coarse end of the multigrid V-cycle in one kernel per design.
//
// The levels from l0 down (at most kTailMaxNodes nodes each) are too small to
// fill the GPU even for a batch of designs: each of their launches is a few
// microseconds of latency for less work than that.  For batched V-cycles this
// kernel runs them in one CTA per design, every vector of those levels in
// shared memory:
// on each level Chebyshev(Jacobi) pre-smoothing, restriction, the coarsest
// solve by the FP64 explicit inverse, and on the way up prolongation and
// post-smoothing — the same steps, coefficients and transfers as the
// per-level kernels of gmg.cu, with CTA barriers between them.  The operator
// is the node-centric gather with the dense k0 (576 FMAs per node; k0 sits in
// the constant bank as a kernel parameter), D^-1 = 1 / (kdiag * the sum of
// the moduli around the node).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "gmg.h"
#include "gmg_tail.h"

namespace topo {

namespace {

constexpr int kTailThreads = 512;

__device__ __forceinline__ int tail_lidx(int dx, int dy, int dz) {
  return 4 * dz + (dy ? (dx ? 2 : 3) : (dx ? 1 : 0));
}

// shared-memory views of one level (dense node order n = i + (nx+1)(j + (ny+1)k),
// component-major; dense element order e = i + nx (j + ny k))
struct LevelView {
  Dims d;
  int nn;
  float* b;
  float* x;
  float* r;
  float* dv[2];
  float* E;
};

__device__ __forceinline__ void node_ijk(const Dims& d, int n, int& i, int& j, int& k) {
  unflatten3(n, d.nx + 1, d.ny + 1, i, j, k);
}

// acc = (K u)(i, j, k) of the unmasked operator and esum = the moduli around
// the node: for each of the 8 elements around the node (E = 0 outside the
// grid) its 8 nodes' u are read from shared memory and contracted with the
// element's rows of k0, which are warp-uniform constant operands (k0 is a
// kernel parameter).
__device__ __forceinline__ void gather_apply(const LevelView& L, const float* u,
                                             const K0<float>& k0, int i, int j, int k,
                                             float (&acc)[3], float& esum) {
  const Dims& d = L.d;
  const int sn = L.nn;
  const int sx = d.nx + 1, sxy = (d.nx + 1) * (d.ny + 1);
  acc[0] = acc[1] = acc[2] = 0.f;
  esum = 0.f;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int ei = i - 1 + a, ej = j - 1 + b, ek = k - 1 + c;
        const bool in = ei >= 0 && ei < d.nx && ej >= 0 && ej < d.ny && ek >= 0 && ek < d.nz;
        if (!in) continue;
        const float Ee = L.E[ei + d.nx * (ej + d.ny * ek)];
        esum += Ee;
        const int ln = tail_lidx(1 - a, 1 - b, 1 - c);
        const int n0 = ei + sx * ej + sxy * ek;
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
          for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
              const int lm = tail_lidx(dx, dy, dz);
              const int n = n0 + dx + sx * dy + sxy * dz;
#pragma unroll
              for (int q = 0; q < 3; ++q) {
                const float uq = u[q * sn + n];
#pragma unroll
                for (int r = 0; r < 3; ++r) s[r] = fmaf(k0.v[(3 * ln + r) * 24 + 3 * lm + q], uq, s[r]);
              }
            }
#pragma unroll
        for (int r = 0; r < 3; ++r) acc[r] = fmaf(Ee, s[r], acc[r]);
      }
}

// the moduli of the (up to 8) elements around node (i, j, k)
__device__ __forceinline__ float node_esum(const LevelView& L, int i, int j, int k) {
  const Dims& d = L.d;
  float es = 0.f;
  for (int c = 0; c < 2; ++c) {
    const int ek = k - 1 + c;
    if (ek < 0 || ek >= d.nz) continue;
    for (int b = 0; b < 2; ++b) {
      const int ej = j - 1 + b;
      if (ej < 0 || ej >= d.ny) continue;
      for (int a = 0; a < 2; ++a) {
        const int ei = i - 1 + a;
        if (ei >= 0 && ei < d.nx) es += L.E[ei + d.nx * (ej + d.ny * ek)];
      }
    }
  }
  return es;
}

// the shared-memory view of tail level t (plan offsets; see tail_plan_smem)
__device__ __forceinline__ LevelView tail_view(const TailPlan& p, float* smem, int t) {
  LevelView V;
  V.d = p.d[t];
  V.nn = (V.d.nx + 1) * (V.d.ny + 1) * (V.d.nz + 1);
  float* base = smem + p.off[t];
  const int v = 3 * V.nn;
  V.b = base;
  V.x = base + v;
  V.r = base + 2 * v;
  V.dv[0] = base + 3 * v;
  V.dv[1] = base + 4 * v;
  V.E = base + 5 * v;
  return V;
}

__device__ __forceinline__ float tail_dinv(float kdiag, float esum) {
  return esum > 0.f ? jacobi_rcp(kdiag * esum) : 1.0f;
}

}  // namespace

__global__ void __launch_bounds__(kTailThreads)
    k_vcycle_tail(const __grid_constant__ TailPlan p, const __grid_constant__ K0<float> k0,
                  const int* __restrict__ done, const DSel S) {
  pdl_start();
  const long long off = S.off(blockIdx.y);
  done = bshift(done, off);
  if (*done) return;  // uniform over the CTA
  extern __shared__ __align__(16) float tail_smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  double* bd = reinterpret_cast<double*>(tail_smem + p.off[p.nt + 1]);
  // inputs: the moduli of the smoothed levels, the right-hand side of level l0
  for (int t = 0; t < p.nt; ++t) {
    const LevelView V = tail_view(p, tail_smem, t);
    const Dims& d = V.d;
    const float* Eg = bshift(p.E[t], off);
    const int ne = d.nx * d.ny * d.nz;
    for (int e = tid; e < ne; e += nth) {
      int i, j, k;
      unflatten3(e, d.nx, d.ny, i, j, k);
      V.E[e] = Eg[d.elem(i, j, k)];
    }
  }
  {
    const LevelView V = tail_view(p, tail_smem, 0);
    const Dims& d = V.d;
    const float* bg = bshift(p.b, off);
    for (int n = tid; n < V.nn; n += nth) {
      int i, j, k;
      node_ijk(d, n, i, j, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) V.b[c * V.nn + n] = bg[c * d.comp + d.node(i, j, k)];
    }
  }
  __syncthreads();
  const int m = p.degree;
  // ------------------------------------------------------------ down
  for (int t = 0; t < p.nt; ++t) {
    const LevelView V = tail_view(p, tail_smem, t);
    const Dims& d = V.d;
    const int sn = V.nn;
    // r = b, d0 = D^-1 b / theta, x = d0
    for (int n = tid; n < sn; n += nth) {
      int i, j, k;
      node_ijk(d, n, i, j, k);
      const float dv = tail_dinv(p.kdiag, node_esum(V, i, j, k));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float bv = V.b[c * sn + n];
        const float d0 = dv * bv * p.inv_theta;
        V.r[c * sn + n] = bv;
        V.dv[0][c * sn + n] = d0;
        V.x[c * sn + n] = d0;
      }
    }
    __syncthreads();
    for (int q = 1; q < m; ++q) {  // r -= A d; d' = c1 d + c2 D^-1 r; x += d'
      const float* din = V.dv[(q - 1) & 1];
      float* dout = V.dv[q & 1];
      for (int n = tid; n < sn; n += nth) {
        int i, j, k;
        node_ijk(d, n, i, j, k);
        float acc[3], es;
        gather_apply(V, din, k0, i, j, k, acc, es);
        const float dv = tail_dinv(p.kdiag, es);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int o = c * sn + n;
          const float Ad = d.fixed(c, i, j, k) ? 0.f : acc[c];
          const float rn = V.r[o] - Ad;
          const float dd = fmaf(p.c1[q], din[o], p.c2[q] * dv * rn);
          V.r[o] = rn;
          dout[o] = dd;
          V.x[o] += dd;
        }
      }
      __syncthreads();
    }
    {  // r -= A d_{m-1}
      const float* din = V.dv[(m - 1) & 1];
      for (int n = tid; n < sn; n += nth) {
        int i, j, k;
        node_ijk(d, n, i, j, k);
        float acc[3], es;
        gather_apply(V, din, k0, i, j, k, acc, es);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (!d.fixed(c, i, j, k)) V.r[c * sn + n] -= acc[c];
      }
    }
    __syncthreads();
    // b_{t+1} = P^T r (trilinear weights 1 and 1/2 per axis offset), 0 on fixed DOFs
    const LevelView C = tail_view(p, tail_smem, t + 1);
    const Dims& dc = C.d;
    for (int n = tid; n < C.nn; n += nth) {
      int I, J, K;
      node_ijk(dc, n, I, J, K);
      float sacc[3] = {0.f, 0.f, 0.f};
      for (int dk = -1; dk <= 1; ++dk) {
        const int k = 2 * K + dk;
        if (k < 0 || k > d.nz) continue;
        const float wk = dk ? 0.5f : 1.0f;
        for (int dj = -1; dj <= 1; ++dj) {
          const int j = 2 * J + dj;
          if (j < 0 || j > d.ny) continue;
          const float wjk = wk * (dj ? 0.5f : 1.0f);
          for (int di = -1; di <= 1; ++di) {
            const int i = 2 * I + di;
            if (i < 0 || i > d.nx) continue;
            const float wt = wjk * (di ? 0.5f : 1.0f);
            const int o = i + (d.nx + 1) * (j + (d.ny + 1) * k);
#pragma unroll
            for (int c = 0; c < 3; ++c) sacc[c] = fmaf(wt, V.r[c * sn + o], sacc[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) C.b[c * C.nn + n] = dc.fixed(c, I, J, K) ? 0.0f : sacc[c];
    }
    __syncthreads();
  }
  // ------------------------------------------------------------ coarsest: x = A^-1 b (FP64)
  {
    const LevelView C = tail_view(p, tail_smem, p.nt);
    const Dims& dc = C.d;
    for (int n = tid; n < C.nn; n += nth)
#pragma unroll
      for (int c = 0; c < 3; ++c) bd[3 * n + c] = (double)C.b[c * C.nn + n];
    __syncthreads();
    const double* A = bshift(p.Ainv, off);
    const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
    for (int row = warp; row < p.nc; row += nw) {
      const double* a = A + (long long)row * p.nc;
      double s = 0.0;
      for (int q = lane; q < p.nc; q += 32) s = fma(a[q], bd[q], s);
      s = warp_sum(s);
      if (lane == 0) {
        const int n = row / 3, c = row - 3 * n;
        int i, j, k;
        node_ijk(dc, n, i, j, k);
        C.x[c * C.nn + n] = dc.fixed(c, i, j, k) ? 0.0f : (float)s;
      }
    }
    __syncthreads();
  }
  // ------------------------------------------------------------ up
  for (int t = p.nt - 1; t >= 0; --t) {
    const LevelView V = tail_view(p, tail_smem, t);
    const LevelView C = tail_view(p, tail_smem, t + 1);
    const Dims& d = V.d;
    const Dims& dc = C.d;
    const int sn = V.nn;
    // x += P x_c on free DOFs (2 x 2 x 2 coarse nodes, weights 1 and 0 or 1/2 and 1/2)
    for (int n = tid; n < sn; n += nth) {
      int i, j, k;
      node_ijk(d, n, i, j, k);
      const int i0 = i >> 1, j0 = j >> 1, k0n = k >> 1;
      const int ci[2] = {i0, min(i0 + 1, dc.nx)}, cj[2] = {j0, min(j0 + 1, dc.ny)},
                ck[2] = {k0n, min(k0n + 1, dc.nz)};
      const float wi[2] = {(i & 1) ? 0.5f : 1.0f, (i & 1) ? 0.5f : 0.0f};
      const float wj[2] = {(j & 1) ? 0.5f : 1.0f, (j & 1) ? 0.5f : 0.0f};
      const float wk[2] = {(k & 1) ? 0.5f : 1.0f, (k & 1) ? 0.5f : 0.0f};
      float sacc[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
          for (int a2 = 0; a2 < 2; ++a2) {
            const int o = ci[a2] + (dc.nx + 1) * (cj[b2] + (dc.ny + 1) * ck[c2]);
            const float wt = wi[a2] * wj[b2] * wk[c2];
#pragma unroll
            for (int c = 0; c < 3; ++c) sacc[c] = fmaf(wt, C.x[c * C.nn + o], sacc[c]);
          }
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (!d.fixed(c, i, j, k)) V.x[c * sn + n] += sacc[c];
    }
    __syncthreads();
    // r = b - A x (0 on fixed DOFs), d0 = D^-1 r / theta
    for (int n = tid; n < sn; n += nth) {
      int i, j, k;
      node_ijk(d, n, i, j, k);
      float acc[3], es;
      gather_apply(V, V.x, k0, i, j, k, acc, es);
      const float dv = tail_dinv(p.kdiag, es);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int o = c * sn + n;
        const float rr = d.fixed(c, i, j, k) ? 0.0f : (V.b[o] - acc[c]);
        V.r[o] = rr;
        V.dv[0][o] = dv * rr * p.inv_theta;
      }
    }
    __syncthreads();
    for (int q = 1; q < m; ++q) {  // as on the way down; the first step also adds d0 to x
      const float* din = V.dv[(q - 1) & 1];
      float* dout = V.dv[q & 1];
      for (int n = tid; n < sn; n += nth) {
        int i, j, k;
        node_ijk(d, n, i, j, k);
        float acc[3], es;
        gather_apply(V, din, k0, i, j, k, acc, es);
        const float dv = tail_dinv(p.kdiag, es);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int o = c * sn + n;
          const float Ad = d.fixed(c, i, j, k) ? 0.f : acc[c];
          const float rn = V.r[o] - Ad;
          const float dd = fmaf(p.c1[q], din[o], p.c2[q] * dv * rn);
          V.r[o] = rn;
          dout[o] = dd;
          V.x[o] += (q == 1) ? (dd + din[o]) : dd;
        }
      }
      __syncthreads();
    }
    if (m == 1) {
      for (int o = tid; o < 3 * sn; o += nth) V.x[o] += V.dv[0][o];
      __syncthreads();
    }
  }
  // output: x of level l0
  {
    const LevelView V = tail_view(p, tail_smem, 0);
    const Dims& d = V.d;
    float* xg = bshift(p.x, off);
    for (int n = tid; n < V.nn; n += nth) {
      int i, j, k;
      node_ijk(d, n, i, j, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) xg[c * d.comp + d.node(i, j, k)] = V.x[c * V.nn + n];
    }
  }
}

// Shared-memory plan of the tail from level l0: per smoothed level 5 node
// vectors and the dense moduli, then the coarsest level's b and x and
// (8-byte aligned) its FP64 right-hand side.
size_t tail_plan_smem(const std::vector<Dims>& lv, int l0, int* offsets) {
  size_t f = 0;
  const int nl = (int)lv.size();
  for (int l = l0; l < nl; ++l) {
    if (offsets) offsets[l - l0] = (int)f;
    const Dims& d = lv[l];
    const size_t nn = (size_t)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
    if (l < nl - 1)
      f += 5 * 3 * nn + (size_t)d.nx * d.ny * d.nz;
    else
      f += 5 * 3 * nn;  // the same view (b, x, r, d0, d1); only b and x are used
    f = (f + 3) / 4 * 4;  // 16-byte boundaries
  }
  if (offsets) offsets[nl - l0] = (int)f;
  const Dims& dc = lv[nl - 1];
  f += 2 * 3 * (size_t)(dc.nx + 1) * (dc.ny + 1) * (dc.nz + 1);  // nc doubles
  return f * sizeof(float);
}

int tail_first_level(const std::vector<Dims>& lv, int degree) {
  const int nl = (int)lv.size();
  if (degree < 1 || degree > kTailMaxDeg) return -1;
  for (int l0 = 1; l0 < nl - 1; ++l0) {
    if (nl - 1 - l0 > kTailMaxLevels) continue;
    const Dims& d = lv[l0];
    if ((long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1) > kTailMaxNodes) continue;
    if (tail_plan_smem(lv, l0, nullptr) <= kTailMaxSmem) return l0;
  }
  return -1;
}

cudaError_t launch_vcycle_tail(const TailPlan& p, size_t smem, const K0<float>& k0,
                               const int* done, cudaStream_t s, const Bat& bt) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_vcycle_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailMaxSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_vcycle_tail, dim3(1, bt.nb), dim3(kTailThreads), smem, s, p, k0, done,
                    bt.sel());
}

}  // namespace topo
