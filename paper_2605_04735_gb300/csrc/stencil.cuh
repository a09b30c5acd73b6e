// Matrix-free application of the SIMP stiffness operator (Sec. 2.1.1,
// Eq. (2): K(rho) = sum_e E_e k0, E_e from Eq. (1)) as a node-centric gather
// with no atomics, with a pluggable per-node epilogue.
//
// FP32 kernel (k_stencil): each thread owns a column of nodes (i, j, kb..ke)
// and marches up in z, holding the 3x3x3 node neighbourhood (3 components)
// and the 2x2x2 surrounding element moduli in registers; per z step it loads
// one new node plane (9 nodes) and element plane (4 elements).  For node n
//     (K x)_n = sum_{e owns n} E_e * (k0[row block of n in e] . x_e),
// 8 elements x 72 FMAs, k0 read as constant-bank operands (compile-time
// indices into a __grid_constant__ parameter).
// FP64 kernel (k_stencil_direct): same sum, no register window (81 doubles
// would spill); the FP64 pipe bounds it, not the loads.
//
// The epilogue receives (K x)_n (before any masking) and x_n and decides what
// to write; it returns the node's contribution to an optional reduction.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tma.cuh"

namespace topo {

// local node number of the corner at offsets (dx, dy, dz) in {0,1}^3
__host__ __device__ constexpr int lidx(int dx, int dy, int dz) {
  return 4 * dz + (dy ? (dx ? 2 : 3) : (dx ? 1 : 0));
}

constexpr int kStencilBX = 32;
constexpr int kStencilBY = 8;

template <typename T, class Epi>
__global__ void __launch_bounds__(kStencilBX* kStencilBY)
    k_stencil(const T* __restrict__ x, const T* __restrict__ E, const Dims d,
              const __grid_constant__ K0<T> k0, const Epi epi, const Red red, const int zchunk,
              const int* __restrict__ done) {
  if (done != nullptr && *done) return;  // uniform over the grid
  const int i = blockIdx.x * kStencilBX + threadIdx.x;
  const int j = blockIdx.y * kStencilBY + threadIdx.y;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool act = (i <= d.nx) && (j <= d.ny);
  T part = T(0);
  if (act) {
    const long long ps = d.plane_stride();
    const long long eps = d.eplane();
    const long long cs = d.comp;
    T w[3][3][3][3];  // w[z][y][x][c]: node (i-1+x, j-1+y, k-1+z)
    T e[2][2][2];     // e[z][y][x]: element (i-1+x, j-1+y, k-1+z)
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
      const long long np = nb + (long long)(k - kb + 2) * ps;   // node plane k+1
      const long long ep = eb + (long long)(k - kb + 1) * eps;  // element plane k
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

      // Every row of k0 sums to zero per displacement component (a rigid
      // translation is stress-free), so k0 x_e = k0 (x_e - 1 (x) x_n) for the
      // owning node n.  Gathering the differences x_m - x_n keeps FP32 from
      // cancelling large rigid displacements against each other, and the
      // centre terms vanish (72 FMAs fewer, 78 subtractions more).
      const T ctr[3] = {w[1][1][1][0], w[1][1][1][1], w[1][1][1][2]};
      T t[3][3][3][3];  // shifted window, formed once per node (each entry feeds up to 8 elements)
#pragma unroll
      for (int zz = 0; zz < 3; ++zz)
#pragma unroll
        for (int yy = 0; yy < 3; ++yy)
#pragma unroll
          for (int xx = 0; xx < 3; ++xx)
#pragma unroll
            for (int c = 0; c < 3; ++c) t[zz][yy][xx][c] = w[zz][yy][xx][c] - ctr[c];
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
                  if (a + dx == 1 && b + dy == 1 && c + dz == 1) continue;  // the node itself
                  const int lm = lidx(dx, dy, dz);
#pragma unroll
                  for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                      s[r] = fma(k0.v[(3 * ln + r) * 24 + 3 * lm + q],
                                 t[c + dz][b + dy][a + dx][q], s[r]);
                }
            const T ee = e[c][b][a];
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[r] = fma(ee, s[r], acc[r]);
          }
      part += epi_one(epi, i, j, k, d.node(i, j, k), acc, ctr, d);
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
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red);
  }
}

template <typename T, class Epi>
__global__ void __launch_bounds__(kStencilBX* kStencilBY)
    k_stencil_direct(const T* __restrict__ x, const T* __restrict__ E, const Dims d,
                     const __grid_constant__ K0<T> k0, const Epi epi, const Red red,
                     const int zchunk, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int i = blockIdx.x * kStencilBX + threadIdx.x;
  const int j = blockIdx.y * kStencilBY + threadIdx.y;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool act = (i <= d.nx) && (j <= d.ny);
  T part = T(0);
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
    const T ctr[3] = {x[o], x[cs + o], x[2 * cs + o]};
    part += epi_one(epi, i, j, k, o, acc, ctr, d);
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red);
  }
}


// ---------------------------------------------------------------------------
// TMA-staged FP32 variant.  A CTA owns a 32 x 8 tile of node columns and a
// z range; node planes (36 x 10 halo box, 3 components) and element planes
// (36 x 9 box) stream through a kTmaStages-deep shared-memory ring, each
// stage filled by one elected thread with cp.async.bulk.tensor and
// completed on an mbarrier.  Threads copy their 3x3 node and 2x2 element
// neighbourhoods from the stage into the same register window as above, the
// slot is refilled right away (kTmaStages - 1 planes ahead of the compute),
// and the 576-FMA gather runs from registers.  Box starts are multiples of 4
// floats (16 bytes) because of the one-element ghost layer: node i0-1 and
// element i0-1 are both stored at x = i0.
constexpr int kTmaStages = 4;
constexpr int kBoxX = kStencilBX + 4;        // 36 >= 32 + 2 halo, 144 bytes
constexpr int kBoxYN = kStencilBY + 2;       // node rows
constexpr int kBoxYE = kStencilBY + 1;       // element rows
constexpr int kNodeStage = kBoxX * kBoxYN * 3;  // floats
constexpr int kElemStage = kBoxX * kBoxYE;      // floats
constexpr uint32_t kStageTx = (uint32_t)(kNodeStage + kElemStage) * 4u;

struct __align__(128) TmaStage {
  float node[kNodeStage];
  alignas(128) float elem[kElemStage];
};

template <class Epi>
__global__ void __launch_bounds__(kStencilBX* kStencilBY)
    k_stencil_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap emap,
                  const Dims d, const __grid_constant__ K0<float> k0, const Epi epi, const Red red,
                  const int zchunk, const int* __restrict__ done, int* __restrict__ errflag) {
  if (done != nullptr && *done) return;  // uniform over the grid
  __shared__ TmaStage st[kTmaStages];
  __shared__ uint64_t bar[kTmaStages];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kStencilBX + tx;
  const int i0 = blockIdx.x * kStencilBX, j0 = blockIdx.y * kStencilBY;
  const int i = i0 + tx, j = j0 + ty;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const int nst = (ke - kb) + 2;  // stage s: node plane kb-1+s, element plane kb-2+s
  const bool act = (i <= d.nx) && (j <= d.ny);
  if (tid == 0) {
    for (int q = 0; q < kTmaStages; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
    tma_prefetch_desc(&xmap);
    tma_prefetch_desc(&emap);
  }
  __syncthreads();
  auto issue = [&](int s) {
    const int slot = s % kTmaStages;
    mbar_arrive_expect_tx(&bar[slot], kStageTx);
    // storage coordinates: +1 for the ghost layer in every direction
    tma_load_5d(st[slot].node, &xmap, &bar[slot], i0, j0, kb + s, 0, 0);
    tma_load_4d(st[slot].elem, &emap, &bar[slot], i0, j0, kb - 1 + s, 0);
  };
  if (tid == 0)
    for (int s = 0; s < kTmaStages && s < nst; ++s) issue(s);
  auto release = [&](int s) {
    __syncthreads();  // every thread has copied stage s out of its slot
    if (tid == 0 && s + kTmaStages < nst) {
      // order the generic-proxy reads of the slot before the async-proxy refill
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(s + kTmaStages);
    }
  };
  float w[3][3][3][3];
  float e[2][2][2];
  auto read_nodes = [&](int s, int zslot) {
    const float* nd = st[s % kTmaStages].node;
#pragma unroll
    for (int yy = 0; yy < 3; ++yy)
#pragma unroll
      for (int xx = 0; xx < 3; ++xx)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          w[zslot][yy][xx][c] = nd[c * (kBoxX * kBoxYN) + (ty + yy) * kBoxX + tx + xx];
  };
  auto read_elems = [&](int s, int zslot) {
    const float* el = st[s % kTmaStages].elem;
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int xx = 0; xx < 2; ++xx) e[zslot][yy][xx] = el[(ty + yy) * kBoxX + tx + xx];
  };
  mbar_wait_bounded(&bar[0], 0, errflag);
  read_nodes(0, 0);
  release(0);
  mbar_wait_bounded(&bar[1 % kTmaStages], (1 / kTmaStages) & 1, errflag);
  read_nodes(1, 1);
  read_elems(1, 0);
  release(1);
  float part = 0.f;
  for (int k = kb; k < ke; ++k) {
    const int s = k - kb + 2;
    mbar_wait_bounded(&bar[s % kTmaStages], (uint32_t)((s / kTmaStages) & 1), errflag);
    // plain shared-memory loads of the stage (the ordering of the TMA write
    // before them is given by the mbarrier wait)
#pragma unroll
    for (int yy = 0; yy < 3; ++yy)
#pragma unroll
      for (int xx = 0; xx < 3; ++xx)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          w[2][yy][xx][c] =
              st[s % kTmaStages].node[c * (kBoxX * kBoxYN) + (ty + yy) * kBoxX + tx + xx];
#pragma unroll
    for (int yy = 0; yy < 2; ++yy)
#pragma unroll
      for (int xx = 0; xx < 2; ++xx)
        e[1][yy][xx] = st[s % kTmaStages].elem[(ty + yy) * kBoxX + tx + xx];
    release(s);
    if (act) {
      const float ctr[3] = {w[1][1][1][0], w[1][1][1][1], w[1][1][1][2]};
      float t[3][3][3][3];  // shifted window (see k_stencil)
#pragma unroll
      for (int zz = 0; zz < 3; ++zz)
#pragma unroll
        for (int yy = 0; yy < 3; ++yy)
#pragma unroll
          for (int xx = 0; xx < 3; ++xx)
#pragma unroll
            for (int c = 0; c < 3; ++c) t[zz][yy][xx][c] = w[zz][yy][xx][c] - ctr[c];
      float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            const int ln = lidx(1 - a, 1 - b, 1 - c);
            float sv[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
              for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                  if (a + dx == 1 && b + dy == 1 && c + dz == 1) continue;
                  const int lm = lidx(dx, dy, dz);
#pragma unroll
                  for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                      sv[r] = fmaf(k0.v[(3 * ln + r) * 24 + 3 * lm + q], t[c + dz][b + dy][a + dx][q],
                                   sv[r]);
                }
            const float ee = e[c][b][a];
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[r] = fmaf(ee, sv[r], acc[r]);
          }
      part += epi_one(epi, i, j, k, d.node(i, j, k), acc, ctr, d);
    }
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
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red);
  }
}

// host: tensor maps of a node vector (4-D: x, y, z, component) and of an
// element array (3-D) in the ghosted layout, cached by base address
bool stencil_maps(const float* x, const float* E, const Dims& d, CUtensorMap* xmap,
                  CUtensorMap* emap);

// z planes per thread: enough blocks for ~4 waves of 152 SMs at 2 resident
// blocks each, a 2-plane halo reload below ~15%, and at most kMaxPartials blocks
inline int stencil_zchunk(const Dims& d) {
  const long long xy = (long long)((d.nx + kStencilBX) / kStencilBX) * ((d.ny + kStencilBY) / kStencilBY);
  const int planes = d.nz + 1;
  int z = (int)((xy * planes) / (152 * 2 * 4));
  if (z < 2) z = 2;
  if (z > 32) z = 32;
  while (xy * ((planes + z - 1) / z) > kMaxPartials) ++z;
  return z;
}

template <typename T, class Epi>
cudaError_t launch_stencil(const T* x, const T* E, const Dims& d, const K0<T>& k0, const Epi& epi,
                           const Red& red, const int* done, int* errflag, cudaStream_t s) {
  const int z = stencil_zchunk(d);
  dim3 block(kStencilBX, kStencilBY, 1);
  dim3 grid((d.nx + kStencilBX) / kStencilBX, (d.ny + kStencilBY) / kStencilBY, (d.nz + z) / z);
  if constexpr (sizeof(T) == 8) {
    k_stencil_direct<T, Epi><<<grid, block, 0, s>>>(x, E, d, k0, epi, red, z, done);
  } else {
    CUtensorMap xm, em;
    if (stencil_maps(x, E, d, &xm, &em))
      k_stencil_tma<Epi><<<grid, block, 0, s>>>(xm, em, d, k0, epi, red, z, done, errflag);
    else  // grids too small for the TMA boxes: same arithmetic from plain loads
      k_stencil<T, Epi><<<grid, block, 0, s>>>(x, E, d, k0, epi, red, z, done);
  }
  return cudaGetLastError();
}

}  // namespace topo
