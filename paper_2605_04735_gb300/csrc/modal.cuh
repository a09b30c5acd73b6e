// Element-centric application of the SIMP stiffness operator in the modal
// (tensor-product Walsh-Hadamard) basis of the trilinear brick.
//
// For an element with nodal values u (3 components x 8 corners, corner
// b = dx + 2 dy + 4 dz), k0 u = H (K~ (H^T u)) with H[b][m] = (-1)^popcount(b & m)
// and K~ = H^T k0 H / 64.  Because the 1-D factors of k0 (mass, stiffness and
// mixed hat-function integrals) are diagonal or single off-diagonal in the
// (1,1)/(1,-1) basis, K~ has only 45 non-zeros: per component p a diagonal
// D[p][m] (m = 1..7; the constant mode is rigid translation) and, for q != p,
// one coupling C[p][q][m] between mode m and mode m ^ (1<<p) ^ (1<<q) when
// bits p and q of m differ.  An element then costs two 8-point transforms per
// component (24 add/sub each) plus 45 FMAs instead of the 576 of a dense
// 24x24 product; the values are shifted by corner 0 first so that large rigid
// displacements never meet in one FP32 sum.
//
// Work split (no atomics): a CTA is 32 x 8 threads; thread (tx, ty) owns the
// element column (x0-1+tx, y0-1+ty, *) and marches up in z, one element
// layer per step.  Its element's 8 nodal results are combined with its
// neighbours' as follows: the +x face goes to lane tx+1 by warp shuffle, the
// +y face to thread row ty+1 through a double-buffered shared-memory slot, and
// the +z face is carried in registers to the next layer.  Thread (tx, ty) with
// tx, ty >= 1 then holds the complete result of node (x0-1+tx, y0-1+ty, z)
// after layer z: a CTA owns a 31 x 7 tile of node columns, recomputing one
// halo element layer on its -x and -y sides.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tma.cuh"

namespace topo {

template <typename T>
struct ModalCoef {
  T D[3][8];     // diagonal of K~ per component and mode (mode 0 unused)
  T C[3][3][8];  // coupling of (p, m) with (q, m ^ (1<<p) ^ (1<<q)), bits p, q of m differ
};

// in-place 8-point Walsh-Hadamard transform: v[m] <- sum_b (-1)^{b.m} v[b]
template <typename T>
__device__ __forceinline__ void fwht8(T (&v)[8]) {
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (!(b & bit)) {
        const T a = v[b], c = v[b | bit];
        v[b] = a + c;
        v[b | bit] = a - c;
      }
}

// y = E k0 u for one element (u, y: [component][corner])
template <typename T>
__device__ __forceinline__ void modal_element(const T (&u)[3][8], T E, const ModalCoef<T>& kc,
                                              T (&y)[3][8]) {
  T uh[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uh[c][0] = T(0);
#pragma unroll
    for (int b = 1; b < 8; ++b) uh[c][b] = u[c][b] - u[c][0];
    fwht8(uh[c]);
#pragma unroll
    for (int m = 1; m < 8; ++m) uh[c][m] *= E;
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    y[p][0] = T(0);
#pragma unroll
    for (int m = 1; m < 8; ++m) {
      T acc = kc.D[p][m] * uh[p][m];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q == p) continue;
        if (((m >> p) & 1) == ((m >> q) & 1)) continue;
        acc = fma(kc.C[p][q][m], uh[q][m ^ (1 << p) ^ (1 << q)], acc);
      }
      y[p][m] = acc;
    }
    fwht8(y[p]);
  }
}

constexpr int kModalTX = 32, kModalTY = 8;
constexpr int kModalOwnX = kModalTX - 1, kModalOwnY = kModalTY - 1;
constexpr int kModalStages = 4;
constexpr int kMBoxX = 40;               // >= 3 (alignment slack) + 33 columns
constexpr int kMBoxNY = kModalTY + 1;    // node rows y0-1 .. y0+7
constexpr int kMBoxEY = kModalTY;        // element rows y0-1 .. y0+6
constexpr int kMNode = 3 * kMBoxNY * kMBoxX;
constexpr int kMElem = kMBoxEY * kMBoxX;
constexpr uint32_t kMStageTx = (uint32_t)(kMNode + kMElem) * 4u;

struct __align__(128) ModalStage {
  float node[kMNode];
  alignas(128) float elem[kMElem];
};

// Shared by both variants: combine one element layer's results into node
// results (x by shuffle, y through smem, z by the register carry) and run
// the epilogue for the completed node plane.
template <typename T, class Epi>
__device__ __forceinline__ T modal_combine(const T (&y)[3][8], T (&carry)[3],
                                           T (*xch)[kModalTX][6], int tx, int ty, int ex, int ey,
                                           int ez, bool emit, const T (&ctr)[3], const Dims& d,
                                           const Epi& epi) {
  // x: the +x face (odd corners) moves to lane tx+1
  T s[2][2][3];  // [dy][dz][c] for node column x = ex
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T right = y[c][1 + 2 * dy + 4 * dz];
        const T recv = __shfl_up_sync(0xffffffffu, right, 1);
        s[dy][dz][c] = y[c][2 * dy + 4 * dz] + (tx > 0 ? recv : T(0));
      }
  // y: the +y face goes to thread row ty+1 (double-buffered slot, one barrier)
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int c = 0; c < 3; ++c) xch[ty][tx][3 * dz + c] = s[1][dz][c];
  __syncthreads();
  T part = T(0);
  T bot[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T r0 = ty > 0 ? xch[ty - 1][tx][c] : T(0);
    const T r1 = ty > 0 ? xch[ty - 1][tx][3 + c] : T(0);
    bot[c] = s[0][0][c] + r0 + carry[c];  // node (ex, ey, ez) is complete
    carry[c] = s[0][1][c] + r1;           // node (ex, ey, ez+1) so far
  }
  if (emit) part = epi(ex, ey, ez, d.node(ex, ey, ez), bot, ctr, d);
  return part;
}

template <class Epi>
__global__ void __launch_bounds__(kModalTX* kModalTY)
    k_modal_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap emap,
                const Dims d, const __grid_constant__ ModalCoef<float> kc, const Epi epi,
                const Red red, const int zchunk, const int* __restrict__ done,
                int* __restrict__ errflag) {
  if (done != nullptr && *done) return;  // uniform over the grid
  __shared__ ModalStage st[kModalStages];
  __shared__ uint64_t bar[kModalStages];
  __shared__ float xch[2][kModalTY][kModalTX][6];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kModalTX + tx;
  const int x0 = blockIdx.x * kModalOwnX, y0 = blockIdx.y * kModalOwnY;
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const int bx = x0 & ~3;  // 16-byte aligned box start (storage x of node x0-1 is x0)
  const int ox = x0 - bx;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const int nst = (ke - kb) + 2;  // stage t: node plane kb-2+t+1, element layer kb-2+t
  if (tid == 0) {
    for (int q = 0; q < kModalStages; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
    tma_prefetch_desc(&xmap);
    tma_prefetch_desc(&emap);
  }
  __syncthreads();
  auto issue = [&](int t) {
    const int slot = t % kModalStages;
    mbar_arrive_expect_tx(&bar[slot], kMStageTx);
    tma_load_4d(st[slot].node, &xmap, &bar[slot], bx, y0, kb + t, 0);
    tma_load_3d(st[slot].elem, &emap, &bar[slot], bx, y0, kb - 1 + t);
  };
  if (tid == 0)
    for (int t = 0; t < kModalStages && t < nst; ++t) issue(t);
  const bool own = tx > 0 && ty > 0 && ex <= d.nx && ey <= d.ny;
  float bot[2][2][3], top[2][2][3];  // [dy][dx][c]
  float carry[3] = {0.f, 0.f, 0.f};
  float part = 0.f;  // this thread's nodes only (at most zchunk); widened to FP64 below
  for (int t = 0; t < nst; ++t) {
    const int slot = t % kModalStages;
    mbar_wait_bounded(&bar[slot], (uint32_t)((t / kModalStages) & 1), errflag);
    const float* nd = st[slot].node;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          top[dy][dx][c] = nd[c * (kMBoxNY * kMBoxX) + (ty + dy) * kMBoxX + ox + tx + dx];
    const float E = st[slot].elem[ty * kMBoxX + ox + tx];
    if (t == 0) {  // the first node plane only seeds the bottom face
      __syncthreads();
      if (tid == 0 && kModalStages < nst) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(kModalStages);
      }
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
          for (int c = 0; c < 3; ++c) bot[dy][dx][c] = top[dy][dx][c];
      continue;
    }
    float u[3][8], y[3][8];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            u[c][dx + 2 * dy + 4 * dz] = dz ? top[dy][dx][c] : bot[dy][dx][c];
    modal_element<float>(u, E, kc, y);
    const int ez = kb - 2 + t;
    const float ctr[3] = {bot[0][0][0], bot[0][0][1], bot[0][0][2]};
    // the barrier inside modal_combine also retires this stage's slot
    part += modal_combine<float, Epi>(y, carry, xch[t & 1], tx, ty, ex, ey, ez,
                                      own && t >= 2, ctr, d, epi);
    if (tid == 0 && t + kModalStages < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + kModalStages);
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) bot[dy][dx][c] = top[dy][dx][c];
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red);
  }
}

// Plain-load variant (FP64, and FP32 grids too small for the TMA boxes):
// same work split, inputs read with bounds checks from the ghosted arrays.
template <typename T, class Epi>
__global__ void __launch_bounds__(kModalTX* kModalTY)
    k_modal_plain(const T* __restrict__ x, const T* __restrict__ E, const Dims d,
                  const __grid_constant__ ModalCoef<T> kc, const Epi epi, const Red red,
                  const int zchunk, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ T xch[2][kModalTY][kModalTX][6];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * kModalOwnX, y0 = blockIdx.y * kModalOwnY;
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const int kb = blockIdx.z * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool own = tx > 0 && ty > 0 && ex <= d.nx && ey <= d.ny;
  auto node_val = [&](int i, int j, int k, int c) -> T {
    if (i > d.nx + 1 || j > d.ny + 1 || k > d.nz + 1) return T(0);  // beyond the ghost ring
    return __ldg(x + c * d.comp + d.node(i, j, k));
  };
  T bot[2][2][3], top[2][2][3];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
      for (int c = 0; c < 3; ++c) bot[dy][dx][c] = node_val(ex + dx, ey + dy, kb - 1, c);
  T carry[3] = {T(0), T(0), T(0)};
  T part = T(0);
  for (int ez = kb - 1; ez < ke; ++ez) {
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) top[dy][dx][c] = node_val(ex + dx, ey + dy, ez + 1, c);
    const T Ee = (ex <= d.nx && ey <= d.ny && ez <= d.nz) ? __ldg(E + d.elem(ex, ey, ez)) : T(0);
    T u[3][8], y[3][8];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            u[c][dx + 2 * dy + 4 * dz] = dz ? top[dy][dx][c] : bot[dy][dx][c];
    modal_element<T>(u, Ee, kc, y);
    const T ctr[3] = {bot[0][0][0], bot[0][0][1], bot[0][0][2]};
    part += modal_combine<T, Epi>(y, carry, xch[(ez - kb + 1) & 1], tx, ty, ex, ey, ez,
                                  own && ez >= kb, ctr, d, epi);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) bot[dy][dx][c] = top[dy][dx][c];
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red);
  }
}

// z planes per CTA for the modal kernels: a few waves over 152 SMs, a one-
// layer warm-up below ~10%, and no more CTAs than partial-sum slots
inline int modal_zchunk(const Dims& d) {
  const long long xy = (long long)((d.nx + kModalOwnX) / kModalOwnX) *
                       ((d.ny + kModalOwnY) / kModalOwnY);
  const int planes = d.nz + 1;
  int z = (int)((xy * planes) / (152 * 2 * 4));
  if (z < 4) z = 4;
  if (z > 32) z = 32;
  while (xy * ((planes + z - 1) / z) > kMaxPartials) ++z;
  return z;
}

bool modal_maps(const float* x, const float* E, const Dims& d, CUtensorMap* xmap,
                CUtensorMap* emap);

template <typename T, class Epi>
cudaError_t launch_modal(const T* x, const T* E, const Dims& d, const ModalCoef<T>& kc,
                         const Epi& epi, const Red& red, const int* done, int* errflag,
                         cudaStream_t s) {
  const int z = modal_zchunk(d);
  dim3 block(kModalTX, kModalTY, 1);
  dim3 grid((d.nx + kModalOwnX) / kModalOwnX, (d.ny + kModalOwnY) / kModalOwnY,
            (d.nz + z) / z);
  if constexpr (sizeof(T) == 4) {
    CUtensorMap xm, em;
    if (modal_maps(x, E, d, &xm, &em)) {
      k_modal_tma<Epi><<<grid, block, 0, s>>>(xm, em, d, kc, epi, red, z, done, errflag);
      return cudaGetLastError();
    }
  }
  k_modal_plain<T, Epi><<<grid, block, 0, s>>>(x, E, d, kc, epi, red, z, done);
  return cudaGetLastError();
}

}  // namespace topo
