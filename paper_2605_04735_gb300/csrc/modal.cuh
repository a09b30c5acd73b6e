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
// Work split (no atomics): a CTA is kModalTX x kModalTY threads (16 x 12 by
// default, see below); thread (tx, ty) owns the
// element column (x0-1+tx, y0-1+ty, *) and marches up in z, one element
// layer per step.  The transform is split into its x-y part (per node plane)
// and its z part (per element): the x-y transform of a node plane is computed
// once and shared by the element below and the element above it, and on the
// way back the two elements' contributions to a node plane are summed in the
// x-y modal domain before one inverse x-y transform.  The plane's four
// corner results are then combined with the neighbours': the +x corners go
// to lane tx+1 by warp shuffle and the +y corner to thread row ty+1 through a
// double-buffered shared-memory slot.  Thread (tx, ty) with tx, ty >= 1 then
// holds the complete result of node (x0-1+tx, y0-1+ty, z): a CTA owns a
// (kModalTX-1) x (kModalTY-1) tile of node columns, recomputing one halo
// element layer on its -x and -y sides.  The K~ product runs on the
// unscaled displacement; E multiplies the element's two z faces of the
// result.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace topo {

// The FP32 one-column kernels march with components 0 and 1 packed
// (ModalColumnP: fewer issued instructions); 0 keeps the scalar march of
// modal_layer for comparison.
#ifndef TOPO_MODAL_PACKED
#define TOPO_MODAL_PACKED 1
#endif

template <typename T>
struct ModalCoef {
  T D[3][8];     // diagonal of K~ per component and mode (mode 0 unused)
  T C[3][3][8];  // coupling of (p, m) with (q, m ^ (1<<p) ^ (1<<q)), bits p, q of m differ
  T kdiag;       // every diagonal entry of k0 (the cube's symmetry makes them equal)
  int form;  // FP32 kernel form: 0 automatic, 1 one column per thread, 2 two columns (packed),
             // 3 tensor cores, 4 one column per thread with the x tiles in a cluster
};

// a * b + c (overloaded for the double-word type)
template <typename T>
__device__ __forceinline__ T fmadd(T a, T b, T c) {
  return fma(a, b, c);
}

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

// 4-point (x-y) Walsh-Hadamard transform, corner index dx + 2 dy
template <typename T>
__device__ __forceinline__ void fwht4(T (&v)[4]) {
  T a = v[0] + v[1], b = v[0] - v[1], c = v[2] + v[3], e = v[2] - v[3];
  v[0] = a + c;
  v[1] = b + e;
  v[2] = a - c;
  v[3] = b - e;
}

// Per-thread state of the z march (see the work split above).
template <typename T>
struct ModalColumn {
  T bxy[3][4];   // x-y transform of the bottom node plane, shifted by ref
  T ref[3];      // raw displacement of node (ex, ey, ez): the element's corner 0
  T carry[3][4]; // z-upper half of the previous element's result (x-y modal)
};

// start of the march: node plane kb-1 (raw corner values [dy][dx][c])
template <typename T>
__device__ __forceinline__ void modal_seed(ModalColumn<T>& col, const T (&raw)[2][2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    col.ref[c] = raw[0][0][c];
    T v[4] = {T(0), raw[0][1][c] - col.ref[c], raw[1][0][c] - col.ref[c],
              raw[1][1][c] - col.ref[c]};
    fwht4(v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      col.bxy[c][q] = v[q];
      col.carry[c][q] = T(0);
    }
  }
}

// One element layer: top node plane raw values in, the finished result of
// node plane ez (x-y corners [c][dx + 2 dy], before the neighbour exchange)
// out.  ctr receives the raw displacement of node (ex, ey, ez).  The modal
// product runs on the unscaled displacement (E multiplies the two z faces of
// the result), so `dot` is the element's strain energy
// (u_e - u_0)^T k0 (u_e - u_0) itself.
template <typename T>
__device__ __forceinline__ void modal_layer(ModalColumn<T>& col, const T (&top)[2][2][3], T E,
                                           const ModalCoef<T>& kc, T (&plane)[3][4],
                                           T (&ctr)[3], T* dot = nullptr) {
  T uh[3][8];  // [c][0], the rigid mode, is never formed (no K~ entry touches it)
  T txy[3][4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ctr[c] = col.ref[c];
    T v[4] = {top[0][0][c] - col.ref[c], top[0][1][c] - col.ref[c], top[1][0][c] - col.ref[c],
              top[1][1][c] - col.ref[c]};
    fwht4(v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      txy[c][q] = v[q];
      if (q > 0) uh[c][q] = col.bxy[c][q] + v[q];  // z mode 0
      uh[c][q + 4] = col.bxy[c][q] - v[q];         // z mode 1
    }
  }
  T yh[3][8];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
#pragma unroll
    for (int m = 1; m < 8; ++m) {
      T acc = kc.D[p][m] * uh[p][m];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q == p) continue;
        if (((m >> p) & 1) == ((m >> q) & 1)) continue;
        acc = fmadd(kc.C[p][q][m], uh[q][m ^ (1 << p) ^ (1 << q)], acc);
      }
      yh[p][m] = acc;
    }
  }
  if (dot) {  // uh . K~ uh = (u_e - u_0)^T k0 (u_e - u_0)
    T e = T(0);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int m = 1; m < 8; ++m) e = fmadd(uh[p][m], yh[p][m], e);
    *dot = e;
  }
  const T nE = -E;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // bottom face E (yh_q + yh_q+4) plus the previous element's top face;
    // this element's top face E (yh_q - yh_q+4) is carried up (yh_0 = 0)
    T w[4];
    w[0] = fmadd(E, yh[c][4], col.carry[c][0]);
    col.carry[c][0] = nE * yh[c][4];
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      w[q] = fmadd(E, yh[c][q] + yh[c][q + 4], col.carry[c][q]);
      col.carry[c][q] = E * (yh[c][q] - yh[c][q + 4]);
    }
    fwht4(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) plane[c][q] = w[q];
    // the top plane becomes the next bottom plane, re-referenced to its corner 0
    const T nref = top[0][0][c];
    col.bxy[c][0] = fmadd(T(4), col.ref[c] - nref, txy[c][0]);
#pragma unroll
    for (int q = 1; q < 4; ++q) col.bxy[c][q] = txy[c][q];
    col.ref[c] = nref;
  }
}

// Packed two-wide FP32 arithmetic (add/sub/mul/fma .f32x2, sm_100+): each
// half rounds exactly as the scalar instruction does, so a computation moved
// onto pairs keeps every bit of its scalar result.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
        "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}

// in-place 4-point (x-y) Walsh-Hadamard transform on pairs
__device__ __forceinline__ void pfwht4(float2 (&v)[4]) {
  const float2 a = padd(v[0], v[1]), b = psub(v[0], v[1]);
  const float2 c = padd(v[2], v[3]), e = psub(v[2], v[3]);
  v[0] = padd(a, c);
  v[1] = padd(b, e);
  v[2] = psub(a, c);
  v[3] = psub(b, e);
}

// The FP32 z march with components 0 and 1 of every per-component quantity
// held as one pair (.x = component 0, .y = component 1) and component 2 as a
// scalar: the shift, the x-y and z transforms, the face sums with E and the
// inverse transform of components 0 and 1 then issue as one packed
// instruction each.  The operations and their order are modal_layer's; the
// K~ product stays scalar, its operands read from the halves.  The results
// agree with modal_layer<float> to FP32 rounding, not to the bit: there the
// compiler may fuse the lone product of mode 7 (no coupling term) into the
// face sums, which the packed sums do not.
struct ModalColumnP {
  float2 bxy01[4];
  float bxy2[4];
  float2 ref01;
  float ref2;
  float2 carry01[4];
  float carry2[4];
};

__device__ __forceinline__ void modal_seed_p(ModalColumnP& col, const float (&raw)[2][2][3]) {
  col.ref01 = make_float2(raw[0][0][0], raw[0][0][1]);
  col.ref2 = raw[0][0][2];
  float2 v[4] = {make_float2(0.f, 0.f),
                 psub(make_float2(raw[0][1][0], raw[0][1][1]), col.ref01),
                 psub(make_float2(raw[1][0][0], raw[1][0][1]), col.ref01),
                 psub(make_float2(raw[1][1][0], raw[1][1][1]), col.ref01)};
  pfwht4(v);
  float u[4] = {0.f, raw[0][1][2] - col.ref2, raw[1][0][2] - col.ref2, raw[1][1][2] - col.ref2};
  fwht4(u);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    col.bxy01[q] = v[q];
    col.bxy2[q] = u[q];
    col.carry01[q] = make_float2(0.f, 0.f);
    col.carry2[q] = 0.f;
  }
}

__device__ __forceinline__ void modal_layer_p(ModalColumnP& col, const float (&top)[2][2][3],
                                              float E, const ModalCoef<float>& kc,
                                              float (&plane)[3][4], float (&ctr)[3]) {
  // x-y transform of the top plane (shifted by corner 0) and the z butterfly
  float2 uh01[8];  // [m] = (component 0, component 1) of mode m; [0] never formed
  float uh2[8];
  float2 t01[4];
  float t2[4];
  {
    const float2 r = col.ref01;
    ctr[0] = r.x;
    ctr[1] = r.y;
    ctr[2] = col.ref2;
    t01[0] = psub(make_float2(top[0][0][0], top[0][0][1]), r);
    t01[1] = psub(make_float2(top[0][1][0], top[0][1][1]), r);
    t01[2] = psub(make_float2(top[1][0][0], top[1][0][1]), r);
    t01[3] = psub(make_float2(top[1][1][0], top[1][1][1]), r);
    pfwht4(t01);
    t2[0] = top[0][0][2] - col.ref2;
    t2[1] = top[0][1][2] - col.ref2;
    t2[2] = top[1][0][2] - col.ref2;
    t2[3] = top[1][1][2] - col.ref2;
    fwht4(t2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q > 0) {
        uh01[q] = padd(col.bxy01[q], t01[q]);
        uh2[q] = col.bxy2[q] + t2[q];
      }
      uh01[q + 4] = psub(col.bxy01[q], t01[q]);
      uh2[q + 4] = col.bxy2[q] - t2[q];
    }
  }
  // the 45 entries of K~ (scalar; components 0 and 1 land in one pair)
  auto uh = [&](int c, int m) -> float { return c == 0 ? uh01[m].x : (c == 1 ? uh01[m].y : uh2[m]); };
  float2 yh01[8];
  float yh2[8];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
#pragma unroll
    for (int m = 1; m < 8; ++m) {
      float acc = kc.D[p][m] * uh(p, m);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q == p) continue;
        if (((m >> p) & 1) == ((m >> q) & 1)) continue;
        acc = fmaf(kc.C[p][q][m], uh(q, m ^ (1 << p) ^ (1 << q)), acc);
      }
      if (p == 0)
        yh01[m].x = acc;
      else if (p == 1)
        yh01[m].y = acc;
      else
        yh2[m] = acc;
    }
  }
  // E on the two z faces, the previous element's top face, inverse x-y transform
  const float nE = -E;
  {
    const float2 E2 = make_float2(E, E), nE2 = make_float2(nE, nE);
    float2 w[4];
    w[0] = pfma(E2, yh01[4], col.carry01[0]);
    col.carry01[0] = pmul(nE2, yh01[4]);
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      w[q] = pfma(E2, padd(yh01[q], yh01[q + 4]), col.carry01[q]);
      col.carry01[q] = pmul(E2, psub(yh01[q], yh01[q + 4]));
    }
    pfwht4(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      plane[0][q] = w[q].x;
      plane[1][q] = w[q].y;
    }
    const float2 nref = make_float2(top[0][0][0], top[0][0][1]);
    col.bxy01[0] = pfma(make_float2(4.f, 4.f), psub(col.ref01, nref), t01[0]);
#pragma unroll
    for (int q = 1; q < 4; ++q) col.bxy01[q] = t01[q];
    col.ref01 = nref;
  }
  {
    float w[4];
    w[0] = fmaf(E, yh2[4], col.carry2[0]);
    col.carry2[0] = nE * yh2[4];
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      w[q] = fmaf(E, yh2[q] + yh2[q + 4], col.carry2[q]);
      col.carry2[q] = E * (yh2[q] - yh2[q + 4]);
    }
    fwht4(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) plane[2][q] = w[q];
    const float nref = top[0][0][2];
    col.bxy2[0] = fmaf(4.f, col.ref2 - nref, t2[0]);
#pragma unroll
    for (int q = 1; q < 4; ++q) col.bxy2[q] = t2[q];
    col.ref2 = nref;
  }
}

// The z march of the one-column kernels: the packed form for FP32 (every
// FP32 one-column kernel, TMA-staged or plain, so that they agree to the
// bit), the scalar template for FP64 and the double-word type.
template <typename T>
using MarchColumn = typename std::conditional<TOPO_MODAL_PACKED && std::is_same<T, float>::value,
                                              ModalColumnP, ModalColumn<T>>::type;
template <typename T>
__device__ __forceinline__ void march_seed(ModalColumn<T>& col, const T (&raw)[2][2][3]) {
  modal_seed<T>(col, raw);
}
__device__ __forceinline__ void march_seed(ModalColumnP& col, const float (&raw)[2][2][3]) {
  modal_seed_p(col, raw);
}
template <typename T>
__device__ __forceinline__ void march_layer(ModalColumn<T>& col, const T (&top)[2][2][3], T E,
                                            const ModalCoef<T>& kc, T (&plane)[3][4],
                                            T (&ctr)[3], T* dot = nullptr) {
  modal_layer<T>(col, top, E, kc, plane, ctr, dot);
}
// (the FP32 kernels form no element energies: `dot` is never requested)
__device__ __forceinline__ void march_layer(ModalColumnP& col, const float (&top)[2][2][3],
                                            float E, const ModalCoef<float>& kc,
                                            float (&plane)[3][4], float (&ctr)[3],
                                            float* = nullptr) {
  modal_layer_p(col, top, E, kc, plane, ctr);
}

// the value of lane - 1 (overloaded for the double-word type)
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) {
  return __shfl_up_sync(0xffffffffu, v, 1);
}

// Thread tile of the single-column kernels: kModalTX threads along x (a
// divisor of 32: a warp then holds 32 / kModalTX thread rows, and the +x
// shuffle from the previous row's last lane reaches only a halo thread, which
// discards it) by kModalTY rows.  A tile owns (kModalTX - 1) x (kModalTY - 1)
// node columns.
#ifndef TOPO_MODAL_TX
#define TOPO_MODAL_TX 16
#endif
#ifndef TOPO_MODAL_TY
#define TOPO_MODAL_TY 12
#endif
constexpr int kModalTX = TOPO_MODAL_TX, kModalTY = TOPO_MODAL_TY;

static_assert(32 % kModalTX == 0 && kModalTX >= 8, "x tile: 8, 16 or 32 threads");
static_assert(kModalTX * kModalTY % 32 == 0 && kModalTX * kModalTY <= 512, "whole warps");

// exchange a finished plane's corners with the neighbours: res = the sums at
// the node (ex, ey) of the plane (includes the CTA barrier).  Only threads
// with tx, ty >= 1 own a node: what the others receive (a tx = 0 lane gets
// the previous thread row's last lane, or its own value) and the slot they
// write (read only by the tx = 0 thread of the next row) is never used, so
// no select guards the shuffled values; the row above is guarded (ty = 0
// has none).
template <typename T>
__device__ __forceinline__ void modal_exchange(const T (&plane)[3][4], T (*xch)[kModalTX][3], int tx,
                                               int ty, T (&res)[3]) {
  T n0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T r1 = shfl_up1(plane[c][1]);
    const T r3 = shfl_up1(plane[c][3]);
    n0[c] = plane[c][0] + r1;
    xch[ty][tx][c] = plane[c][2] + r3;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) res[c] = n0[c] + (ty > 0 ? xch[ty - 1][tx][c] : T(0));
}

// the exchange, then the epilogue on the owned node (ex, ey, ez), operands
// read from global memory; `clean`: the tile holds no fixed DOF (no support test)
template <typename T, class Epi>
__device__ __forceinline__ T modal_finish(const T (&plane)[3][4], T (*xch)[kModalTX][3], int tx,
                                          int ty, int ex, int ey, int ez, bool emit, bool clean,
                                          const T (&ctr)[3], const Dims& d, const Epi& epi) {
  T res[3];
  modal_exchange<T>(plane, xch, tx, ty, res);
  if (!emit) return T(0);
  const long long o = d.node(ex, ey, ez);
  return clean ? epi_one(epi, ex, ey, ez, o, res, ctr, FreeDims{d.comp})
               : epi_one(epi, ex, ey, ez, o, res, ctr, d);
}

constexpr int kModalOwnX = kModalTX - 1, kModalOwnY = kModalTY - 1;
constexpr int kModalStages = 4;
constexpr int kClRing = 4;       // halo-ring slots of the cluster form
constexpr int kClMaxCtas = 8;    // portable cluster size: x extents up to 8 x 16 elements

// The cluster form's exchange: as modal_exchange, but lane 0's left
// neighbour corners (h1, h3) come from the CTA on the left instead of the
// shuffle, and with `xn` (lane 15 of the last CTA when nx is a multiple of
// 16) the +x corners of the thread's element also make the node column
// x = nx: resX = its (1,0) corner plus the (1,1) corner of the row below,
// passed through xchx.
__device__ __forceinline__ void modal_exchange_cl(const float (&plane)[3][4],
                                                  float (*xch)[kModalTX][3], float* xchx, int tx,
                                                  int ty, const float (&h1)[3],
                                                  const float (&h3)[3], bool xn, float (&res)[3],
                                                  float (&resx)[3]) {
  float n0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float r1 = shfl_up1(plane[c][1]);
    float r3 = shfl_up1(plane[c][3]);
    if (tx == 0) {
      r1 = h1[c];
      r3 = h3[c];
    }
    n0[c] = plane[c][0] + r1;
    xch[ty][tx][c] = plane[c][2] + r3;
    if (xn) xchx[ty * 3 + c] = plane[c][3];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    res[c] = n0[c] + (ty > 0 ? xch[ty - 1][tx][c] : 0.f);
    if (xn) resx[c] = plane[c][1] + (ty > 0 ? xchx[(ty - 1) * 3 + c] : 0.f);
  }
}
// node box columns: >= 3 (alignment slack) + kModalTX + 1, a multiple of 4
constexpr int kMBoxX = kModalTX == 32 ? 40 : (kModalTX + 4 + 3) / 4 * 4;
constexpr int kMAuxX = (kModalTX + 3 + 3) / 4 * 4;  // >= 3 (alignment slack) + kModalTX columns

// Boxes and shared-memory layout of the TMA kernel for a tile of TY thread
// rows (TY - 1 owned node rows).  Stage layout (floats): node box, element
// box at a 128-byte boundary, then the epilogue's operand planes (Epi::kAux
// boxes of kMAuxX x (TY - 1) x 3 nodes: the owned rows of the node plane the
// stage's epilogue writes).
template <int TY>
struct MTile {
  static constexpr int OwnY = TY - 1;
  static constexpr int BoxNY = TY + 1;  // node rows y0-1 .. y0+OwnY
  static constexpr int BoxEY = TY;      // element rows y0-1 .. y0+OwnY-1
  static constexpr int Node = 3 * BoxNY * kMBoxX;
  static constexpr int Elem = BoxEY * kMBoxX;
  static constexpr uint32_t StageTx = (uint32_t)(Node + Elem) * 4u;
  static constexpr int ElemOff = (Node + 31) / 32 * 32;
  static constexpr int StageBase = (ElemOff + Elem + 31) / 32 * 32;
  static constexpr int AuxY = OwnY;
  static constexpr int Aux = 3 * AuxY * kMAuxX;
  static constexpr int AuxStride = (Aux + 31) / 32 * 32;
  static constexpr uint32_t AuxTx = (uint32_t)Aux * 4u;
  static constexpr size_t XchBytes = sizeof(float) * 2 * TY * kModalTX * 3;
  // cluster form: the halo ring (kClRing slots of TY rows x 6 values, written
  // by the CTA on the left), the exchange slot of the extra node column, and
  // the ring's full and empty mbarriers
  static constexpr int ClRingFloats = kClRing * TY * 6;
  static constexpr int ClXchXFloats = 2 * TY * 3;
  __host__ __device__ static constexpr int stage_floats(int naux) {
    return StageBase + naux * AuxStride;
  }
  __host__ __device__ static constexpr size_t smem(int naux, bool cl = false) {
    return sizeof(float) * stage_floats(naux) * kModalStages + XchBytes +
           sizeof(uint64_t) * kModalStages + 128 +  // + alignment slack
           (cl ? sizeof(uint64_t) * 2 * kClRing + sizeof(float) * (ClRingFloats + ClXchXFloats)
               : 0);
  }
};

// Grid: (x tiles, y tiles, zc z-chunks x designs); design b reads and writes
// its own buffers at b * S bytes from design 0's (the TMA maps carry the
// design as their outermost dimension).
//
// CL (the cluster form): the x tiles of a (y tile, z chunk, design) are one
// thread-block cluster of gridDim.x CTAs, CTA k covering element columns
// 16 k .. 16 k + 15 with no halo column: lane tx owns the corner-0 node of
// its own element, and the +x corners of the left neighbour element (lane 15
// of CTA k - 1) come through a ring of kClRing slots in this CTA's shared
// memory that CTA k - 1 writes with st.async, each store completing its
// bytes on the slot's full mbarrier here (armed with the slot's TY x 24
// bytes by thread 0 per use; no fence on the writer's side).  Thread 0 (row
// 0 owns no node, so it has no global stores in flight) frees a slot for the
// writer by a release arrival on the writer's empty mbarrier once the
// layer's barrier shows every row has read it.  When nx = 16 x (CTAs), lane
// 15 of the last CTA also finishes node column nx.
template <class Epi, int TY, bool CL = false>
__global__ void __launch_bounds__(kModalTX* TY, CL ? 4 : 0)
    k_modal_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap emap,
                const __grid_constant__ CUtensorMap amap0,
                const __grid_constant__ CUtensorMap amap1, const Dims d,
                const __grid_constant__ ModalCoef<float> kc, const Epi epi0, const Red red0,
                const int zchunk, const int zc, const DSel S, const int* __restrict__ done,
                int* __restrict__ errflag) {
  constexpr int NA = epi_staged<Epi>();  // staged operand vectors
  constexpr int DI = Epi::kDinvAux;      // >= 0: D^-1 formed from the moduli
  static_assert(NA <= 2, "at most two staged operand vectors");
  static_assert(DI < 0 || DI == Epi::kAux - 1, "D^-1 is the last operand");
  using Tl = MTile<TY>;
  constexpr int SF = Tl::stage_floats(NA);
  pdl_start();
  const int slot = blockIdx.z / zc, chunk = blockIdx.z - slot * zc;
  const int design = S.id(slot);
  const long long off = design * S.S;
  done = bshift(done, off);
  errflag = bshift(errflag, off);
  if (done != nullptr && *done) return;  // uniform over the design's blocks
  const Epi epi = epi0.shifted(off);
  const Red red = red0.shifted(off);
  extern __shared__ __align__(128) unsigned char modal_dyn[];
  // TMA destinations on 128-byte boundaries whatever the dynamic window's offset
  unsigned char* base = modal_dyn + ((128u - (smem_u32(modal_dyn) & 127u)) & 127u);
  float* stg = reinterpret_cast<float*>(base);
  auto xch = reinterpret_cast<float(*)[TY][kModalTX][3]>(
      base + sizeof(float) * SF * kModalStages);
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(base + sizeof(float) * SF * kModalStages + Tl::XchBytes);
  // cluster form: ring mbarriers, ring values, the extra column's exchange
  uint64_t* cl_full = bar + kModalStages;
  uint64_t* cl_empty = cl_full + kClRing;
  float* ring = reinterpret_cast<float*>(cl_empty + kClRing);
  float* xchx = ring + Tl::ClRingFloats;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kModalTX + tx;
  const int crank = CL ? (int)blockIdx.x : 0, ncl = CL ? (int)gridDim.x : 1;
  // x0 - 1: the first element column (the halo's in the tiled form); CL: 16 k
  const int x0 = CL ? crank * kModalTX + 1 : blockIdx.x * kModalOwnX;
  const int y0 = blockIdx.y * Tl::OwnY;
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const int bx = x0 & ~3;  // 16-byte aligned box start (storage x of node x0-1 is x0)
  const int ox = x0 - bx;
  const int kb = chunk * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const int nst = (ke - kb) + 2;  // stage t: node plane kb-2+t+1, element layer kb-2+t
  if (tid == 0) {
    for (int q = 0; q < kModalStages; ++q) mbar_init(&bar[q], 1);
    if constexpr (CL)
      for (int q = 0; q < kClRing; ++q) {
        mbar_init(&cl_full[q], 1);
        mbar_init(&cl_empty[q], 1);
      }
    fence_mbar_init();
    if constexpr (CL)
      if (crank > 0)  // every slot armed for its first use
        for (int q = 0; q < kClRing; ++q) mbar_arrive_expect_tx(&cl_full[q], TY * 24u);
    tma_prefetch_desc(&xmap);
    tma_prefetch_desc(&emap);
    if (NA > 0) tma_prefetch_desc(&amap0);
    if (NA > 1) tma_prefetch_desc(&amap1);
    // Fault-injection hook (errflag[1] == 1, set by topo_debug_inject_timeout):
    // one CTA of the design runs one bounded wait on a barrier that nothing
    // ever completes (no copy is issued on it), with a 64-poll limit, so the
    // wait runs out and records a timeout the way a lost transfer would.
    // Nothing is in flight on that barrier; the stage copies are unaffected.
    if (errflag != nullptr && atomicCAS(errflag + 1, 1, 0) == 1) {
      __shared__ uint64_t never_bar;
      mbar_init(&never_bar, 1);
      fence_mbar_init();
      mbar_wait_bounded(&never_bar, 0u, errflag, 64u);
    }
  }
  if constexpr (CL)
    cluster_sync();  // every CTA's ring barriers exist before any remote arrival
  else
    __syncthreads();
  // stage t: node plane kb-1+t, element layer kb-2+t and, once that plane
  // has an epilogue (t >= 2), the operand planes of node plane kb-2+t
  auto issue = [&](int t) {
    const int slot = t % kModalStages;
    float* sp = stg + slot * SF;
    const bool ax = NA > 0 && t >= 2;
    mbar_arrive_expect_tx(&bar[slot], Tl::StageTx + (ax ? NA * Tl::AuxTx : 0u));
    tma_load_5d(sp, &xmap, &bar[slot], bx, y0, kb + t, 0, design);
    tma_load_4d(sp + Tl::ElemOff, &emap, &bar[slot], bx, y0, kb - 1 + t, design);
    if (ax) {
      tma_load_5d(sp + Tl::StageBase, &amap0, &bar[slot], bx, y0 + 1, kb - 1 + t, 0, design);
      if (NA > 1)
        tma_load_5d(sp + Tl::StageBase + Tl::AuxStride, &amap1, &bar[slot], bx, y0 + 1, kb - 1 + t,
                    0, design);
    }
  };
  if (tid == 0)
    for (int t = 0; t < kModalStages && t < nst; ++t) issue(t);
  const bool own = (CL || tx > 0) && ty > 0 && ex <= d.nx && ey <= d.ny;
  // CL: lane 15 of the last CTA also owns node column nx when no lane's
  // element column is nx
  const bool xn = CL && crank == ncl - 1 && tx == kModalTX - 1 && d.nx == ncl * kModalTX;
  const bool xown = xn && ty > 0 && ey <= d.ny;
  // tiles without any fixed DOF run the epilogue without the per-DOF support test
  const bool clean = CL ? !d.box_may_fix(x0 - 1, min(x0 + kModalTX - 1, d.nx), y0, kb)
                        : !d.box_may_fix(x0, x0 + kModalOwnX - 1, y0, kb);
  const FreeDims fd{d.comp};
  MarchColumn<float> col;
  float part = 0.f;  // this thread's nodes only (at most zchunk); widened to FP64 below
  float es_prev = 0.f;  // (DI) moduli of the 2 x 2 elements below node (ex, ey), layer before
  float esx_prev = 0.f;  // the same for node (nx, ey) (xn)
  float xr[3] = {0.f, 0.f, 0.f};  // (xn) raw node (nx, ey) of the last plane read
  // stage (slot, phase) -> registers: the top node plane, the element
  // modulus and (DI) the moduli of the 2 x 2 elements around (ex, ey)
  auto read_stage = [&](int r, uint32_t ph, float(&top)[2][2][3], float& E, float& es,
                        float& esx) {
    mbar_wait_bounded(&bar[r], ph, errflag);
    const float* nd = stg + r * SF;
    es = 0.f;
    esx = 0.f;
    if (DI >= 0) {  // used by owned nodes only; the others read inside the stage too
      const float* e0 = nd + Tl::ElemOff + (ty - 1) * kMBoxX + ox + tx - 1;
      es = (e0[0] + e0[1]) + (e0[kMBoxX] + e0[kMBoxX + 1]);
      if (xn) esx = (e0[1] + e0[2]) + (e0[kMBoxX + 1] + e0[kMBoxX + 2]);
    }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          top[dy][dx][c] = nd[c * (Tl::BoxNY * kMBoxX) + (ty + dy) * kMBoxX + ox + tx + dx];
    E = nd[Tl::ElemOff + ty * kMBoxX + ox + tx];
  };
  {  // the first node plane only seeds the march
    float top[2][2][3], E;
    read_stage(0, 0u, top, E, es_prev, esx_prev);
#pragma unroll
    for (int c = 0; c < 3; ++c) xr[c] = top[0][1][c];
    __syncthreads();
    if (tid == 0 && kModalStages < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(kModalStages);
    }
    march_seed(col, top);
  }
  const long long o_col = d.node(ex, ey, 0), ps = d.plane_stride();  // node (ex, ey, ez): + ez ps
  int rs = 1;  // stage t's ring slot t % kModalStages, and its mbarrier phase
  uint32_t phase = 0u;
  for (int t = 1; t < nst; ++t) {
    const float* nd = stg + rs * SF;
    float top[2][2][3], E, es, esx;
    read_stage(rs, phase, top, E, es, esx);
    float plane[3][4], ctr[3];
    march_layer(col, top, E, kc, plane, ctr);
    const int ez = kb - 2 + t;
    float res[3], resx[3], ctrx[3];
    if constexpr (CL) {
      // layer t - 1 (from 0) uses halo-ring slot (t - 1) % kClRing for the
      // (t - 1) / kClRing-th time
      const int hs = (t - 1) % kClRing;
      const uint32_t use = (uint32_t)(t - 1) / kClRing;
      if (tx == kModalTX - 1 && crank + 1 < ncl) {  // this row's +x corners to the right
        if (use > 0) mbar_wait_cluster_bounded(&cl_empty[hs], (use - 1u) & 1u, errflag);
        const uint32_t dst = cluster_map(smem_u32(ring + (hs * TY + ty) * 6), crank + 1);
        const uint32_t rb = cluster_map(smem_u32(&cl_full[hs]), crank + 1);
        cluster_st_async_v2(dst, plane[0][1], plane[1][1], rb);
        cluster_st_async_v2(dst + 8u, plane[2][1], plane[0][3], rb);
        cluster_st_async_v2(dst + 16u, plane[1][3], plane[2][3], rb);
      }
      float h1[3] = {0.f, 0.f, 0.f}, h3[3] = {0.f, 0.f, 0.f};  // the left element's corners
      if (tx == 0 && crank > 0) {
        mbar_wait_bounded(&cl_full[hs], use & 1u, errflag);
        const float* src = ring + (hs * TY + ty) * 6;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          h1[c] = src[c];
          h3[c] = src[3 + c];
        }
      }
      modal_exchange_cl(plane, xch[t & 1], xchx + (t & 1) * (TY * 3), tx, ty, h1, h3, xn, res,
                        resx);
      if (tid == 0 && crank > 0) {  // every row has read slot hs: re-arm it, free it
        mbar_arrive_expect_tx(&cl_full[hs], TY * 24u);
        mbar_arrive_remote(cluster_map(smem_u32(&cl_empty[hs]), crank - 1));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {  // raw node (nx, ey, ez), then the top plane's
        ctrx[c] = xr[c];
        xr[c] = top[0][1][c];
      }
    } else {
      modal_exchange<float>(plane, xch[t & 1], tx, ty, res);
    }
    // the slot the exchange barrier retires: stage t's (its node data is
    // read), or with staged operands stage t-1's (its epilogue, before this
    // barrier, was the last reader; stage 0's slot was refilled after the seed)
    const int freed = NA > 0 ? t - 1 : t;
    if (tid == 0 && freed >= 1 && freed + kModalStages < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(freed + kModalStages);
    }
    if (own && t >= 2) {
      const int ii[1] = {ex};
      const long long oo[1] = {o_col + (long long)ez * ps};
      const bool ow[1] = {true};
      const float rr[1][3] = {{res[0], res[1], res[2]}};
      const float cc[1][3] = {{ctr[0], ctr[1], ctr[2]}};
      float av[epi_slots<Epi>()][1][3];
      const float* ap = nd + Tl::StageBase + (ty - 1) * kMAuxX + ox + tx;
#pragma unroll
      for (int q = 0; q < NA; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) av[q][0][c] = ap[q * Tl::AuxStride + c * (Tl::AuxY * kMAuxX)];
      if constexpr (DI >= 0) {  // D^-1 of the masked operator, 1 where no stiffness
        const float sum = es_prev + es;
        const float dv = sum > 0.f ? jacobi_rcp(kc.kdiag * sum) : 1.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) av[DI][0][c] = dv;
      }
      if (clean)
        part += epi.template finish<1>(ii, ey, ez, oo, ow, rr, cc, av, fd);
      else
        part += epi.template finish<1>(ii, ey, ez, oo, ow, rr, cc, av, d);
    }
    if constexpr (CL) {
      if (xown && t >= 2) {  // node column nx (lane 15 of the last CTA)
        const int ii[1] = {d.nx};
        const long long oo[1] = {d.node(d.nx, ey, ez)};
        const bool ow[1] = {true};
        const float rr[1][3] = {{resx[0], resx[1], resx[2]}};
        const float cc[1][3] = {{ctrx[0], ctrx[1], ctrx[2]}};
        float av[epi_slots<Epi>()][1][3];
        const float* ap = nd + Tl::StageBase + (ty - 1) * kMAuxX + ox + tx + 1;
#pragma unroll
        for (int q = 0; q < NA; ++q)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            av[q][0][c] = ap[q * Tl::AuxStride + c * (Tl::AuxY * kMAuxX)];
        if constexpr (DI >= 0) {
          const float sum = esx_prev + esx;
          const float dv = sum > 0.f ? jacobi_rcp(kc.kdiag * sum) : 1.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) av[DI][0][c] = dv;
        }
        if (clean)
          part += epi.template finish<1>(ii, ey, ez, oo, ow, rr, cc, av, fd);
        else
          part += epi.template finish<1>(ii, ey, ez, oo, ow, rr, cc, av, d);
      }
      esx_prev = esx;
    }
    es_prev = es;
    if (++rs == kModalStages) {
      rs = 0;
      phase ^= 1u;
    }
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * chunk),
                       gridDim.x * gridDim.y * zc);
  }
  if constexpr (CL) cluster_sync();  // no CTA leaves while a neighbour may reach its ring
}

// Plain-load variant (FP64, and FP32 grids too small for the TMA boxes):
// same work split, inputs read with bounds checks from the ghosted arrays.
// The FP64 form asks for registers that leave TOPO_PLAIN64_MINB CTAs per SM
// (its FP64 pipe needs warps to hide latency across the per-plane barriers).
#ifndef TOPO_PLAIN64_MINB
#define TOPO_PLAIN64_MINB 2
#endif
template <typename T, class Epi>
__global__ void __launch_bounds__(kModalTX* kModalTY, sizeof(T) == 8 ? TOPO_PLAIN64_MINB : 1)
    k_modal_plain(const T* __restrict__ x, const T* __restrict__ E, const Dims d,
                  const __grid_constant__ ModalCoef<T> kc, const Epi epi0, const Red red0,
                  const int zchunk, const int zc, const DSel S,
                  const int* __restrict__ done, T* __restrict__ energy) {
  pdl_start();
  const int slot = blockIdx.z / zc, chunk = blockIdx.z - slot * zc;
  const long long off = S.off(slot);
  done = bshift(done, off);
  if (done != nullptr && *done) return;
  x = bshift(x, off);
  E = bshift(E, off);
  energy = bshift(energy, off);
  const Epi epi = epi0.shifted(off);
  const Red red = red0.shifted(off);
  __shared__ T xch[2][kModalTY][kModalTX][3];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * kModalOwnX, y0 = blockIdx.y * kModalOwnY;
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const int kb = chunk * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool own = tx > 0 && ty > 0 && ex <= d.nx && ey <= d.ny;
  const bool clean = !d.box_may_fix(x0, x0 + kModalOwnX - 1, y0, kb);
  auto node_val = [&](int i, int j, int k, int c) -> T {
    if (i > d.nx + 1 || j > d.ny + 1 || k > d.nz + 1) return T(0);  // beyond the ghost ring
    return __ldg(x + c * d.comp + d.node(i, j, k));
  };
  MarchColumn<T> col;
  {
    T raw[2][2][3];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) raw[dy][dx][c] = node_val(ex + dx, ey + dy, kb - 1, c);
    march_seed(col, raw);
  }
  T part = T(0);
  for (int ez = kb - 1; ez < ke; ++ez) {
    T top[2][2][3];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) top[dy][dx][c] = node_val(ex + dx, ey + dy, ez + 1, c);
    const T Ee = (ex <= d.nx && ey <= d.ny && ez <= d.nz) ? __ldg(E + d.elem(ex, ey, ez)) : T(0);
    T plane[3][4], ctr[3], dot = T(0);
    march_layer(col, top, Ee, kc, plane, ctr, energy ? &dot : nullptr);
    // element energies (u_e - u_0)^T k0 (u_e - u_0), written by the CTA and
    // z-chunk that own the element (the others compute it as halo / warm-up)
    if (energy && tx > 0 && ty > 0 && ex < d.nx && ey < d.ny && ez >= kb && ez < d.nz)
      energy[d.elem(ex, ey, ez)] = Ee != T(0) ? dot : T(0);
    part += modal_finish<T, Epi>(plane, xch[(ez - kb + 1) & 1], tx, ty, ex, ey, ez,
                                 own && ez >= kb, clean, ctr, d, epi);
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * chunk),
                       gridDim.x * gridDim.y * zc);
  }
}

// z planes per CTA for the modal kernels: a few waves over 152 SMs counting
// all `nb` designs of a launch, a one-layer warm-up below ~10%, and no more
// CTAs per design than partial-sum slots; a launch of many designs marches
// whole columns (up to 64 planes), and the chunks of a column are equal
// (a floor of 8 or 16 planes measured 1-5 % more solves/s with 64 designs in
// flight on 96x32x32 but 57-147 % more latency for one design: 4 it is)
// z chunks per launch: planes per CTA column ~ the launch's (tiles x planes
// x designs) over 152 SMs x 2 x TOPO_ZCHUNK_WAVES (at least 4, at most 64);
// full 256-design batches of 96x32x32 keep whole columns, narrower launches
// (the lockstep tail, where few designs still iterate) split them.  Measured
// on the batched 96x32x32 Chebyshev step: 4 -> 2.003, 8 -> 1.987 us per
// design and launch.
#ifndef TOPO_ZCHUNK_WAVES
#define TOPO_ZCHUNK_WAVES 8
#endif
inline int modal_zchunk(const Dims& d, int nb = 1, int own_y = kModalOwnY) {
  const long long xy = (long long)((d.nx + kModalOwnX) / kModalOwnX) *
                       ((d.ny + own_y) / own_y);
  const int planes = d.nz + 1;
  int z = (int)((xy * planes * nb) / (152 * 2 * TOPO_ZCHUNK_WAVES));
  if (z < 4) z = 4;
  if (z > 64) z = 64;
  while (xy * ((planes + z - 1) / z) > kMaxPartials) ++z;
  // equal chunks: each costs one warm-up layer, a short last one more than its share
  const int zc = (planes + z - 1) / z;
  return (planes + zc - 1) / zc;
}

// ty: thread rows of the tile (box heights ty + 1 node rows, ty element rows)
bool modal_maps(const float* x, const float* E, const Dims& d, const Bat& bt, int ty,
                CUtensorMap* xmap, CUtensorMap* emap);
bool modal_aux_map(const float* v, const Dims& d, const Bat& bt, int ty, CUtensorMap* map);

// Tile height of a launch: kModalTY, or for a batched launch (several
// designs; one design keeps the 12-row tiles, more and smaller CTAs, for its
// latency) kModalTallTY or kModalShortTY where that launches fewer thread
// rows per x column of tiles and its node box fits the grid (ty + 1 <= ny + 3).
// 96x32x32: the second level's 17 node rows take one 18-row tile instead of
// two 12-row ones (72 % of the threads own a node instead of 54 %); the
// third level's 9 rows one 10-row tile (the 12-row box does not fit there,
// which left that level to the plain-load kernel).
constexpr int kModalTallTY = 18, kModalShortTY = 10;

inline int modal_pick_ty(const Dims& d, int nb) {
  const auto fits = [&](int ty) { return ty + 1 <= d.ny + 3; };
  const auto rows = [&](int ty) { return (long long)((d.ny + ty - 1) / (ty - 1)) * ty; };
  if (nb < 2) return kModalTY;
  int best = fits(kModalTY) ? kModalTY : -1;
  for (int ty : {kModalTallTY, kModalShortTY})
    if (fits(ty) && (best < 0 || rows(ty) < rows(best))) best = ty;
  return best < 0 ? kModalTY : best;
}

// Use the cluster form?  form 4 asks for it; the automatic form takes it
// with TOPO_MODAL_CLUSTER_AUTO.  It needs the x extent within one portable
// cluster (nx <= 8 x 16).
#ifndef TOPO_MODAL_CLUSTER_AUTO
#define TOPO_MODAL_CLUSTER_AUTO 0
#endif
inline bool modal_use_cluster(const Dims& d, int form) {
  const int ncl = (d.nx + kModalTX - 1) / kModalTX;
  return (form == 4 || (form == 0 && TOPO_MODAL_CLUSTER_AUTO)) && ncl <= kClMaxCtas;
}

template <class Epi, int TY, bool CL>
cudaError_t launch_modal_tma_form(const CUtensorMap& xm, const CUtensorMap& em,
                                  const CUtensorMap (&am)[2], const Dims& d,
                                  const ModalCoef<float>& kc, const Epi& epi, const Red& red,
                                  const int* done, int* errflag, cudaStream_t s, const Bat& bt) {
  constexpr size_t smem = MTile<TY>::smem(epi_staged<Epi>(), CL);
  static bool attr = false;  // per instantiation; setting it twice is harmless
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_modal_tma<Epi, TY, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int z = modal_zchunk(d, bt.nb, TY - 1);
  const int zc = (d.nz + z) / z;
  dim3 block(kModalTX, TY, 1);
  const int gx = CL ? (d.nx + kModalTX - 1) / kModalTX : (d.nx + kModalOwnX) / kModalOwnX;
  dim3 grid(gx, (d.ny + TY - 1) / (TY - 1), zc * bt.nb);
  if constexpr (CL) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)gx;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_modal_tma<Epi, TY, true>, xm, em, am[0], am[1], d, kc, epi,
                              red, z, zc, bt.sel(), done, errflag);
  } else {
    return launch_pdl(k_modal_tma<Epi, TY, false>, grid, block, smem, s, xm, em, am[0], am[1], d,
                      kc, epi, red, z, zc, bt.sel(), done, errflag);
  }
}

template <class Epi, int TY>
cudaError_t launch_modal_tma(const float* x, const float* E, const Dims& d,
                             const ModalCoef<float>& kc, const Epi& epi, const Red& red,
                             const int* done, int* errflag, cudaStream_t s, const Bat& bt,
                             bool* launched) {
  *launched = false;
  CUtensorMap xm, em, am[2];
  std::memset(am, 0, sizeof(am));
  bool ok = modal_maps(x, E, d, bt, TY, &xm, &em);
  for (int q = 0; q < epi_staged<Epi>() && ok; ++q)
    ok = modal_aux_map(epi.aux(q), d, bt, TY, &am[q]);
  if (!ok) return cudaSuccess;  // the boxes do not fit: the plain kernel
  *launched = true;
  if (modal_use_cluster(d, kc.form))
    return launch_modal_tma_form<Epi, TY, true>(xm, em, am, d, kc, epi, red, done, errflag, s,
                                                bt);
  return launch_modal_tma_form<Epi, TY, false>(xm, em, am, d, kc, epi, red, done, errflag, s, bt);
}

template <typename T, class Epi>
cudaError_t launch_modal_single(const T* x, const T* E, const Dims& d, const ModalCoef<T>& kc,
                                const Epi& epi, const Red& red, const int* done, int* errflag,
                                cudaStream_t s, const Bat& bt, T* energy = nullptr) {
  if constexpr (sizeof(T) == 4) {
    if (energy) return cudaErrorInvalidValue;  // element energies: the FP64 kernel only
    bool launched = false;
    cudaError_t e;
    switch (modal_pick_ty(d, bt.nb)) {
      case kModalTallTY:
        e = launch_modal_tma<Epi, kModalTallTY>(x, E, d, kc, epi, red, done, errflag, s, bt,
                                                &launched);
        break;
      case kModalShortTY:
        e = launch_modal_tma<Epi, kModalShortTY>(x, E, d, kc, epi, red, done, errflag, s, bt,
                                                 &launched);
        break;
      default:
        e = launch_modal_tma<Epi, kModalTY>(x, E, d, kc, epi, red, done, errflag, s, bt,
                                            &launched);
        break;
    }
    if (e != cudaSuccess || launched) return e;
  }
  const int z = modal_zchunk(d, bt.nb);
  const int zc = (d.nz + z) / z;
  dim3 block(kModalTX, kModalTY, 1);
  dim3 grid((d.nx + kModalOwnX) / kModalOwnX, (d.ny + kModalOwnY) / kModalOwnY, zc * bt.nb);
  return launch_pdl(k_modal_plain<T, Epi>, grid, block, 0, s, x, E, d, kc, epi, red, z, zc, bt.sel(),
                    done, energy);
}

}  // namespace topo
