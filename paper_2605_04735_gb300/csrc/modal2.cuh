// Column-paired FP32 form of the modal (Walsh-Hadamard) element operator,
// with packed two-wide FP32 arithmetic (add/sub/mul/fma .f32x2, sm_100+).
//
// The element arithmetic is the one in modal.cuh (k0 u = H K~ H^T u, 45
// non-zeros of K~, x-y transform per node plane shared by the elements above
// and below, modal-domain plane combine, corner-0 shift).  What changes is
// the work split: thread (tx, ty) marches two element columns,
// A = (x0 - 1 + tx, y0 - 1 + ty) and B = A + (32, 0), and keeps every
// quantity as the pair (A, B) in one 64-bit register pair, so each
// instruction of the element arithmetic does the work of two elements.
// The two columns never share a node, so the pairs come straight out of
// shared memory (two 32-bit loads into the halves of a pair).
//
// A CTA is 32 x 8 threads over element columns x0-1 .. x0+62 and rows
// y0-1 .. y0+6 and owns the node columns x0 .. x0+62, y0 .. y0+6 (63 x 7):
// the +x corners of column A of lane tx go to lane tx+1 (and those of lane
// 31's A to lane 0's B) by one rotating warp shuffle, the +y corner through
// a double-buffered shared-memory slot as in modal.cuh.  Node planes and
// element layers stream through a 4-stage TMA ring (boxes of 68 x 9 x 3
// nodes and 68 x 8 elements, x start rounded down to 16 bytes).
//
// Tiles without any fixed DOF run the epilogue without the per-DOF support
// test (`FreeDims`).
#pragma once

#include <cuda.h>
#include <algorithm>
#include <cstring>
#include <cuda_runtime.h>

#include "common.cuh"
#include "modal.cuh"
#include "tma.cuh"

namespace topo {

// ModalCoef<float> with every coefficient duplicated into both halves
struct ModalCoef2 {
  float2 D[3][8];
  float2 C[3][3][8];
  float kdiag;  // every diagonal entry of k0
};

inline ModalCoef2 pair_coef(const ModalCoef<float>& k) {
  ModalCoef2 p{};
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < 8; ++m) {
      p.D[a][m] = make_float2(k.D[a][m], k.D[a][m]);
      for (int b = 0; b < 3; ++b) p.C[a][b][m] = make_float2(k.C[a][b][m], k.C[a][b][m]);
    }
  p.kdiag = k.kdiag;
  return p;
}

struct PairColumn {
  float2 bxy[3][4];  // x-y transform of the bottom node plane, shifted by ref
  float2 ref[3];     // raw displacement of the element's corner 0
  float2 carry[3][4];  // previous element's top-face result; [c][0] holds its negative
};

__device__ __forceinline__ void pair_seed(PairColumn& col, const float2 (&raw)[2][2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    col.ref[c] = raw[0][0][c];
    float2 v[4] = {make_float2(0.f, 0.f), psub(raw[0][1][c], col.ref[c]),
                   psub(raw[1][0][c], col.ref[c]), psub(raw[1][1][c], col.ref[c])};
    pfwht4(v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      col.bxy[c][q] = v[q];
      col.carry[c][q] = make_float2(0.f, 0.f);
    }
  }
}

// One element layer for the pair; see modal_layer in modal.cuh for the
// meaning of every step.  plane[c][q]: x-y corner q of node plane ez.
__device__ __forceinline__ void pair_layer(PairColumn& col, const float2 (&top)[2][2][3],
                                           float2 E, float2 nE, const ModalCoef2& kc,
                                           float2 (&plane)[3][4], float2 (&ctr)[3]) {
  float2 uh[3][8];  // [c][0] (the rigid mode) is never formed
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 r = col.ref[c];
    ctr[c] = r;
    float2 v[4] = {psub(top[0][0][c], r), psub(top[0][1][c], r), psub(top[1][0][c], r),
                   psub(top[1][1][c], r)};
    pfwht4(v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 s = pmul(col.bxy[c][q], E);
      if (q > 0) uh[c][q] = pfma(v[q], E, s);  // z mode 0: (bottom + top) E
      uh[c][q + 4] = pfma(v[q], nE, s);        // z mode 1: (bottom - top) E
    }
    // the top plane becomes the next bottom plane, re-referenced to its corner 0
    const float2 nref = top[0][0][c];
    col.bxy[c][0] = pfma(psub(r, nref), make_float2(4.f, 4.f), v[0]);
#pragma unroll
    for (int q = 1; q < 4; ++q) col.bxy[c][q] = v[q];
    col.ref[c] = nref;
  }
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    float2 yh[8];
#pragma unroll
    for (int m = 1; m < 8; ++m) {
      float2 acc = pmul(kc.D[p][m], uh[p][m]);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q == p) continue;
        if (((m >> p) & 1) == ((m >> q) & 1)) continue;
        acc = pfma(kc.C[p][q][m], uh[q][m ^ (1 << p) ^ (1 << q)], acc);
      }
      yh[m] = acc;
    }
    float2 w[4];
    w[0] = psub(yh[4], col.carry[p][0]);  // bottom face (mode 0 of yh is 0) + previous top
    col.carry[p][0] = yh[4];              // stored negated
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      w[q] = padd(padd(yh[q], yh[q + 4]), col.carry[p][q]);
      col.carry[p][q] = psub(yh[q], yh[q + 4]);
    }
    pfwht4(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) plane[p][q] = w[q];
  }
}

constexpr int kPairTX = 32, kPairTY = 8;
constexpr int kPairOwnX = 2 * kPairTX - 1, kPairOwnY = kPairTY - 1;
constexpr int kPairStages = 4;
constexpr int kPBoxX = 68;             // >= 3 (alignment slack) + 65 node columns
constexpr int kPBoxNY = kPairTY + 1;   // node rows y0-1 .. y0+7
constexpr int kPBoxEY = kPairTY;       // element rows y0-1 .. y0+6
constexpr int kPNode = 3 * kPBoxNY * kPBoxX;
constexpr int kPElem = kPBoxEY * kPBoxX;
constexpr int kPNodeStride = (kPNode + 31) / 32 * 32;          // floats, 128-byte multiple
constexpr int kPStageFloats = (kPNodeStride + kPElem + 31) / 32 * 32;
constexpr uint32_t kPStageTx = (uint32_t)(kPNode + kPElem) * 4u;
// The epilogue's operand vectors (Epi::kAux of them) ride in the same ring:
// for the node plane the stage's epilogue writes, a box of 68 x 7 x 3 nodes
// (the owned rows y0 .. y0+6) per vector.
constexpr int kPAuxY = kPairOwnY;
constexpr int kPAux = 3 * kPAuxY * kPBoxX;
constexpr int kPAuxStride = (kPAux + 31) / 32 * 32;  // floats, 128-byte multiple
constexpr uint32_t kPAuxTx = (uint32_t)kPAux * 4u;
__host__ __device__ constexpr int pair_stage_floats(int naux) {
  return kPStageFloats + naux * kPAuxStride;
}
constexpr size_t kPairXchBytes = sizeof(float2) * 2 * kPairTY * kPairTX * 3;
// CTAs resident per SM (the register budget).  Holding the kernel to one CTA
// per SM (one wave) measured 49% slower at 320x160x160: two CTAs per SM it is.
constexpr int kPairCtasPerSm = 2;
__host__ __device__ constexpr size_t pair_smem(int naux) {
  return sizeof(float) * pair_stage_floats(naux) * kPairStages + kPairXchBytes +
         sizeof(uint64_t) * kPairStages + 128;  // + alignment slack
}

// Grid: (G CTAs per design, 1, designs).  The work of a design is the list of
// (x-y tile, node plane) pairs in tile-major order; CTA b takes the equal
// share [b W / G, (b + 1) W / G) of its W entries and marches it as one or
// two z segments (a segment that starts inside a tile's march pays the
// two-layer warm-up again).  G is one resident wave, so no SM idles while
// others finish a second CTA.
template <class Epi>
__global__ void __launch_bounds__(kPairTX* kPairTY, 2)
    k_modal_pair(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap emap,
                 const __grid_constant__ CUtensorMap amap0,
                 const __grid_constant__ CUtensorMap amap1, const Dims d,
                 const __grid_constant__ ModalCoef2 kc, const Epi epi0, const Red red0,
                 const int gx, const int gy, const DSel S, const int* __restrict__ done,
                 int* __restrict__ errflag) {
  constexpr int NA = epi_staged<Epi>();  // staged operand vectors
  constexpr int DI = Epi::kDinvAux;      // >= 0: D^-1 formed from the moduli
  static_assert(NA <= 2, "at most two staged operand vectors");
  static_assert(DI < 0 || DI == Epi::kAux - 1, "D^-1 is the last operand");
  constexpr int SF = pair_stage_floats(NA);
  pdl_start();
  const int design = S.id(blockIdx.z);
  const long long off = design * S.S;
  done = bshift(done, off);
  errflag = bshift(errflag, off);
  if (done != nullptr && *done) return;  // uniform over the design's blocks
  const Epi epi = epi0.shifted(off);
  const Red red = red0.shifted(off);
  extern __shared__ __align__(128) unsigned char pair_dyn[];
  // TMA destinations on 128-byte boundaries whatever the dynamic window's offset
  unsigned char* pair_smem = pair_dyn + ((128u - (smem_u32(pair_dyn) & 127u)) & 127u);
  float* stg = reinterpret_cast<float*>(pair_smem);
  auto xch = reinterpret_cast<float2(*)[3][kPairTY][kPairTX]>(
      pair_smem + sizeof(float) * SF * kPairStages);
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(pair_smem + sizeof(float) * SF * kPairStages + kPairXchBytes);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kPairTX + tx;
  const int planes = d.nz + 1;
  const long long W = (long long)gx * gy * planes;
  const long long L0 = (long long)blockIdx.x * W / gridDim.x;
  const long long L1 = (long long)(blockIdx.x + 1) * W / gridDim.x;
  if (tid == 0) {
    for (int q = 0; q < kPairStages; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
    tma_prefetch_desc(&xmap);
    tma_prefetch_desc(&emap);
    if (NA > 0) tma_prefetch_desc(&amap0);
    if (NA > 1) tma_prefetch_desc(&amap1);
  }
  __syncthreads();
  const FreeDims fd{d.comp};
  const int src = (tx + kPairTX - 1) & (kPairTX - 1);
  float part = 0.f;
  int gs = 0;  // stages consumed so far over all segments (mbarrier phases)
  for (long long L = L0; L < L1;) {
    const long long T = L / planes;
    const int kb = (int)(L - T * planes);
    const int ke = (int)min((long long)planes, kb + (L1 - L));
    L += ke - kb;
    const int x0 = (int)(T % gx) * kPairOwnX, y0 = (int)(T / gx) * kPairOwnY;
    const int exA = x0 - 1 + tx, ey = y0 - 1 + ty;
    const int bx = x0 & ~3;  // 16-byte aligned box start (storage x of node x0-1 is x0)
    const int ox = x0 - bx;
    const int nst = (ke - kb) + 2;  // stage t: node plane kb-1+t, element layer kb-2+t
    // stage t also carries the operand planes of node plane kb-2+t (storage
    // plane kb-1+t, rows y0 .. y0+6) once that plane has an epilogue (t >= 2)
    auto issue = [&](int t) {
      const int slot = (gs + t) % kPairStages;
      float* sp = stg + slot * SF;
      const bool ax = NA > 0 && t >= 2;
      mbar_arrive_expect_tx(&bar[slot], kPStageTx + (ax ? NA * kPAuxTx : 0u));
      tma_load_5d(sp, &xmap, &bar[slot], bx, y0, kb + t, 0, design);
      tma_load_4d(sp + kPNodeStride, &emap, &bar[slot], bx, y0, kb - 1 + t, design);
      if (ax) {
        tma_load_5d(sp + kPStageFloats, &amap0, &bar[slot], bx, y0 + 1, kb - 1 + t, 0, design);
        if (NA > 1)
          tma_load_5d(sp + kPStageFloats + kPAuxStride, &amap1, &bar[slot], bx, y0 + 1,
                      kb - 1 + t, 0, design);
      }
    };
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int t = 0; t < kPairStages && t < nst; ++t) issue(t);
    }
    const bool ownA = tx > 0 && ty > 0 && exA <= d.nx && ey <= d.ny;
    const bool ownB = ty > 0 && exA + 32 <= d.nx && ey <= d.ny;
    const bool clean = !d.box_may_fix(x0, x0 + kPairOwnX - 1, y0, kb);
    const int lx = ox + tx;  // this thread's column A inside a box row
    long long oA = d.node(exA, ey, kb);

    // stage t -> registers: the top node plane (pairs A, B) and the element moduli
    // (DI) es: moduli of the 2 x 2 elements around the nodes (A, B) in the stage's layer
    auto load_stage = [&](int t, float2(&top)[2][2][3], float2& E, float2& es) {
      const int g = gs + t;
      const int slot = g % kPairStages;
      mbar_wait_bounded(&bar[slot], (uint32_t)((g / kPairStages) & 1), errflag);
      const float* nd = stg + slot * SF;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float* p = nd + c * (kPBoxNY * kPBoxX) + (ty + dy) * kPBoxX + lx + dx;
            top[dy][dx][c] = make_float2(p[0], p[32]);
          }
      const float* el = nd + kPNodeStride + ty * kPBoxX + lx;
      E = make_float2(el[0], el[32]);
      es = make_float2(0.f, 0.f);
      if (DI >= 0 && ty > 0) {  // owned nodes only: no read left of the box
        const float* e0 = el - kPBoxX - 1;
        if (tx > 0) es.x = (e0[0] + e0[1]) + (e0[kPBoxX] + e0[kPBoxX + 1]);
        es.y = (e0[32] + e0[33]) + (e0[kPBoxX + 32] + e0[kPBoxX + 33]);
      }
    };
    // one stage per layer: wait, read, compute, exchange, barrier, refill,
    // epilogue.  (Reading stage t+1 before the barrier, to overlap its latency
    // with the exchange, measured slower: it spills at the 128-register cap.)
    PairColumn col;
    float2 top[2][2][3], E, es, es_prev;
    load_stage(0, top, E, es_prev);
    pair_seed(col, top);
    __syncthreads();  // stage 0 read everywhere; the previous segment's exchange slots retired
    if (tid == 0 && kPairStages < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(kPairStages);
    }
#pragma unroll 2
    for (int t = 1; t < nst; ++t) {
      load_stage(t, top, E, es);
      const float2 nE = make_float2(-E.x, -E.y);
      float2 plane[3][4], ctr[3];
      pair_layer(col, top, E, nE, kc, plane, ctr);
      float2 n0[3];
      float2(*xb)[kPairTY][kPairTX] = xch[t & 1];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float r1a = __shfl_sync(0xffffffffu, plane[c][1].x, src);
        const float r1b = __shfl_sync(0xffffffffu, plane[c][1].y, src);
        const float r3a = __shfl_sync(0xffffffffu, plane[c][3].x, src);
        const float r3b = __shfl_sync(0xffffffffu, plane[c][3].y, src);
        n0[c] = padd(plane[c][0], make_float2(r1a, tx > 0 ? r1b : r1a));
        xb[c][ty][tx] = padd(plane[c][2], make_float2(r3a, tx > 0 ? r3b : r3a));
      }
      __syncthreads();
      // the slot this barrier retires: stage t's (its node data is read), or
      // with staged operands stage t-1's (its epilogue, before this barrier,
      // was the last reader; stage 0's slot was refilled after the seed)
      const int freed = NA > 0 ? t - 1 : t;
      if (tid == 0 && freed >= 1 && freed + kPairStages < nst) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(freed + kPairStages);
      }
      const int ez = kb - 2 + t;
      if (ty > 0 && t >= 2) {
        float res[2][3], cc[2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 r = padd(n0[c], xb[c][ty - 1][tx]);
          res[0][c] = r.x;
          res[1][c] = r.y;
          cc[0][c] = ctr[c].x;
          cc[1][c] = ctr[c].y;
        }
        const int ii[2] = {exA, exA + 32};
        const long long oo[2] = {oA, oA + 32};
        const bool own[2] = {ownA, ownB};
        float av[epi_slots<Epi>()][2][3];
        const float* ap = stg + ((gs + t) % kPairStages) * SF + kPStageFloats +
                          (ty - 1) * kPBoxX + lx;
#pragma unroll
        for (int q = 0; q < NA; ++q)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            av[q][0][c] = ap[q * kPAuxStride + c * (kPAuxY * kPBoxX)];
            av[q][1][c] = ap[q * kPAuxStride + c * (kPAuxY * kPBoxX) + 32];
          }
        if constexpr (DI >= 0) {  // D^-1 of the masked operator, 1 where no stiffness
          const float sa = es_prev.x + es.x, sb = es_prev.y + es.y;
          const float da = sa > 0.f ? jacobi_rcp(kc.kdiag * sa) : 1.0f;
          const float db = sb > 0.f ? jacobi_rcp(kc.kdiag * sb) : 1.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            av[DI][0][c] = da;
            av[DI][1][c] = db;
          }
        }
        if (clean)
          part += epi.template finish<2>(ii, ey, ez, oo, own, res, cc, av, fd);
        else
          part += epi.template finish<2>(ii, ey, ez, oo, own, res, cc, av, d);
        oA += d.plane_stride();
      }
      es_prev = es;
    }
    gs += nst;
    // the next segment's prologue refills every slot, this segment's last
    // operand planes included: their readers must be done
    if (NA > 0) __syncthreads();
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red, blockIdx.x, gridDim.x);
  }
}

bool pair_maps(const float* x, const float* E, const Dims& d, const Bat& bt, CUtensorMap* xmap,
               CUtensorMap* emap);
bool pair_aux_map(const float* v, const Dims& d, const Bat& bt, CUtensorMap* map);

// CTAs per design of the paired kernel: one resident wave over the designs
// of the launch (two CTAs per SM), at least 4 node planes of work each, and
// no more than the partial-sum slots.  (Measured: 123 us at 320x160x160 and
// 35.0 us at 192x96x96, against 133 and 37.1 us for whole-tile z-chunks.)
inline int pair_ctas(const Dims& d, int nb = 1) {
  const long long W = (long long)((d.nx + kPairOwnX) / kPairOwnX) *
                      ((d.ny + kPairOwnY) / kPairOwnY) * (d.nz + 1);
  long long g = 152LL * kPairCtasPerSm / nb;
  g = std::min(g, W / 4);
  g = std::min<long long>(g, kMaxPartials);
  return (int)std::max(1LL, g);
}

template <class Epi>
cudaError_t launch_modal_pair(const CUtensorMap& xm, const CUtensorMap& em, const Dims& d,
                              const ModalCoef<float>& kc, const Epi& epi, const Red& red,
                              const int* done, int* errflag, cudaStream_t s, const Bat& bt) {
  constexpr size_t smem = pair_smem(epi_staged<Epi>());
  static bool attr = false;  // per instantiation; setting it twice is harmless
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_modal_pair<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  CUtensorMap am[2];
  std::memset(am, 0, sizeof(am));
  for (int q = 0; q < epi_staged<Epi>(); ++q)
    if (!pair_aux_map(epi.aux(q), d, bt, &am[q])) return cudaErrorInvalidValue;
  const int gx = (d.nx + kPairOwnX) / kPairOwnX, gy = (d.ny + kPairOwnY) / kPairOwnY;
  dim3 block(kPairTX, kPairTY, 1);
  dim3 grid(pair_ctas(d, bt.nb), 1, bt.nb);
  return launch_pdl(k_modal_pair<Epi>, grid, block, smem, s, xm, em, am[0], am[1], d,
                    pair_coef(kc), epi, red, gx, gy, bt.sel(), done, errflag);
}

// Smallest nx for which the automatic form picks the paired kernel.  Measured
// on GB300 (one plain FP32 application, inputs above L2): 96x32x32 10.3 us
// one-column; 192x96x96 35.0 us paired vs 41.2 us one-column; 320x160x160
// 123 us vs 145 us.
constexpr int kPairAutoMinNx = 150;

// The operator launch of both modal forms: the paired kernel where it is
// selected and the grid is wide enough for its boxes (px, ex >= 68), the
// one-column kernels otherwise.
template <typename T, class Epi>
cudaError_t launch_modal(const T* x, const T* E, const Dims& d, const ModalCoef<T>& kc,
                         const Epi& epi, const Red& red, const int* done, int* errflag,
                         cudaStream_t s, const Bat& bt = Bat{}, T* energy = nullptr) {
  if constexpr (sizeof(T) == 4) {
    CUtensorMap xm, em;
    const bool want = kc.form == 2 || (kc.form == 0 && d.nx >= kPairAutoMinNx);
    if (want && pair_maps(x, E, d, bt, &xm, &em))
      return launch_modal_pair<Epi>(xm, em, d, kc, epi, red, done, errflag, s, bt);
  }
  return launch_modal_single<T, Epi>(x, E, d, kc, epi, red, done, errflag, s, bt, energy);
}

}  // namespace topo
