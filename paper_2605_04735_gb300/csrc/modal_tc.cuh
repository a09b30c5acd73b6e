// Element-centric application of the SIMP stiffness operator with the
// element products K0 U_e on the fifth-generation tensor cores (tcgen05).
//
// The k_e = E_e k0 product of Sec. 2.1.2 (Eq. (3)) is, over a layer of
// elements, a dense GEMM: the 128 elements of a CTA's tile are the M = 128
// rows of A (each row the element's 24 nodal values, shifted by its corner 0
// so that large rigid displacements never meet in one sum; k0 annihilates the
// shift), B is k0 (N = 24 padded to 32, K = 24 = three MMA K-steps of 8 in
// TF32), and D = A B^T lands in tensor memory (TMEM, 32 columns x 128 lanes,
// one lane per element).  One elected thread issues the MMAs; their
// completion is tracked by an mbarrier (tcgen05.commit); every thread then
// reads its element's 24 results from its TMEM lane (tcgen05.ld), scales
// them by E_e and combines them into node sums exactly as the SIMT modal
// kernel does (register carry in z, warp shuffle in x, a shared-memory slot
// in y): no atomics, a node owned by one thread.
//
// Precision: PASSES = 1 is a single TF32 product (k0 and the shifted values
// rounded to TF32: ~2^-11 relative), for the multigrid smoother, which only
// has to be an approximation; PASSES = 2 splits the values into a TF32 high
// part and an FP32 remainder (hi*k0 + lo*k0, k0 in TF32): the exact product
// with a TF32-rounded k0, linear in the values; PASSES = 3 splits both
// operands and accumulates hi*hi + hi*lo + lo*hi (~2^-21 relative, FP32
// level), for the CG operator and residuals.
//
// Work split and data movement are those of k_modal_tma (modal.cuh): a CTA
// is kTcTX x kTcTY = 16 x 8 threads, thread (tx, ty) owns the element column
// (x0-1+tx, y0-1+ty, *) and marches up in z; node and element planes (and the
// epilogue's operand planes) stream through the same 4-stage TMA ring with
// bounded mbarrier waits.  The A tile (and its low part) and the k0 tile sit
// in shared memory in the no-swizzle K-major layout of the MMA (8-row x
// 16-byte core matrices; 128 B between core matrices along K, 768 B between
// 8-row groups).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "modal.cuh"
#include "tma.cuh"

namespace topo {

constexpr int kTcTX = kModalTX;  // 16: must equal the exchange's x tile
constexpr int kTcTY = 8;         // 16 x 8 = 128 threads = the MMA's M
static_assert(kTcTX * kTcTY == 128, "one MMA row per thread");
// TF32 passes of the smoother's operator (1: one pass; 2: values split, the
// linear form)
#ifndef TOPO_TC_SMOOTH_PASSES
#define TOPO_TC_SMOOTH_PASSES 1
#endif
constexpr int kTcN = 32;          // MMA N (24 results padded)
constexpr int kTcCols = 32;       // TMEM columns allocated per CTA
constexpr uint32_t kTcIdesc =     // kind::tf32: D f32, A/B tf32, K-major, N = 32, M = 128
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((128u >> 4) << 24);

// float offset of (row, k) in a no-swizzle K-major tile with 24 K values
__host__ __device__ constexpr int tc_koff(int row, int k) {
  return (row >> 3) * 192 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

// shared-memory matrix descriptor (tcgen05): start, leading (K) and stride
// (8-row group) byte offsets, fixed field 0b001 at bit 46, no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ float to_tf32(float v) {
  float r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D (TMEM) (+)= A B^T for one 8-deep K step
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc ? 1u : 0u)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// this warp's 32 lanes, columns [col, col + 16) and [col + 16, col + 24)
__device__ __forceinline__ void tc_ld24(uint32_t taddr, float (&v)[24]) {
  uint32_t r[24];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                 "=r"(r[22]), "=r"(r[23])
               : "r"(taddr + 16u));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 24; ++q) v[q] = __uint_as_float(r[q]);
}

// k0 in the corner order b = dx + 2 dy + 4 dz of the tensor-core kernels
// (row and column 3 b + c), FP32
struct TcK0 {
  float v[24 * 24];
};

// Shared memory of the tensor-core kernel beyond MTile<kTcTY>: the A tile
// (PASSES == 3: its high and low parts), the k0 tile(s), the MMA barrier and
// the TMEM address.
template <int PASSES>
struct TcSmem {
  static constexpr int ATile = 128 * 24;            // floats
  static constexpr int BTile = kTcN * 24;           // floats
  static constexpr int NP = PASSES >= 2 ? 2 : 1;    // parts (high, low)
  static constexpr size_t bytes() {
    return sizeof(float) * (NP * ATile + NP * BTile) + 16 + 128;  // + barrier, slot, alignment
  }
};

// One element layer per iteration: read the stage, write the A rows, one
// CTA barrier, the elected thread issues the MMAs and commits them to the
// MMA barrier, everyone waits for it and reads its row of D from TMEM, then
// the node-plane sums, the neighbour exchange (the second barrier) and the
// epilogue.  (A software-pipelined variant that wrote layer t+1's rows into
// a second A buffer while layer t's MMA ran, with two TMEM accumulators and
// one barrier per layer, measured slower: 301 against 220 us for the
// three-pass CG operator on 320x160x160, the extra 12-24 KB of shared memory
// and the one-stage-deeper TMA read-ahead costing more than the MMA latency
// it hid.)
template <class Epi, int PASSES>
__global__ void __launch_bounds__(128)
    k_tc_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap emap,
             const __grid_constant__ CUtensorMap amap0, const __grid_constant__ CUtensorMap amap1,
             const Dims d, const __grid_constant__ TcK0 k0, const float kdiag, const Epi epi0,
             const Red red0, const int zchunk, const int zc, const DSel S,
             const int* __restrict__ done, int* __restrict__ errflag) {
  constexpr int TY = kTcTY;
  constexpr int NA = epi_staged<Epi>();  // staged operand vectors
  constexpr int DI = Epi::kDinvAux;      // >= 0: D^-1 formed from the moduli
  static_assert(NA <= 2, "at most two staged operand vectors");
  static_assert(DI < 0 || DI == Epi::kAux - 1, "D^-1 is the last operand");
  using Tl = MTile<TY>;
  using Ts = TcSmem<PASSES>;
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
  unsigned char* base = modal_dyn + ((128u - (smem_u32(modal_dyn) & 127u)) & 127u);
  float* stg = reinterpret_cast<float*>(base);
  auto xch = reinterpret_cast<float(*)[TY][kModalTX][3]>(base + sizeof(float) * SF * kModalStages);
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(base + sizeof(float) * SF * kModalStages + Tl::XchBytes);
  // tensor-core tiles after the ring, the exchange slots and the ring barriers
  unsigned char* tcb = reinterpret_cast<unsigned char*>(bar + kModalStages);
  tcb += (128u - (smem_u32(tcb) & 127u)) & 127u;
  float* sa = reinterpret_cast<float*>(tcb);         // A: part p at p ATile
  float* sb = sa + Ts::NP * Ts::ATile;               // k0: part p at p BTile
  uint64_t* mma_bar = reinterpret_cast<uint64_t*>(sb + Ts::NP * Ts::BTile);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_bar + 1);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kModalTX + tx;
  const int warp = tid >> 5;
  const int x0 = blockIdx.x * kModalOwnX, y0 = blockIdx.y * Tl::OwnY;
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const int bx = x0 & ~3;  // 16-byte aligned box start (storage x of node x0-1 is x0)
  const int ox = x0 - bx;
  const int kb = chunk * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const int nst = (ke - kb) + 2;  // stage t: node plane kb-2+t+1, element layer kb-2+t
  if (warp == 0) {  // the accumulator: 32 TMEM columns (one warp allocates)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"((uint32_t)kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < kModalStages; ++q) mbar_init(&bar[q], 1);
    mbar_init(mma_bar, 1);
    fence_mbar_init();
    tma_prefetch_desc(&xmap);
    tma_prefetch_desc(&emap);
    if (NA > 0) tma_prefetch_desc(&amap0);
    if (NA > 1) tma_prefetch_desc(&amap1);
  }
  // the k0 tile(s): rows n < 24 hold k0's row n, rows 24..31 zero
  for (int q = tid; q < Ts::BTile; q += 128) {
    const int n = q / 24, k = q - 24 * (q / 24);
    const float v = n < 24 ? k0.v[24 * n + k] : 0.0f;
    const float hi = PASSES >= 2 ? to_tf32(v) : v;
    sb[tc_koff(n, k)] = hi;
    if (PASSES >= 2) sb[Ts::BTile + tc_koff(n, k)] = v - hi;
  }
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
  tc_fence_before();
  __syncthreads();  // barriers and the TMEM address set before anyone uses them
  if (tid == 0)
    for (int t = 0; t < kModalStages && t < nst; ++t) issue(t);
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
  const bool own = tx > 0 && ty > 0 && ex <= d.nx && ey <= d.ny;
  const bool clean = !d.box_may_fix(x0, x0 + kModalOwnX - 1, y0, kb);
  const FreeDims fd{d.comp};
  float part = 0.f;
  float es_prev = 0.f;
  auto read_stage = [&](int r, uint32_t ph, float(&top)[2][2][3], float& E, float& es) {
    mbar_wait_bounded(&bar[r], ph, errflag);
    const float* nd = stg + r * SF;
    es = 0.f;
    if (DI >= 0) {  // used by owned nodes only; the others read inside the stage too
      const float* e0 = nd + Tl::ElemOff + (ty - 1) * kMBoxX + ox + tx - 1;
      es = (e0[0] + e0[1]) + (e0[kMBoxX] + e0[kMBoxX + 1]);
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
  float bot[2][2][3];  // raw values of the element's bottom node plane
  float carry[3][4];   // the previous element's top-face results (E-scaled)
  {  // the first node plane only seeds the march
    float E;
    read_stage(0, 0u, bot, E, es_prev);
    __syncthreads();
    if (tid == 0 && kModalStages < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(kModalStages);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int v = 0; v < 4; ++v) carry[c][v] = 0.f;
  }
  const long long o_col = d.node(ex, ey, 0), ps = d.plane_stride();
  int rs = 1;
  uint32_t phase = 0u, mphase = 0u;
  const uint32_t sa_u = smem_u32(sa), sb_u = smem_u32(sb);
  for (int t = 1; t < nst; ++t) {
    const float* nd = stg + rs * SF;
    float top[2][2][3], E, es;
    read_stage(rs, phase, top, E, es);
    // this thread's A row: corners b = dx + 2 dy + 4 dz minus corner 0
    float ctr[3];
    {
      float a[24];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ctr[c] = bot[0][0][c];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          a[3 * v + c] = bot[v >> 1][v & 1][c] - ctr[c];
          a[3 * (4 + v) + c] = top[v >> 1][v & 1][c] - ctr[c];
        }
      }
#pragma unroll
      for (int kc = 0; kc < 6; ++kc) {
        float4 h = make_float4(a[4 * kc], a[4 * kc + 1], a[4 * kc + 2], a[4 * kc + 3]);
        if (PASSES >= 2) {
          const float4 v = h;
          h = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
          *reinterpret_cast<float4*>(sa + Ts::ATile + tc_koff(tid, 4 * kc)) =
              make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
        *reinterpret_cast<float4*>(sa + tc_koff(tid, 4 * kc)) = h;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {  // D = A k0^T: three K-steps per pass (hi hi, hi lo, lo hi)
      tc_fence_after();
      const uint32_t ah = sa_u, al = sa_u + 4u * Ts::ATile;
      const uint32_t bh = sb_u, bl = sb_u + 4u * Ts::BTile;
#pragma unroll
      for (int p = 0; p < PASSES; ++p) {  // 1: hi hi; 2: + lo hi; 3: + hi lo, lo hi
        const uint32_t pa = (PASSES == 2 ? p == 1 : p == 2) ? al : ah;
        const uint32_t pb = (PASSES == 3 && p == 1) ? bl : bh;
#pragma unroll
        for (int s = 0; s < 3; ++s)
          tc_mma(tmem, tc_sdesc(pa + 256u * s, 128u, 768u), tc_sdesc(pb + 256u * s, 128u, 768u),
                 p > 0 || s > 0);
      }
      tc_commit(mma_bar);
    }
    mbar_wait_bounded(mma_bar, mphase, errflag);
    mphase ^= 1u;
    tc_fence_after();
    float y[24];
    tc_ld24(tlane, y);
    tc_fence_before();  // this thread's reads precede the next MMA (after the barriers below)
    // node-plane sums: this element's bottom face plus the previous one's top face
    float plane[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        plane[c][v] = fmaf(E, y[3 * v + c], carry[c][v]);
        carry[c][v] = E * y[3 * (4 + v) + c];
      }
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) bot[dy][dx][c] = top[dy][dx][c];
    const int ez = kb - 2 + t;
    float res[3];
    modal_exchange<float>(plane, xch[t & 1], tx, ty, res);
    // the slot the exchange barrier retires (as in k_modal_tma)
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
        const float dv = sum > 0.f ? jacobi_rcp(kdiag * sum) : 1.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) av[DI][0][c] = dv;
      }
      if (clean)
        part += epi.template finish<1>(ii, ey, ez, oo, ow, rr, cc, av, fd);
      else
        part += epi.template finish<1>(ii, ey, ez, oo, ow, rr, cc, av, d);
    }
    es_prev = es;
    if (++rs == kModalStages) {
      rs = 0;
      phase ^= 1u;
    }
  }
  // release the accumulator once every thread's last read is done
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)kTcCols)
                 : "memory");
  }
  if (Epi::kReduce) {
    double v[1] = {(double)part};
    reduce_finalize<1>(v, red, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * chunk),
                       gridDim.x * gridDim.y * zc);
  }
}

// Build the corner-ordered k0 of the tensor-core kernels from the library's
// local-node order (lidx: (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) ...).
inline TcK0 tc_k0(const K0<float>& k0) {
  auto lidx = [](int b) {  // corner b = dx + 2 dy + 4 dz -> local node
    const int dx = b & 1, dy = (b >> 1) & 1, dz = b >> 2;
    return 4 * dz + (dy ? (dx ? 2 : 3) : (dx ? 1 : 0));
  };
  TcK0 t{};
  for (int b = 0; b < 8; ++b)
    for (int c = 0; c < 3; ++c)
      for (int b2 = 0; b2 < 8; ++b2)
        for (int c2 = 0; c2 < 3; ++c2)
          t.v[24 * (3 * b + c) + 3 * b2 + c2] = k0.v[24 * (3 * lidx(b) + c) + 3 * lidx(b2) + c2];
  return t;
}

// Launch over the grid (one design, or the designs of a mesh group); false
// in *launched when the TMA boxes do not fit the grid (the caller falls back
// to the SIMT kernels).
template <class Epi, int PASSES>
cudaError_t launch_tc_tma(const float* x, const float* E, const Dims& d, const K0<float>& k0f,
                          const Epi& epi, const Red& red, const int* done, int* errflag,
                          cudaStream_t s, const Bat& bt, bool* launched) {
  *launched = false;
  CUtensorMap xm, em, am[2];
  std::memset(am, 0, sizeof(am));
  bool ok = modal_maps(x, E, d, bt, kTcTY, &xm, &em);
  for (int q = 0; q < epi_staged<Epi>() && ok; ++q)
    ok = modal_aux_map(epi.aux(q), d, bt, kTcTY, &am[q]);
  if (!ok) return cudaSuccess;
  constexpr size_t smem = MTile<kTcTY>::smem(epi_staged<Epi>()) + TcSmem<PASSES>::bytes();
  static bool attr = false;  // per instantiation; setting it twice is harmless
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_tc_tma<Epi, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int z = modal_zchunk(d, bt.nb, kTcTY - 1);
  const int zc = (d.nz + z) / z;
  dim3 block(kModalTX, kTcTY, 1);
  dim3 grid((d.nx + kModalOwnX) / kModalOwnX, (d.ny + kTcTY - 1) / (kTcTY - 1), zc * bt.nb);
  *launched = true;
  return launch_pdl(k_tc_tma<Epi, PASSES>, grid, block, smem, s, xm, em, am[0], am[1], d,
                    tc_k0(k0f), k0f.v[0], epi, red, z, zc, bt.sel(), done, errflag);
}

}  // namespace topo

namespace topo {

// The operator launch of the modal forms with the tensor-core form among
// them: kc.form == 3 runs k_tc_tma with PASSES TF32 passes where its boxes
// fit the grid (FP32 only), the SIMT modal kernels otherwise.
template <int PASSES, typename T, class Epi>
cudaError_t launch_modal_any(const T* x, const T* E, const Dims& d, const ModalCoef<T>& kc,
                             const K0<T>& k0, const Epi& epi, const Red& red, const int* done,
                             int* errflag, cudaStream_t s, const Bat& bt = Bat{},
                             T* energy = nullptr) {
  if constexpr (sizeof(T) == 4) {
    if (kc.form == 3 && !energy) {
      bool launched = false;
      const cudaError_t e =
          launch_tc_tma<Epi, PASSES>(x, E, d, k0, epi, red, done, errflag, s, bt, &launched);
      if (e != cudaSuccess || launched) return e;
    }
  }
  return launch_modal<T>(x, E, d, kc, epi, red, done, errflag, s, bt, energy);
}

}  // namespace topo
