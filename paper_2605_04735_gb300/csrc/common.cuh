// Shared device-side definitions of the SIMP state-solve library.
//
// Data layout in HBM (one mesh, one grid level):
//   * vectors (displacement-like, 3 components) are SoA: component c lives at
//     c * comp_stride; inside a component, node (i, j, k) with -1 <= i <= nx+1
//     etc. is at (i+1) + px * ((j+1) + (ny+3) * (k+1)).  The ring i = -1,
//     i = nx+1 (and likewise in j, k) is a ghost layer that always holds 0, so
//     the 27-node gather never needs a bounds test, and px (a multiple of 4)
//     keeps every row 16-byte aligned;
//   * element arrays (E, rho) use the same idea with one ghost layer:
//     element (i, j, k), -1 <= i <= nx, at (i+1) + ex * ((j+1) + (ny+2) * (k+1)),
//     ghost elements hold E = 0, so they contribute nothing.
//   Every vector entry of a fixed (Dirichlet) DOF is kept at 0 by all
//   kernels, which is what lets the operator skip input masking.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace topo {

enum Bc {
  BC_CANTILEVER = 0,
  BC_MBB = 1,
  BC_ROLLER_BOX = 2,
  BC_CORNERS = 3,
  BC_MBB_STRIP = 4,
  BC_NONE = 5  // no support: a slab of a larger grid (operator applications only)
};

// k0 as a kernel parameter: 24x24 row-major, unit Young's modulus.  Read
// with compile-time indices only, so every access is a constant-bank
// operand of the FMA that uses it.
template <typename T>
struct K0 {
  T v[576];
};

struct Dims {
  int nx, ny, nz;    // elements per direction
  int px;            // node row pitch (entries), >= nx + 3, multiple of 4
  int ex;            // element row pitch, >= nx + 2, multiple of 4
  int bc;            // Bc
  int pin_j;         // MBB: j index of the single u_y pin (ny / 2)
  int corner_j;      // BC_CORNERS: supported rows j <= corner_j or j >= ny - corner_j
  int corner_k;      //             and layers k <= corner_k or k >= nz - corner_k
  long long comp;    // entries per vector component = px * (ny+3) * (nz+3)
  long long ecount;  // entries of an element array = ex * (ny+2) * (nz+2)
  __host__ __device__ long long node(int i, int j, int k) const {
    return (long long)(i + 1) + (long long)px * ((j + 1) + (long long)(ny + 3) * (k + 1));
  }
  __host__ __device__ long long elem(int i, int j, int k) const {
    return (long long)(i + 1) + (long long)ex * ((j + 1) + (long long)(ny + 2) * (k + 1));
  }
  __host__ __device__ long long row_stride() const { return px; }
  __host__ __device__ long long plane_stride() const { return (long long)px * (ny + 3); }
  __host__ __device__ long long erow() const { return ex; }
  __host__ __device__ long long eplane() const { return (long long)ex * (ny + 2); }
  // May a DOF of a node with i in [i0, i1], j >= j0, k >= k0 be fixed?
  // (Conservative: false only when no such node is on a support.)
  __host__ __device__ bool box_may_fix(int i0, int i1, int j0, int k0) const {
    switch (bc) {
      case BC_CANTILEVER:
      case BC_CORNERS:
        return i0 <= 0;
      case BC_MBB:
        return i0 <= 0 || (i1 >= nx && k0 <= 0);
      case BC_MBB_STRIP:
        return i0 <= 0 || (i1 >= nx - 1 && k0 <= 0);
      case BC_NONE:
        return false;
      default:
        return i0 <= 0 || j0 <= 0 || k0 <= 0;
    }
  }
  // Is DOF c of node (i, j, k) held at zero?
  __host__ __device__ bool fixed(int c, int i, int j, int k) const {
    switch (bc) {
      case BC_CANTILEVER:
        return i == 0;
      case BC_MBB:
        return (c == 0 && i == 0) || (c == 2 && i == nx && k == 0) ||
               (c == 1 && i == nx && k == 0 && j == pin_j);
      case BC_CORNERS:
        return i == 0 && (j <= corner_j || j >= ny - corner_j) &&
               (k <= corner_k || k >= nz - corner_k);
      case BC_MBB_STRIP:
        return (c == 0 && i == 0) || (c == 2 && i >= nx - 1 && k == 0) ||
               (c == 1 && i == nx && k == 0 && j == pin_j);
      case BC_NONE:
        return false;
      default:
        return (c == 0 && i == 0) || (c == 1 && j == 0) || (c == 2 && k == 0);
    }
  }
};

// A view of Dims for a region that holds no fixed DOF: the epilogues skip
// their support test.
struct FreeDims {
  long long comp;
  __device__ __forceinline__ bool fixed(int, int, int, int) const { return false; }
};

// Layout of a grid of nx*ny*nz elements (pitches padded to 4 entries).
inline Dims make_dims(int nx, int ny, int nz, int bc, int pin_j) {
  Dims d{};
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.px = ((nx + 3) + 3) / 4 * 4;
  d.ex = ((nx + 2) + 3) / 4 * 4;
  d.bc = bc;
  d.pin_j = pin_j;
  // paper Sec. 4.2: 0.3 x 0.3 corner squares of the unit cross-section
  d.corner_j = (int)(0.3 * ny + 1e-9);
  d.corner_k = (int)(0.3 * nz + 1e-9);
  d.comp = (long long)d.px * (ny + 3) * (nz + 3);
  d.ecount = (long long)d.ex * (ny + 2) * (nz + 2);
  return d;
}

// Device-resident scalars of one preconditioned CG run.  All decisions
// (alpha, beta, convergence) are taken on the device, so the host only reads
// this struct once per chunk of iterations.
struct PcgScalars {
  double rz;      // r . z of the current iterate
  double pq;      // p . A p
  double alpha, beta;
  double rr;      // r . r of the current iterate (recursive residual)
  double rr0;     // r . r at the start
  double tol2;    // stop when rr <= tol2
  double aux[4];  // results of stand-alone reductions (dots, norms)
  int iter;       // iterations done
  int max_iter;   // stop (not converged) when iter reaches it
  int done;       // 1: converged or stopped; every loop kernel returns at once
  int status;     // 0 ok, 1 hit max_iter, 2 breakdown / non-finite
  unsigned counter[8];  // last-block counters of the reductions (reset by the last block)
  // per-design settings of the next inner solve, written by the host for
  // batched solves (FIN_INIT with a negative launch tolerance reads rtol2_next;
  // rtol2_next >= 1 finishes the inner solve at once: the design sits out,
  // and sat_out = 1 lets the batched refinement kernels skip it: its u and
  // FP64 residual stay as they are)
  double rtol2_next;
  int max_iter_next;
  int sat_out;
  // the refinement residual of a batched outer step: in double-word
  // arithmetic for some designs, in FP64 for the others; each launch skips
  // the designs whose flag is set
  int skip_dword;
  int skip_fp64;
};

// The designs of a batched launch, as kernels see them: grid slot b (a grid
// dimension) runs design id(b), whose buffers sit at id(b) * S bytes from
// design 0's; ids == nullptr means slot b is design b.
struct DSel {
  long long S;
  const int* ids;
  __device__ __forceinline__ int id(int b) const { return ids ? __ldg(ids + b) : b; }
  __device__ __forceinline__ long long off(int b) const { return (long long)id(b) * S; }
};

// A batch of designs with identical grids whose buffers sit at a fixed byte
// stride S from design 0's (the designs of a mesh group share one arena): a
// kernel launched for nb designs offsets every pointer by design * S.  With
// ids (device, nb entries) the launch covers only the listed designs of a
// group of ntot (the TMA maps span all ntot designs).
struct Bat {
  int nb = 1;
  long long S = 0;
  const int* ids = nullptr;
  int ntot = 0;
  DSel sel() const { return DSel{S, ids}; }
  int designs() const { return ntot > 0 ? ntot : nb; }
};

template <typename T>
__host__ __device__ __forceinline__ T* bshift(T* p, long long off) {
  return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<void*>(
                 static_cast<const void*>(p))) + off)
           : p;
}

enum FinalizeOp {
  FIN_NONE = 0,
  FIN_ALPHA = 1,     // v0 = p.q           -> alpha = rz / pq
  FIN_UPDATE = 2,    // v0 = r.z, v1 = r.r -> beta, iter++, convergence test
  FIN_INIT = 3,      // v0 = r.z, v1 = r.r -> start values, tol2
  FIN_AUX = 4,       // v0.. -> aux[0..]
  FIN_RR_ONLY = 5,   // v0 = r.r           -> rr (used before a separate z = M r)
  FIN_RZ_BETA = 6,   // v0 = r.z           -> beta, iter++, convergence test on rr
  FIN_SET_RZ = 7     // v0 = r.z           -> rz, beta = 0 (first direction p = z)
};

constexpr int kMaxPartials = 16384;  // block partials per reduced value

struct Red {
  double* partials;   // [NV][kMaxPartials]
  PcgScalars* sc;
  int slot;           // which counter
  int op;             // FinalizeOp
  double rtol2;       // FIN_INIT: relative tolerance squared (< 0: sc->rtol2_next)
  __host__ __device__ Red shifted(long long off) const {
    Red r = *this;
    r.partials = bshift(partials, off);
    r.sc = bshift(sc, off);
    return r;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void finalize(const Red& red, const double* tot, int nv) {
  PcgScalars* s = red.sc;
  switch (red.op) {
    case FIN_ALPHA: {
      s->pq = tot[0];
      double a = s->rz / tot[0];
      if (!(tot[0] > 0.0) || !isfinite(a)) {  // breakdown: stop with status 2
        s->status = 2;
        s->done = 1;
        a = 0.0;
      }
      s->alpha = a;
      break;
    }
    case FIN_UPDATE:
    case FIN_RZ_BETA: {
      double rz_new = tot[0];
      if (red.op == FIN_UPDATE && nv > 1) s->rr = tot[1];
      s->beta = rz_new / s->rz;
      s->rz = rz_new;
      s->iter += 1;
      if (!isfinite(s->rr) || !isfinite(rz_new) || !(rz_new > 0.0)) {
        s->status = 2;
        s->done = 1;
      } else if (s->rr <= s->tol2) {
        s->done = 1;
      } else if (s->iter >= s->max_iter) {
        s->status = 1;
        s->done = 1;
      }
      break;
    }
    case FIN_INIT: {
      const double rt2 = (red.rtol2 >= 0.0) ? red.rtol2 : s->rtol2_next;
      s->rz = tot[0];
      s->rr = tot[nv - 1];
      s->rr0 = tot[nv - 1];
      s->tol2 = rt2 * tot[nv - 1];
      s->iter = 0;
      s->status = 0;
      s->done = (tot[nv - 1] <= 0.0 || rt2 >= 1.0) ? 1 : 0;
      break;
    }
    case FIN_AUX:
      for (int q = 0; q < nv && q < 4; ++q) s->aux[q] = tot[q];
      break;
    case FIN_SET_RZ:
      s->rz = tot[0];
      s->beta = 0.0;
      if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
        s->status = 2;
        s->done = 1;
      }
      break;
    case FIN_RR_ONLY:
      s->rr = tot[0];
      if (!isfinite(tot[0])) {
        s->status = 2;
        s->done = 1;
      } else if (tot[0] <= s->tol2) {  // converged: skip the preconditioner
        s->iter += 1;
        s->done = 1;
      }
      break;
    default:
      break;
  }
}

// (i, j, k) of the linear index n = i + X (j + Y k) of an X x Y x Z box, in
// 32-bit unsigned arithmetic (n < 2^32: meshes hold fewer than 2^31 nodes)
__device__ __forceinline__ void unflatten3(long long n, int X, int Y, int& i, int& j, int& k) {
  const unsigned u = (unsigned)n;
  const unsigned t = u / (unsigned)X;
  i = (int)(u - t * (unsigned)X);
  const unsigned kk = t / (unsigned)Y;
  j = (int)(t - kk * (unsigned)Y);
  k = (int)kk;
}

// 1 / x for an FP32 Jacobi diagonal entry (x > 0, a sum of element moduli
// times k0's diagonal: never subnormal).  Every FP32 kernel that forms D^-1
// uses this one function.  By default it is the hardware approximation
// (rcp.approx.ftz: within about one unit in the last place, ample for a
// preconditioner's diagonal), which also spares the correctly rounded
// reciprocal's slow-path branch in the operator epilogues (measured on the
// batched 96x32x32 Chebyshev step: 1-5 % faster); TOPO_FAST_RCP=0 selects
// the correctly rounded one.
#ifndef TOPO_FAST_RCP
#define TOPO_FAST_RCP 1
#endif
__device__ __forceinline__ float jacobi_rcp(float x) {
#if TOPO_FAST_RCP
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return __frcp_rn(x);
#endif
}

// *p += v as a fire-and-forget reduction performed at L2 (no load round trip
// and no register kept for the old value).  Used where one thread owns the
// entry, so the result is the same sum in the same order as a load-add-store
// (round to nearest; subnormal inputs and results flush to zero).
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// Operator epilogues.  An epilogue names kAux operand vectors (aux(q), read
// at the node) and implements finish<N>() over N owned nodes of one plane,
// given the operands in av[q][n][c]; it only stores.  epi_run() loads every
// operand of the N nodes before the first store, so the group costs one
// memory round trip (the compiler must otherwise assume a store may alias
// the next load and serialises them); kernels that stage the operand planes
// in shared memory call finish() directly.  epi_one() runs one node.
template <class Epi>
__host__ __device__ constexpr int epi_slots() {
  return Epi::kAux > 0 ? Epi::kAux : 1;
}

// Operand vectors a TMA kernel stages: all but the Jacobi inverse diagonal
// (Epi::kDinvAux, the last aux when present), which those kernels form from
// the element moduli they already hold: D^-1 = 1 / (kdiag * sum of the 8
// moduli around the node).
template <class Epi>
__host__ __device__ constexpr int epi_staged() {
  return Epi::kAux - (Epi::kDinvAux >= 0 ? 1 : 0);
}

template <class Epi, int N, typename T, class DD>
__device__ __forceinline__ T epi_run(const Epi& e, const int (&i)[N], int j, int k,
                                     const long long (&o)[N], const bool (&own)[N],
                                     const T (&acc)[N][3], const T (&ctr)[N][3], const DD& d) {
  T av[epi_slots<Epi>()][N][3];
#pragma unroll
  for (int q = 0; q < Epi::kAux; ++q)
#pragma unroll
    for (int n = 0; n < N; ++n)
      if (own[n])
#pragma unroll
        for (int c = 0; c < 3; ++c) av[q][n][c] = e.aux(q)[c * d.comp + o[n]];
  return e.template finish<N>(i, j, k, o, own, acc, ctr, av, d);
}

template <class Epi, typename T, class DD>
__device__ __forceinline__ T epi_one(const Epi& e, int i, int j, int k, long long o,
                                     const T (&acc)[3], const T (&ctr)[3], const DD& d) {
  const int ii[1] = {i};
  const long long oo[1] = {o};
  const bool own[1] = {true};
  const T a[1][3] = {{acc[0], acc[1], acc[2]}};
  const T c[1][3] = {{ctr[0], ctr[1], ctr[2]}};
  return epi_run<Epi, 1>(e, ii, j, k, oo, own, a, c, d);
}

// Programmatic dependent launch.  Kernels of the solve path start with
// pdl_start(): wait until the kernel launched before them on the stream has
// completed and its writes are visible (a no-op when there is no programmatic
// dependency), then allow the next kernel to be launched, so its CTAs are
// resident and waiting when this one ends.  launch_pdl() launches a kernel
// with that dependency (stream order otherwise unchanged; kept by graph
// capture).  Every kernel launched with launch_pdl must begin with pdl_start.
__device__ __forceinline__ void pdl_start() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Deterministic block-partial reduction of NV doubles with a last-block
// finalisation: every block writes its partials, the last block to arrive
// sums them in block order (fixed order => bitwise reproducible) and calls
// finalize().  Must be called by every thread of every block.
// Block reduction over the blocks of one design: `bid` in [0, nblocks) is the
// block's number among the design's blocks (the whole grid for one design).
template <int NV>
__device__ __forceinline__ void reduce_finalize(double (&v)[NV], const Red& red, int bid,
                                                int nblocks) {
  __shared__ double sh[NV][32];
  __shared__ bool last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int warp = tid >> 5;
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int nwarps = (nthreads + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double w = warp_sum(v[q]);
    if ((tid & 31) == 0) sh[q][warp] = w;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double acc = 0.0;
      for (int w = 0; w < nwarps; ++w) acc += sh[q][w];
      red.partials[q * kMaxPartials + bid] = acc;
    }
    __threadfence();
    unsigned prev = atomicAdd(&red.sc->counter[red.slot], 1u);
    last = (prev == (unsigned)(nblocks - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double acc = 0.0;
    for (int b = tid; b < nblocks; b += nthreads)
      acc += __ldcg(&red.partials[q * kMaxPartials + b]);
    tot[q] = acc;
  }
  __syncthreads();  // sh reuse
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double w = warp_sum(tot[q]);
    if ((tid & 31) == 0) sh[q][warp] = w;
  }
  __syncthreads();
  if (tid == 0) {
    double fin[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double acc = 0.0;
      for (int w = 0; w < nwarps; ++w) acc += sh[q][w];
      fin[q] = acc;
    }
    finalize(red, fin, NV);
    red.sc->counter[red.slot] = 0u;
    __threadfence();
  }
}

template <int NV>
__device__ __forceinline__ void reduce_finalize(double (&v)[NV], const Red& red) {
  reduce_finalize<NV>(v, red, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                      gridDim.x * gridDim.y * gridDim.z);
}

}  // namespace topo
