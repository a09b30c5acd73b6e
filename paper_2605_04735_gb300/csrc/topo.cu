// Host runtime and C ABI of the SIMP state-solve library (include/topo.h).
//
// The runtime owns one mesh's device state and drives the solver:
//   * FP64 iterative refinement (outer loop): r = f - K u in FP64 on the
//     device, stop when ||r|| / ||f|| <= rtol, else solve K d = r / ||r||
//     approximately with preconditioned CG and set u += ||r|| d;
//   * the inner preconditioned CG runs in FP32 (or, for the plain FP64
//     reference path, in FP64 to the final tolerance in one outer step);
//     alpha, beta and the convergence test are taken on the device, and the
//     host only reads the scalars once every `check_every` iterations.
// The paper (Sec. 2.1.1) states the equilibrium K(rho) U = F but not how it
// is solved; the refinement loop and CG are this library's choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "../../include/topo.h"
#include "common.cuh"
#include "gmg.h"
#include "kernels.h"

using namespace topo;

namespace topo {

// --------------------------------------------------------------------------
// k0 of the unit cube for E = 1 (Sec. 2.1.2), built from exact 1-D integrals
// of the linear hat functions on [0, 1]:
//   K[(a,p),(b,q)] = lam I(a,b; p,q) + mu I(a,b; q,p) + mu delta_pq sum_r I(a,b; r,r),
//   I(a,b; s,t) = int dN_a/dx_s dN_b/dx_t dV = prod over directions of
//   {int N'N', int N'N, int N N', int N N} of the 1-D factors.
// --------------------------------------------------------------------------
void build_k0(double nu, double* k) {
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double M[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};  // int N_a N_b
  const double S[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};                      // int N_a' N_b'
  const double L[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};                      // int N_a' N_b
  static const int loc[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  auto I = [&](int a, int b, int s, int t) {
    double v = 1.0;
    for (int r = 0; r < 3; ++r) {
      const int ia = loc[a][r], ib = loc[b][r];
      if (r == s && r == t)
        v *= S[ia][ib];
      else if (r == s)
        v *= L[ia][ib];
      else if (r == t)
        v *= L[ib][ia];
      else
        v *= M[ia][ib];
    }
    return v;
  };
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
          double v = lam * I(a, b, p, q) + mu * I(a, b, q, p);
          if (p == q) v += mu * (I(a, b, 0, 0) + I(a, b, 1, 1) + I(a, b, 2, 2));
          k[(3 * a + p) * 24 + 3 * b + q] = v;
        }
}

}  // namespace topo

namespace {

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double seconds() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

}  // namespace

struct ChunkGraph {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels in one replay
};

struct MeshGroup;

struct topo_mesh {
  int dev = 0;
  // mesh groups (topo_create_batch): this design's region of the group arena;
  // while region_open, allocations come from the region (fixed order and sizes,
  // so every design's buffer sits at gidx * S bytes from design 0's)
  MeshGroup* group = nullptr;
  int gidx = 0;
  char* region = nullptr;
  long long region_size = 0, region_used = 0;
  bool region_open = false;
  cudaStream_t stream = nullptr;  // the mesh's own non-blocking stream (all work runs here)
  cudaStream_t user = nullptr;    // the caller's stream (NULL = legacy default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // fences between the two
  bool own_stream = false;
  Dims d{};
  topo_params prm{};
  K0<double> k0d{};
  K0<float> k0f{};
  ModalCoef<double> mcd{};  // k0 in the modal basis (element-centric kernels)
  ModalCoef<float> mcf{};
  bool use_modal = true;    // false: node-centric gather kernels
  long long nvec = 0;  // entries of one 3-component vector (3 * comp)

  // element data (ghosted)
  float* rho_g = nullptr;
  float* E32 = nullptr;
  double* E64 = nullptr;
  // FP64 state
  double* f64 = nullptr;
  double* u64 = nullptr;
  double* r64 = nullptr;
  // FP32 inner CG
  float *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr,
        *b32 = nullptr, *dinv32 = nullptr;
  // FP64 inner CG (allocated on first FP64 solve)
  double *x64 = nullptr, *s64 = nullptr, *z64 = nullptr, *p64 = nullptr, *q64 = nullptr,
         *dinv64 = nullptr;
  // scratch
  PcgScalars* sc = nullptr;
  PcgScalars* h_sc = nullptr;  // pinned mirror
  int* h_flag = nullptr;       // pinned mirror of the timeout flag
  cudaEvent_t ev_poll = nullptr;  // marks the arrival of h_sc / h_flag
  double* partials = nullptr;
  int* flags = nullptr;
  double* aos = nullptr;       // n_dof doubles (ABI transfers)
  double* dc = nullptr;        // n_elem doubles
  double* energy = nullptr;    // element energies of u (element layout), by the FP64 residual
  bool energy_fresh = false;   // energy belongs to the current u
  bool e_positive = false;     // every element modulus > 0 (energies are recoverable)
  float* rho_in = nullptr;     // n_elem floats: the current densities, dense element order
  double* phi_in = nullptr;    // n_node doubles: the nodal level set (ersatz material)
  // level-set stage (lazily allocated): second level-set buffer, shape
  // right-hand sides, the extension solve's CG vectors and Dirichlet mask
  double* phi_tmp = nullptr;
  double ls_eta = 1.0, ls_eps0 = 1e-3;
  bool ls_ready = false;       // phi_in holds the level set the moduli came from
  double* ls_part = nullptr;   // 16 n_elem doubles: element shares of bJ, bV
  double* ls_bJ = nullptr;     // n_node doubles each
  double* ls_bV = nullptr;
  double *hx = nullptr, *hr = nullptr, *hz = nullptr, *hp = nullptr, *hq = nullptr,
         *hdinv = nullptr, *hb = nullptr;  // padded to a multiple of 4 nodes
  uint8_t* hdir = nullptr;
  double h_ell2 = -1.0;        // ell^2 the Jacobi diagonal was built for
  unsigned long long* ls_scratch = nullptr;
  double* ls_dt = nullptr;
  // geometry transfer: nodal densities, the last extracted triangle soup
  // (9 doubles per triangle, grouped by cell) and its per-cell offsets
  double* tr_rho_n = nullptr;
  long long* tr_counts = nullptr;
  long long* tr_off = nullptr;
  long long* tr_scratch = nullptr;
  double* tr_tris = nullptr;
  long long tr_cap = 0, tr_n = 0;
  double* dcf = nullptr;       // n_elem doubles: filtered sensitivities
  float* rho_next = nullptr;   // n_elem floats: densities after an OC update
  void* oc_state = nullptr;    // device OC bracketing state
  double* oc_part = nullptr;   // OC block partials
  unsigned char* oc_host = nullptr;  // pinned copy of the OC state

  bool has_density = false, solved = false, diag32 = false, diag64 = false;
  double fnorm2 = 0.0;
  long long bytes = 0;

  bool prof = false;
  std::vector<cudaEvent_t> ev;
  double prof_ms = 0.0;
  long long prof_launches = 0;
  // finest-level Chebyshev steps of the V-cycle (profiling): event pairs,
  // kChebSlots per CG iteration; per slot whether the step stores x; totals
  std::vector<cudaEvent_t> evc;
  int cheb_slots = 0;
  unsigned char cheb_store[16] = {};
  double profc_ms = 0.0, profc_bytes = 0.0;
  long long profc_launches = 0;
  long long launches = 0;  // every kernel this mesh launched

  // captured CG chunks, keyed by (kind, iterations, profiling)
  std::map<long long, ChunkGraph> graphs;

  // multigrid hierarchy (built on the first GMG solve, set up per density)
  Gmg gmg;
  bool gmg_built = false;
  bool throughput = false;  // build the hierarchy in its throughput form
  int gmg_levels_req = -1, gmg_degree = -1;
  double lam_max = 0.0;
};

// A mesh group: designs of one grid, BC, load and material whose solve
// buffers live in one arena, design b's region at b * S bytes from design
// 0's, so one launch with a design index can serve all of them (batched
// solves, topo_solve_many).
struct MeshGroup {
  int nb = 0;
  long long S = 0;
  char* arena = nullptr;
  int refs = 0;
  std::vector<topo_mesh*> meshes;
  std::map<long long, ChunkGraph> graphs;  // batched CG chunks
  PcgScalars* h_sc = nullptr;              // nb pinned host copies
  int* h_flag = nullptr;                   // nb
  struct Next {  // the layout of PcgScalars' tail from rtol2_next on
    double rtol2;
    int max_iter;
    int sat_out;
    int skip_dword;
    int skip_fp64;
  };
  Next* h_next = nullptr;  // nb: per-design settings of the next inner solve
  int* h_ids = nullptr;    // nb pinned: the designs a compacted CG chunk covers
  int* d_ids = nullptr;    // nb: their device copy
  void* stage = nullptr;   // batched host<->device transfers of densities / sensitivities
  size_t stage_bytes = 0;
  // FP64 inner-CG vectors of every design (batched FP64 Jacobi-PCG), made on
  // first use: design b's at arena64 + b * S, so they keep the group stride
  char* arena64 = nullptr;
  long long arena64_bytes = 0;
  int gmg_levels = -1, gmg_degree = -1;
  topo_params prm{};
};

namespace {

topo_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TOPO_OK;
  if (e == cudaErrorMemoryAllocation) return TOPO_ERR_OOM;
  return TOPO_ERR_CUDA;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t err__ = (call);                   \
    if (err__ != cudaSuccess) return cuda_status(err__); \
  } while (0)

template <typename T>
topo_status dalloc(topo_mesh* m, T** p, long long count) {
  const size_t bytes = (size_t)count * sizeof(T);
  if (m->region_open) {  // bump allocation in the group arena (zero-filled at creation)
    const long long off = (m->region_used + 255) / 256 * 256;
    if (off + (long long)bytes > m->region_size) return TOPO_ERR_OOM;
    *p = reinterpret_cast<T*>(m->region + off);
    m->region_used = off + (long long)bytes;
    m->bytes += (long long)bytes;
    return TOPO_OK;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TOPO_ERR_OOM;
  }
  e = cudaMemsetAsync(q, 0, bytes, m->stream);
  if (e != cudaSuccess) {
    cudaFree(q);
    return TOPO_ERR_CUDA;
  }
  *p = static_cast<T*>(q);
  m->bytes += (long long)bytes;
  return TOPO_OK;
}

#define MCD(m) ((m)->use_modal ? &(m)->mcd : nullptr)
#define MCF(m) ((m)->use_modal ? &(m)->mcf : nullptr)

// count one kernel launch of this mesh, then check the launch
#define LK(mesh, call)          \
  do {                          \
    ++(mesh)->launches;         \
    CK(call);                   \
  } while (0)

#define CKS(call)                        \
  do {                                   \
    topo_status st__ = (call);           \
    if (st__ != TOPO_OK) return st__;    \
  } while (0)

Red red_of(topo_mesh* m, int op, double rtol2 = 0.0) {
  Red r{};
  r.partials = m->partials;
  r.sc = m->sc;
  r.slot = 0;
  r.op = op;
  r.rtol2 = rtol2;
  return r;
}

topo_status sync_scalars(topo_mesh* m) {
  CK(cudaMemcpyAsync(m->h_sc, m->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

// Orders a call's work after everything the caller enqueued on its stream
// before the call, and everything the caller enqueues afterwards after it.
struct Fence {
  topo_mesh* m;
  topo_status st = TOPO_OK;
  explicit Fence(topo_mesh* mm) : m(mm) {
    if (cudaSetDevice(m->dev) != cudaSuccess || cudaEventRecord(m->ev_in, m->user) != cudaSuccess ||
        cudaStreamWaitEvent(m->stream, m->ev_in, 0) != cudaSuccess)
      st = TOPO_ERR_CUDA;
  }
  ~Fence() {
    if (cudaEventRecord(m->ev_out, m->stream) == cudaSuccess)
      cudaStreamWaitEvent(m->user, m->ev_out, 0);
  }
  Fence(const Fence&) = delete;
  Fence& operator=(const Fence&) = delete;
};

cudaError_t region_alloc(void* ctx, void** p, size_t bytes) {
  topo_mesh* m = static_cast<topo_mesh*>(ctx);
  const long long off = (m->region_used + 255) / 256 * 256;
  if (off + (long long)bytes > m->region_size) return cudaErrorMemoryAllocation;
  *p = m->region + off;
  m->region_used = off + (long long)bytes;
  return cudaSuccess;
}

topo_status ensure_fp64_inner(topo_mesh* m) {
  if (m->x64) return TOPO_OK;
  CKS(dalloc(m, &m->x64, m->nvec));
  CKS(dalloc(m, &m->s64, m->nvec));
  CKS(dalloc(m, &m->z64, m->nvec));
  CKS(dalloc(m, &m->p64, m->nvec));
  CKS(dalloc(m, &m->q64, m->nvec));
  CKS(dalloc(m, &m->dinv64, m->nvec));
  return TOPO_OK;
}

constexpr int kChebSlots = 16;  // finest-level Chebyshev steps timed per V-cycle (at most)

topo_status ensure_profile_events(topo_mesh* m, int n) {
  while ((int)m->ev.size() < 2 * n) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    m->ev.push_back(e);
  }
  while ((int)m->evc.size() < 2 * kChebSlots * n) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    m->evc.push_back(e);
  }
  return TOPO_OK;
}

// V-cycle timing hook for CG iteration c of a chunk (nullptr when not profiling)
GmgProf* cheb_prof(topo_mesh* m, bool profile, int c, GmgProf& gp) {
  if (!profile) return nullptr;
  gp = GmgProf{};
  gp.ev = m->evc.data() + 2 * kChebSlots * c;
  gp.cap = kChebSlots;
  return &gp;
}

// after capturing one V-cycle with the hook: the per-iteration slot pattern
void cheb_prof_done(topo_mesh* m, const GmgProf* gp) {
  if (!gp) return;
  m->cheb_slots = gp->n;
  for (int q = 0; q < gp->n; ++q) m->cheb_store[q] = gp->store[q];
}

// Add the timed Chebyshev steps of CG iteration c of the last chunk, which
// advanced `designs` designs: durations and algorithmic bytes (per node: the
// direction and residual read, r and the new direction written, x written
// (store) or read and written (add); per element the modulus).
topo_status cheb_prof_collect(topo_mesh* m, int c, int designs) {
  const double nn = (double)(m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
  const double ne = (double)m->d.nx * m->d.ny * m->d.nz;
  for (int q = 0; q < m->cheb_slots; ++q) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, m->evc[2 * (kChebSlots * c + q)],
                            m->evc[2 * (kChebSlots * c + q) + 1]));
    m->profc_ms += ms;
    m->profc_launches += designs;
    m->profc_bytes += designs * ((m->cheb_store[q] ? 60.0 : 72.0) * nn + 4.0 * ne);
  }
  return TOPO_OK;
}

enum InnerKind { IK_JAC32 = 0, IK_JAC64 = 1, IK_GMG32 = 2 };

// An inner FP32 solve that could finish the solve aims at kInnerMargin x the
// target relative residual: the FP32 recursion's residual drifts from the
// true one, and a miss costs a whole further outer step.
constexpr double kInnerMargin = 0.5;

// Enqueue `count` CG iterations of the given kind.  Every kernel returns at
// once when the device-side `done` flag is set, so iterations past
// convergence are no-ops and a chunk can be replayed blindly.
topo_status enqueue_iters(topo_mesh* m, int kind, int count, bool profile) {
  cudaStream_t s = m->stream;
  const int* done = &m->sc->done;
  for (int c = 0; c < count; ++c) {
    if (profile) CK(cudaEventRecordWithFlags(m->ev[2 * c], s, cudaEventRecordExternal));
    if (kind == IK_JAC64) {
      LK(m, launch_apply<double>(m->p64, m->q64, m->E64, nullptr, m->d, m->k0d, MCD(m),
                                 red_of(m, FIN_ALPHA), APPLY_DOT, done, m->flags + 1, s));
    } else {
      LK(m, launch_apply<float>(m->p32, m->q32, m->E32, nullptr, m->d, m->k0f, MCF(m),
                                red_of(m, FIN_ALPHA), APPLY_DOT, done, m->flags + 1, s));
    }
    if (profile) CK(cudaEventRecordWithFlags(m->ev[2 * c + 1], s, cudaEventRecordExternal));
    switch (kind) {
      case IK_JAC32:
        LK(m, launch_pcg_update<float>(m->x32, m->r32, m->z32, m->p32, m->q32, m->dinv32, m->nvec,
                                       red_of(m, FIN_UPDATE), true, s));
        LK(m, launch_pcg_direction<float>(m->p32, m->z32, m->nvec, m->sc, s));
        break;
      case IK_JAC64:
        LK(m, launch_pcg_update<double>(m->x64, m->s64, m->z64, m->p64, m->q64, m->dinv64,
                                        m->nvec, red_of(m, FIN_UPDATE), true, s));
        LK(m, launch_pcg_direction<double>(m->p64, m->z64, m->nvec, m->sc, s));
        break;
      default:
        {  // the update also forms the V-cycle's first direction; z = V(r), with
           // r . z (beta) fused into the V-cycle's last smoothing step
          float* d0 = nullptr;
          const float th = gmg_first_direction(m->gmg, &d0);
          LK(m, launch_pcg_update<float>(m->x32, m->r32, d0 ? d0 : m->z32, m->p32, m->q32,
                                         d0 ? m->dinv32 : nullptr, m->nvec,
                                         red_of(m, FIN_RR_ONLY), false, s, Bat{}, th));
          const Red zr = red_of(m, FIN_RZ_BETA);
          GmgProf gp;
          GmgProf* gpp = cheb_prof(m, profile, c, gp);
          CK(gmg_vcycle(m->gmg, m->r32, m->z32, m->k0f, MCF(m), done, m->flags + 1, s,
                        &m->launches, Bat{}, &zr, d0 != nullptr, gpp));
          cheb_prof_done(m, gpp);
        }
        LK(m, launch_pcg_direction<float>(m->p32, m->z32, m->nvec, m->sc, s));
        break;
    }
  }
  return TOPO_OK;
}

void clear_graphs(topo_mesh* m) {
  for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);
  m->graphs.clear();
}

// Run a chunk of iterations as one CUDA graph (captured on first use per
// kind/size/profiling, then replayed): one launch instead of ~40 per
// iteration for the multigrid path.
topo_status run_iters(topo_mesh* m, int kind, int count, bool profile) {
  const long long key = (long long)kind | ((long long)count << 4) | ((long long)profile << 24);
  auto it = m->graphs.find(key);
  if (it == m->graphs.end()) {
    const long long l0 = m->launches;
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    const topo_status st = enqueue_iters(m, kind, count, profile);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (st != TOPO_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != TOPO_OK ? st : cuda_status(e);
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(ei);
    ChunkGraph cg;
    cg.exec = ex;
    cg.launches = m->launches - l0;
    m->launches = l0;
    it = m->graphs.emplace(key, cg).first;
  }
  CK(cudaGraphLaunch(it->second.exec, m->stream));
  m->launches += it->second.launches;
  return TOPO_OK;
}

topo_status ensure_gmg(topo_mesh* m, const topo_solve_opts* o) {
  if (m->gmg_built && (m->gmg_levels_req != o->gmg_levels || m->gmg_degree != o->smooth_degree)) {
    CK(cudaStreamSynchronize(m->stream));
    clear_graphs(m);
    m->bytes -= m->gmg.bytes;
    gmg_free(m->gmg);
    m->gmg = Gmg();
    m->gmg_built = false;
  }
  if (!m->gmg_built) {
    cudaError_t e = gmg_create(m->gmg, m->d, o->gmg_levels, o->smooth_degree, m->lam_max,
                               m->stream, nullptr, m->throughput);
    m->bytes += m->gmg.bytes;
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? TOPO_ERR_OOM : TOPO_ERR_INVALID;
    }
    m->gmg_built = true;
    m->gmg_levels_req = o->gmg_levels;
    m->gmg_degree = o->smooth_degree;
  }
  if (!m->gmg.ready) CK(gmg_setup(m->gmg, m->E32, m->dinv32, m->k0f, m->k0d, m->stream, &m->launches));
  return TOPO_OK;
}

// ---------------------------------------------------------------------------
// Non-blocking solve driver.  A solve is a small state machine that only
// ever enqueues work on its mesh's stream and asks for the device scalars
// with an event; the host advances it when the event has completed.  One
// host thread can thus drive many meshes at once (topo_solve_many), each on
// its own stream, and a single solve simply waits on its event.
// ---------------------------------------------------------------------------
struct SolveTask {
  topo_mesh* m = nullptr;
  topo_solve_opts o{};
  topo_solve_info* info = nullptr;
  enum Phase { P_RESID, P_INNER, P_FINISHED } phase = P_FINISHED;
  topo_status st = TOPO_OK;
  int outer = 0, total = 0, it_before = 0, kind = IK_JAC32;
  int detail = TOPO_FAIL_NONE;
  bool profile = false;
  double fn = 0.0;
  double expect = 1.0;      // relative residual the running inner solve aims at
  bool resid_dword = false; // the last residual was evaluated in double-word arithmetic
  Timer timer;
};

topo_status request_scalars(topo_mesh* m) {
  CK(cudaMemcpyAsync(m->h_sc, m->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaMemcpyAsync(m->h_flag, m->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaEventRecord(m->ev_poll, m->stream));
  return TOPO_OK;
}

void task_finish(SolveTask& t, topo_status st) {
  t.st = st;
  t.phase = SolveTask::P_FINISHED;
  if (st != TOPO_OK && t.detail == TOPO_FAIL_NONE)
    t.detail = (st == TOPO_ERR_NOT_CONVERGED) ? TOPO_FAIL_LIMIT
               : (st == TOPO_ERR_TIMEOUT)     ? TOPO_FAIL_TIMEOUT
               : (st == TOPO_ERR_CUDA || st == TOPO_ERR_OOM) ? TOPO_FAIL_DEVICE
                                                               : TOPO_FAIL_SETUP;
  if (st == TOPO_OK) t.m->solved = true;
  if (t.info) {
    t.info->iters = t.total;
    t.info->outer = t.outer;
    t.info->status = st;
    t.info->detail = t.detail;
    t.info->seconds = t.timer.seconds();
  }
}

// Refinement residual r = f - K u (fixed DOFs 0), ||r||^2 -> aux[0]: in FP64,
// or (dword) K u in double-word arithmetic from u split into the FP32
// vectors p32 / q32, which are free between inner solves.  bt / skip: the
// designs of a mesh group, skipping those that sat out the step.
topo_status enqueue_residual(topo_mesh* m, bool dword, const int* skip = nullptr,
                             const Bat& bt = Bat{}) {
  if (dword) {
    LK(m, launch_split_dw(m->u64, m->p32, m->q32, m->nvec, skip, m->stream, bt));
    LK(m, launch_apply_dw(m->p32, m->q32, m->r64, m->E64, m->f64, m->d, m->mcd,
                          red_of(m, FIN_AUX), APPLY_RESID, skip, m->stream, bt));
  } else {  // FP64; the modal kernel also stores the element energies of u
    LK(m, launch_apply<double>(m->u64, m->r64, m->E64, m->f64, m->d, m->k0d, MCD(m),
                               red_of(m, FIN_AUX), APPLY_RESID, skip, m->flags + 1, m->stream,
                               bt, m->use_modal ? m->energy : nullptr));
  }
  return TOPO_OK;
}

// The residual after an inner solve that aimed at relative residual `expect`
// is evaluated in double-word arithmetic only when it cannot certify
// convergence (expect at least 100 x rtol: it only sets the next right-hand
// side, where ~1e-13 relative rounding is far below what the next inner
// solve resolves); every residual that may end the solve is FP64.
bool dword_residual(const topo_solve_opts& o, double expect) {
  return o.precision == TOPO_PREC_FP32 && o.residual == TOPO_RESIDUAL_DWORD &&
         expect >= 100.0 * o.rtol;
}

// start of an inner CG from x = 0 on the current right-hand side
topo_status enqueue_inner_start(SolveTask& t, double rtol, int max_iter) {
  topo_mesh* m = t.m;
  cudaStream_t s = m->stream;
  const int* done = &m->sc->done;
  LK(m, launch_set_max_iter(m->sc, max_iter, s));
  if (t.kind == IK_JAC64) {
    LK(m, launch_pcg_init<double>(m->r64, m->x64, m->s64, m->z64, m->p64, m->dinv64, m->nvec,
                                  red_of(m, FIN_INIT, rtol * rtol), true, s));
  } else {
    LK(m, launch_narrow_scaled(m->b32, m->r64, m->nvec, m->sc, s));  // b = r / ||r|| in FP32
    if (t.kind == IK_JAC32) {
      LK(m, launch_pcg_init<float>(m->b32, m->x32, m->r32, m->z32, m->p32, m->dinv32, m->nvec,
                                   red_of(m, FIN_INIT, rtol * rtol), true, s));
    } else {
      LK(m, launch_pcg_init<float>(m->b32, m->x32, m->r32, m->z32, m->p32, nullptr, m->nvec,
                                   red_of(m, FIN_INIT, rtol * rtol), false, s));
      {
        const Red zr = red_of(m, FIN_SET_RZ);
        CK(gmg_vcycle(m->gmg, m->r32, m->z32, m->k0f, MCF(m), done, m->flags + 1, s,
                      &m->launches, Bat{}, &zr));
      }
      LK(m, launch_pcg_direction<float>(m->p32, m->z32, m->nvec, m->sc, s));
    }
  }
  return TOPO_OK;
}

topo_status task_start(SolveTask& t) {
  topo_mesh* m = t.m;
  const topo_solve_opts* o = &t.o;
  if (!m->has_density) return TOPO_ERR_NO_DENSITY;
  if (o->precision != TOPO_PREC_FP64 && o->precision != TOPO_PREC_FP32) return TOPO_ERR_INVALID;
  if (o->precond != TOPO_PRECOND_JACOBI && o->precond != TOPO_PRECOND_GMG) return TOPO_ERR_INVALID;
  if (o->precond == TOPO_PRECOND_GMG &&
      (o->precision != TOPO_PREC_FP32 || o->smooth_degree < 1 || o->smooth_degree > 8))
    return TOPO_ERR_INVALID;
  if (!(o->rtol > 0.0) || o->max_iter < 1 || o->max_outer < 1 || o->check_every < 1 ||
      o->check_every > 1024)
    return TOPO_ERR_INVALID;
  if (o->residual != TOPO_RESIDUAL_DWORD && o->residual != TOPO_RESIDUAL_FP64)
    return TOPO_ERR_INVALID;
  cudaStream_t s = m->stream;
  if (o->precision == TOPO_PREC_FP64) {
    t.kind = IK_JAC64;
    CKS(ensure_fp64_inner(m));
    if (!m->diag64) {
      LK(m, launch_diag_inv<double>(m->dinv64, m->E64, m->d, m->k0d, s));
      m->diag64 = true;
    }
  } else {
    t.kind = (o->precond == TOPO_PRECOND_GMG) ? IK_GMG32 : IK_JAC32;
    if (!m->diag32) {
      LK(m, launch_diag_inv<float>(m->dinv32, m->E32, m->d, m->k0f, s));
      m->diag32 = true;
    }
  }
  if (t.kind == IK_GMG32) CKS(ensure_gmg(m, o));
  t.profile = m->prof && t.kind != IK_JAC64;
  if (t.profile) CKS(ensure_profile_events(m, o->check_every));
  m->solved = false;
  t.fn = std::sqrt(m->fnorm2);
  CK(cudaMemsetAsync(m->flags + 1, 0, sizeof(int), s));  // bounded-wait timeout flag
  if (o->warm_start) {
    CKS(enqueue_residual(m, false));  // a warm start may already be converged
    m->energy_fresh = m->use_modal;
  } else {
    CK(cudaMemsetAsync(m->u64, 0, sizeof(double) * m->nvec, s));
    CK(cudaMemcpyAsync(m->r64, m->f64, sizeof(double) * m->nvec, cudaMemcpyDeviceToDevice, s));
    LK(m, launch_dot<double>(m->r64, m->r64, m->nvec, red_of(m, FIN_AUX), s));
    m->energy_fresh = false;
  }
  CKS(request_scalars(m));
  t.phase = SolveTask::P_RESID;
  return TOPO_OK;
}

// Advance a task whose last scalar request has completed.
topo_status task_step(SolveTask& t) {
  topo_mesh* m = t.m;
  const topo_solve_opts& o = t.o;
  const PcgScalars& h = *m->h_sc;
  if (*m->h_flag) {
    t.detail = TOPO_FAIL_TIMEOUT;
    return TOPO_ERR_TIMEOUT;
  }
  if (t.phase == SolveTask::P_RESID) {
    const double rr = h.aux[0];
    if (!std::isfinite(rr)) {
      t.detail = TOPO_FAIL_RESIDUAL;
      return TOPO_ERR_NAN;
    }
    const double rel = t.fn > 0 ? std::sqrt(rr) / t.fn : 0.0;
    if (t.info) t.info->rel_residual = rel;
    if (rel <= o.rtol && !t.resid_dword) {  // only an FP64 residual certifies
      task_finish(t, TOPO_OK);
      return TOPO_OK;
    }
    if (t.outer >= o.max_outer || t.total >= o.max_iter) return TOPO_ERR_NOT_CONVERGED;
    double inner;
    if (t.kind == IK_JAC64)  // the final tolerance directly, with margin
      inner = std::min(std::max(0.5 * o.rtol * t.fn / std::sqrt(rr), 1e-15), 0.5);
    else
      inner = std::min(std::max(o.inner_rtol, kInnerMargin * o.rtol * t.fn / std::sqrt(rr)), 0.5);
    t.expect = inner * rel;
    CKS(enqueue_inner_start(t, inner, o.max_iter - t.total));
    CKS(run_iters(m, t.kind, o.check_every, t.profile));
    t.it_before = 0;
    t.phase = SolveTask::P_INNER;
    return request_scalars(m);
  }
  // P_INNER: one chunk has run
  if (t.profile) {
    const int worked = std::min(o.check_every, h.iter - t.it_before);
    for (int c = 0; c < worked; ++c) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, m->ev[2 * c], m->ev[2 * c + 1]));
      m->prof_ms += ms;
      m->prof_launches += 1;
      if (t.kind == IK_GMG32) CKS(cheb_prof_collect(m, c, 1));
    }
  }
  if (!h.done) {
    if (h.iter == t.it_before) return TOPO_ERR_CUDA;  // no progress without a stop: a bug
    t.it_before = h.iter;
    CKS(run_iters(m, t.kind, o.check_every, t.profile));
    return request_scalars(m);
  }
  t.total += h.iter;
  ++t.outer;
  if (h.status == 2) {
    t.detail = TOPO_FAIL_BREAKDOWN;
    return TOPO_ERR_NAN;
  }
  if (t.kind == IK_JAC64)
    LK(m, launch_accumulate<double>(m->u64, m->x64, m->nvec, m->sc, false, m->stream));
  else  // scale back by ||r|| (aux[0] still holds ||r||^2 from the residual)
    LK(m, launch_accumulate<float>(m->u64, m->x32, m->nvec, m->sc, true, m->stream));
  t.resid_dword = t.kind != IK_JAC64 && dword_residual(o, t.expect);
  CKS(enqueue_residual(m, t.resid_dword));
  m->energy_fresh = !t.resid_dword && m->use_modal;  // u changed; FP64 residuals store energies
  t.phase = SolveTask::P_RESID;
  return request_scalars(m);
}

void task_advance(SolveTask& t) {
  const topo_status st = task_step(t);
  if (st != TOPO_OK) task_finish(t, st);
}

topo_status do_solve(topo_mesh* m, const topo_solve_opts* o, topo_solve_info* info) {
  SolveTask t;
  t.m = m;
  t.o = *o;
  t.info = info;
  topo_status st = task_start(t);
  if (st != TOPO_OK) {
    task_finish(t, st);
    return st;
  }
  while (t.phase != SolveTask::P_FINISHED) {
    const cudaError_t e = cudaEventSynchronize(m->ev_poll);
    if (e != cudaSuccess) {
      task_finish(t, cuda_status(e));
      break;
    }
    task_advance(t);
  }
  return t.st;
}

topo_status upload_f64(topo_mesh* m, const double* src, double* dst_soa, size_t n_dof,
                       int on_device) {
  cudaStream_t s = m->stream;
  const double* a = src;
  if (!on_device) {
    CK(cudaMemcpyAsync(m->aos, src, n_dof * sizeof(double), cudaMemcpyHostToDevice, s));
    a = m->aos;
  }
  LK(m, launch_unpack<double>(a, dst_soa, m->d, s));
  return TOPO_OK;
}

}  // namespace


// ===========================================================================
// Continuous-batching solve server.
//
// A design (one grid, BC and load) is opened once and then receives a stream
// of solve jobs (new densities), as an optimiser would send them.  The
// server admits designs in arrival order while their estimated device
// footprint fits the memory budget and fewer than max_active are resident
// (later designs that fit may pass a blocked one: backfill); an admitted
// design keeps its mesh, densities, displacement (warm start) and multigrid
// hierarchy on the device until it is closed.  Every admitted design runs
// its own solve state machine on its own stream, and topo_server_poll
// advances all of them from the caller's thread, so jobs that arrive while
// others are running start as soon as their design is resident and idle, and
// their kernels overlap with the others' on the GPU.
// ===========================================================================
struct ServerJob {
  int id = 0;
  std::vector<float> rho;
  double submit_s = 0.0, start_s = 0.0;
};

struct ServerDesign {
  int id = 0;
  int nx = 0, ny = 0, nz = 0, bc = 0, load = 0;
  long long footprint = 0;
  topo_mesh* mesh = nullptr;
  std::deque<ServerJob> queue;
  bool running = false, solved = false, closing = false, waiting = false;
  SolveTask task;
  ServerJob current;
  topo_solve_info info{};
  // a job's densities travel through a pinned buffer without a host wait;
  // their validity count arrives in h_bad with the solve's first scalars
  float* pinned = nullptr;
  int* h_bad = nullptr;
  bool check_bad = false;
  bool finishing = false;  // the solve is done; its compliance is on the way
};

struct topo_server {
  cudaStream_t user = nullptr;
  topo_params prm{};
  topo_solve_opts opts{};
  long long budget = 0, in_use = 0, peak = 0;
  int max_active = 0, active = 0;
  int next_design = 1, next_job = 1;
  std::map<int, ServerDesign> designs;
  std::deque<int> admit;                   // designs waiting for admission, in arrival order
  std::deque<topo_job_result> done;        // finished jobs not yet returned
  Timer clock;
};

namespace {

void server_release(topo_server* s, ServerDesign& d) {
  if (d.mesh) {
    topo_free(d.mesh);  // synchronises the design's stream first
    d.mesh = nullptr;
    s->in_use -= d.footprint;
    --s->active;
  }
  if (d.pinned) cudaFreeHost(d.pinned);
  if (d.h_bad) cudaFreeHost(d.h_bad);
  d.pinned = nullptr;
  d.h_bad = nullptr;
}

// A job's densities onto its design's mesh without a host wait (the server's
// form of topo_set_density): the values go through the design's pinned
// buffer, Eq. (1) runs on the mesh's stream after the caller's earlier work,
// and the count of invalid densities is copied to d.h_bad behind it, to be
// read when the solve's first scalars have arrived.
topo_status server_set_density(ServerDesign& d, const std::vector<float>& rho) {
  topo_mesh* m = d.mesh;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  std::memcpy(d.pinned, rho.data(), (size_t)ne * sizeof(float));
  cudaStream_t s = m->stream;
  CK(cudaSetDevice(m->dev));
  CK(cudaEventRecord(m->ev_in, m->user));
  CK(cudaStreamWaitEvent(s, m->ev_in, 0));
  CK(cudaMemcpyAsync(m->rho_in, d.pinned, ne * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(m->flags, 0, sizeof(int), s));
  LK(m, launch_simp(m->rho_in, m->rho_g, m->E32, m->E64, m->d, m->prm.E0, m->prm.Emin,
                    m->prm.penal, m->prm.h, m->flags, s));
  CK(cudaMemcpyAsync(d.h_bad, m->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  m->diag32 = m->diag64 = false;
  m->gmg.ready = false;
  m->solved = false;
  m->energy_fresh = false;
  m->e_positive = m->prm.Emin > 0.0;
  m->has_density = true;  // provisionally: d.check_bad settles it
  d.check_bad = true;
  return TOPO_OK;
}

// one pass over the server: admit, start, advance, retire; true if anything moved
bool server_step(topo_server* s) {
  bool moved = false;
  // admission (arrival order with backfill)
  for (auto it = s->admit.begin(); it != s->admit.end();) {
    ServerDesign& d = s->designs[*it];
    if (s->active < s->max_active && s->in_use + d.footprint <= s->budget) {
      topo_mesh* m = nullptr;
      topo_status st = topo_create_mesh(d.nx, d.ny, d.nz, d.bc, d.load, &s->prm, s->user, &m);
      if (st == TOPO_OK) {
        st = topo_set_throughput_mode(m, 1);
        if (st != TOPO_OK) topo_free(m);
      }
      if (st == TOPO_OK &&
          (cudaMallocHost(&d.pinned, sizeof(float) * (size_t)d.nx * d.ny * d.nz) != cudaSuccess ||
           cudaMallocHost(&d.h_bad, sizeof(int)) != cudaSuccess)) {
        cudaGetLastError();
        topo_free(m);
        if (d.pinned) cudaFreeHost(d.pinned);
        d.pinned = nullptr;
        st = TOPO_ERR_OOM;
      }
      if (st == TOPO_OK) {
        d.mesh = m;
        d.waiting = false;
        s->in_use += d.footprint;
        s->peak = std::max(s->peak, s->in_use);
        ++s->active;
        it = s->admit.erase(it);
        moved = true;
        continue;
      }
      if (st != TOPO_ERR_OOM) {  // a design that can never run: fail its jobs
        for (ServerJob& j : d.queue) {
          topo_job_result r{};
          r.job = j.id;
          r.design = d.id;
          r.status = st;
          r.submit_s = j.submit_s;
          r.finish_s = s->clock.seconds();
          s->done.push_back(r);
        }
        d.queue.clear();
        d.waiting = false;
        it = s->admit.erase(it);
        moved = true;
        continue;
      }
    }
    ++it;
  }
  for (auto& kv : s->designs) {
    ServerDesign& d = kv.second;
    if (!d.mesh) continue;
    // advance a running solve
    if (d.running) {
      cudaSetDevice(d.mesh->dev);
      const cudaError_t q = cudaEventQuery(d.mesh->ev_poll);
      bool report = false;
      if (d.finishing) {  // f^T u (enqueued when the solve ended) has arrived
        if (q == cudaSuccess) {
          d.finishing = false;
          report = true;
        } else if (q != cudaErrorNotReady) {
          cudaGetLastError();
          d.finishing = false;
          d.task.st = cuda_status(q);
          d.info.status = d.task.st;
          d.info.detail = TOPO_FAIL_DEVICE;
          report = true;
        }
      } else {
        if (q == cudaSuccess) {
          if (d.check_bad) {  // the job's densities were checked before these scalars
            d.check_bad = false;
            if (*d.h_bad) {
              d.mesh->has_density = false;
              task_finish(d.task, TOPO_ERR_NAN);
            }
          }
          if (d.task.phase != SolveTask::P_FINISHED) task_advance(d.task);
          moved = true;
        } else if (q != cudaErrorNotReady) {
          cudaGetLastError();
          task_finish(d.task, cuda_status(q));
        }
        if (d.task.phase == SolveTask::P_FINISHED) {
          moved = true;
          topo_mesh* m = d.mesh;
          // compliance J = f^T u (Eq. (2)) without a host wait: the dot and its
          // copy follow the solve on the design's stream, reported when they land
          if (d.task.st == TOPO_OK &&
              launch_dot<double>(m->f64, m->u64, m->nvec, red_of(m, FIN_AUX), m->stream) ==
                  cudaSuccess &&
              cudaMemcpyAsync(m->h_sc, m->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                              m->stream) == cudaSuccess &&
              cudaEventRecord(m->ev_poll, m->stream) == cudaSuccess) {
            ++m->launches;
            d.finishing = true;
          } else {
            if (d.task.st == TOPO_OK) {  // the enqueue failed
              cudaGetLastError();
              d.task.st = TOPO_ERR_CUDA;
              d.info.status = TOPO_ERR_CUDA;
              d.info.detail = TOPO_FAIL_DEVICE;
            }
            report = true;
          }
        }
      }
      if (report) {
        d.running = false;
        moved = true;
        topo_job_result r{};
        r.job = d.current.id;
        r.design = d.id;
        r.status = d.task.st;
        r.detail = d.info.detail;
        r.iters = d.info.iters;
        r.outer = d.info.outer;
        r.rel_residual = d.info.rel_residual;
        r.submit_s = d.current.submit_s;
        r.start_s = d.current.start_s;
        if (r.status == TOPO_OK) {
          r.compliance = d.mesh->h_sc->aux[0];
          d.solved = true;
        }
        {
          Fence fence(d.mesh);  // the caller's stream waits for this design's work
        }
        r.finish_s = s->clock.seconds();
        s->done.push_back(r);
        d.current.rho.clear();
      }
    }
    // start the next job of an idle, resident design
    if (!d.running && !d.queue.empty()) {
      d.current = std::move(d.queue.front());
      d.queue.pop_front();
      d.current.start_s = s->clock.seconds();
      d.info = topo_solve_info{};
      topo_status st = server_set_density(d, d.current.rho);
      d.task = SolveTask();
      d.task.m = d.mesh;
      d.task.o = s->opts;
      d.task.o.warm_start = d.solved ? 1 : 0;
      d.task.info = &d.info;
      if (st == TOPO_OK) st = task_start(d.task);
      moved = true;
      if (st != TOPO_OK) {  // report at once: the job never ran
        task_finish(d.task, st);
        topo_job_result r{};
        r.job = d.current.id;
        r.design = d.id;
        r.status = st;
        r.detail = TOPO_FAIL_SETUP;
        r.submit_s = d.current.submit_s;
        r.start_s = d.current.start_s;
        r.finish_s = s->clock.seconds();
        s->done.push_back(r);
        d.current.rho.clear();
      } else {
        d.running = true;
      }
    }
  }
  // retire closed designs once idle
  for (auto it = s->designs.begin(); it != s->designs.end();) {
    ServerDesign& d = it->second;
    if (d.closing && !d.running && d.queue.empty()) {
      server_release(s, d);
      it = s->designs.erase(it);
      moved = true;
    } else {
      ++it;
    }
  }
  return moved;
}

bool server_busy(const topo_server* s) {
  for (const auto& kv : s->designs)
    if (kv.second.running || !kv.second.queue.empty()) return true;
  return false;
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

void topo_default_params(topo_params* p) {
  if (!p) return;
  p->E0 = 1.0;
  p->Emin = 1e-9;
  p->nu = 0.3;
  p->penal = 3.0;
  p->h = 1.0;
  p->load = 1.0;
}

void topo_default_opts(topo_solve_opts* o) {
  if (!o) return;
  o->precision = TOPO_PREC_FP32;
  o->precond = TOPO_PRECOND_GMG;
  o->rtol = 1e-8;
  o->inner_rtol = 1e-5;
  o->max_iter = 100000;
  o->max_outer = 12;
  o->warm_start = 0;
  o->gmg_levels = 0;
  o->smooth_degree = 3;
  o->check_every = 8;
  o->residual = TOPO_RESIDUAL_DWORD;
}

const char* topo_status_string(int status) {
  switch (status) {
    case TOPO_OK: return "ok";
    case TOPO_ERR_INVALID: return "invalid argument";
    case TOPO_ERR_OOM: return "out of memory";
    case TOPO_ERR_CUDA: return "CUDA error";
    case TOPO_ERR_NO_DENSITY: return "no density set";
    case TOPO_ERR_NOT_SOLVED: return "not solved";
    case TOPO_ERR_NOT_CONVERGED: return "not converged";
    case TOPO_ERR_NAN: return "non-finite or out-of-range value";
    case TOPO_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

void topo_free(topo_mesh* m) {
  if (!m) return;
  cudaSetDevice(m->dev);
  if (m->stream) cudaStreamSynchronize(m->stream);
  void* ptrs[] = {m->rho_g, m->E32,  m->E64,  m->f64, m->u64,  m->r64, m->x32, m->r32,
                  m->z32,   m->p32,  m->q32,  m->b32, m->dinv32, m->x64, m->s64, m->z64,
                  m->p64,   m->q64,  m->dinv64, m->sc, m->partials, m->flags, m->aos, m->dc,
                  m->rho_in, m->dcf, m->rho_next, m->oc_state, m->oc_part, m->phi_in,
                  m->phi_tmp, m->ls_part, m->ls_bJ, m->ls_bV, m->hx, m->hr, m->hz, m->hp,
                  m->hq, m->hdinv, m->hb, m->hdir, m->ls_scratch, m->ls_dt, m->tr_rho_n,
                  m->tr_counts, m->tr_off, m->tr_scratch, m->tr_tris};
  MeshGroup* G = m->group;
  auto in_arena = [&](void* p) {
    const char* c = static_cast<char*>(p);
    return G && ((c >= G->arena && c < G->arena + (long long)G->nb * G->S) ||
                 (G->arena64 && c >= G->arena64 && c < G->arena64 + G->arena64_bytes));
  };
  for (void* p : ptrs)
    if (p && !in_arena(p)) cudaFree(p);
  clear_graphs(m);
  if (m->gmg_built) gmg_free(m->gmg);
  if (G) {
    for (auto& q : G->meshes)
      if (q == m) q = nullptr;
    if (--G->refs == 0) {
      for (auto& kv : G->graphs) cudaGraphExecDestroy(kv.second.exec);
      if (G->arena) cudaFree(G->arena);
      if (G->arena64) cudaFree(G->arena64);
      if (G->h_sc) cudaFreeHost(G->h_sc);
      if (G->h_flag) cudaFreeHost(G->h_flag);
      if (G->h_next) cudaFreeHost(G->h_next);
      if (G->h_ids) cudaFreeHost(G->h_ids);
      if (G->d_ids) cudaFree(G->d_ids);
      if (G->stage) cudaFree(G->stage);
      delete G;
    }
  }
  if (m->h_sc) cudaFreeHost(m->h_sc);
  if (m->h_flag) cudaFreeHost(m->h_flag);
  if (m->oc_host) cudaFreeHost(m->oc_host);
  if (m->ev_poll) cudaEventDestroy(m->ev_poll);
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : m->evc) cudaEventDestroy(e);
  if (m->ev_in) cudaEventDestroy(m->ev_in);
  if (m->ev_out) cudaEventDestroy(m->ev_out);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

static topo_status create_impl(int nx, int ny, int nz, int bc, int load, const topo_params* prm,
                               void* stream, topo_mesh* m) {
  CK(cudaGetDevice(&m->dev));
  m->user = static_cast<cudaStream_t>(stream);
  CK(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
  m->own_stream = true;
  CK(cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming));
  CK(cudaEventRecord(m->ev_in, m->user));
  CK(cudaStreamWaitEvent(m->stream, m->ev_in, 0));
  m->d = make_dims(nx, ny, nz, bc, ny / 2);
  m->nvec = 3 * m->d.comp;
  if (prm)
    m->prm = *prm;
  else
    topo_default_params(&m->prm);
  double k[576];
  build_k0(m->prm.nu, k);
  for (int t = 0; t < 576; ++t) {
    m->k0d.v[t] = k[t];
    m->k0f.v[t] = (float)k[t];
  }
  m->lam_max = k0_jacobi_bound(k);
  if (!build_modal_coef(k, &m->mcd)) return TOPO_ERR_INVALID;
  {
    m->mcf = ModalCoef<float>{};
    for (int a = 0; a < 3; ++a)
      for (int q = 0; q < 8; ++q) {
        m->mcf.D[a][q] = (float)m->mcd.D[a][q];
        for (int b = 0; b < 3; ++b) m->mcf.C[a][b][q] = (float)m->mcd.C[a][b][q];
      }
    m->mcf.kdiag = (float)m->mcd.kdiag;
    m->mcf.form = m->mcd.form;
  }
  const long long ne = m->d.ecount;
  CKS(dalloc(m, &m->rho_in, (long long)nx * ny * nz));
  CKS(dalloc(m, &m->energy, ne));
  CKS(dalloc(m, &m->rho_g, ne));
  CKS(dalloc(m, &m->E32, ne));
  CKS(dalloc(m, &m->E64, ne));
  CKS(dalloc(m, &m->f64, m->nvec));
  CKS(dalloc(m, &m->u64, m->nvec));
  CKS(dalloc(m, &m->r64, m->nvec));
  CKS(dalloc(m, &m->x32, m->nvec));
  CKS(dalloc(m, &m->r32, m->nvec));
  CKS(dalloc(m, &m->z32, m->nvec));
  CKS(dalloc(m, &m->p32, m->nvec));
  CKS(dalloc(m, &m->q32, m->nvec));
  CKS(dalloc(m, &m->b32, m->nvec));
  CKS(dalloc(m, &m->dinv32, m->nvec));
  CKS(dalloc(m, &m->sc, 1));
  CKS(dalloc(m, &m->partials, 4LL * kMaxPartials));
  CKS(dalloc(m, &m->flags, 4));
  const long long nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  CKS(dalloc(m, &m->aos, 3 * nn));
  CK(cudaMallocHost(&m->h_sc, sizeof(PcgScalars)));
  std::memset(m->h_sc, 0, sizeof(PcgScalars));
  CK(cudaMallocHost(&m->h_flag, sizeof(int)));
  *m->h_flag = 0;
  CK(cudaEventCreateWithFlags(&m->ev_poll, cudaEventDisableTiming));
  LK(m, launch_build_load(m->f64, m->d, load, m->prm.load, m->prm.h, m->stream));
  LK(m, launch_dot<double>(m->f64, m->f64, m->nvec, red_of(m, FIN_AUX), m->stream));
  CKS(sync_scalars(m));
  m->fnorm2 = m->h_sc->aux[0];
  CK(cudaEventRecord(m->ev_out, m->stream));
  CK(cudaStreamWaitEvent(m->user, m->ev_out, 0));
  return TOPO_OK;
}

topo_status topo_create_mesh(int nx, int ny, int nz, int bc, int load, const topo_params* prm,
                             void* stream, topo_mesh** out) {
  if (!out) return TOPO_ERR_INVALID;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) return TOPO_ERR_INVALID;
  if ((long long)(nx + 1) * (ny + 1) * (nz + 1) >= (1LL << 31)) return TOPO_ERR_INVALID;
  if (bc < 0 || bc > 5 || load < 0 || load > 4) return TOPO_ERR_INVALID;
  if ((bc == TOPO_BC_MBB || bc == TOPO_BC_MBB_STRIP) && (ny % 2)) return TOPO_ERR_INVALID;
  if (prm && (!(prm->nu >= 0.0 && prm->nu < 0.5) || !(prm->penal >= 1.0) || !(prm->h > 0.0) ||
              !(prm->E0 > 0.0) || !(prm->Emin >= 0.0) || !(prm->Emin < prm->E0)))
    return TOPO_ERR_INVALID;
  topo_mesh* m = new (std::nothrow) topo_mesh();
  if (!m) return TOPO_ERR_OOM;
  topo_status st = create_impl(nx, ny, nz, bc, load, prm, stream, m);
  if (st != TOPO_OK) {
    topo_free(m);
    return st;
  }
  *out = m;
  return TOPO_OK;
}

// Bytes of one design's region: create_impl's buffers and the multigrid
// hierarchy, in their order, each rounded up to 256 bytes (the region
// allocator checks every allocation against this bound).
static long long group_region_bytes(const Dims& d, int levels) {
  const long long nvec = 3 * d.comp, ne = d.ecount;
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  long long b = 0;
  auto add = [&](long long bytes) { b += (bytes + 255) / 256 * 256 + 256; };
  add((long long)d.nx * d.ny * d.nz * 4);  // rho_in
  add(ne * 8);                             // element energies
  add(ne * 4);
  add(ne * 4);
  add(ne * 8);
  for (int q = 0; q < 3; ++q) add(nvec * 8);
  for (int q = 0; q < 7; ++q) add(nvec * 4);
  add(sizeof(PcgScalars));
  add(4LL * kMaxPartials * 8);
  add(4 * 4);
  add(3 * nn * 8);
  const std::vector<Dims> lv = gmg_plan(d, levels);
  for (size_t l = 0; l < lv.size(); ++l) {
    const long long n = 3 * lv[l].comp;
    for (int q = 0; q < 3; ++q) add(n * 4);
    if (l > 0) {
      add(lv[l].ecount * 4);
      for (int q = 0; q < 3; ++q) add(n * 4);
    }
  }
  const Dims& dc = lv.back();
  const long long nc = 3LL * (dc.nx + 1) * (dc.ny + 1) * (dc.nz + 1);
  add(nc * nc * 8);
  add(4 * nc * 8);
  add(nc * 8);
  return (b + 4095) / 4096 * 4096;
}

topo_status topo_create_batch(int nx, int ny, int nz, int bc, int load, const topo_params* prm,
                              void* stream, int n_designs, int gmg_levels, int smooth_degree,
                              topo_mesh** out) {
  if (!out || n_designs < 1 || n_designs > 1024 || smooth_degree < 1 || smooth_degree > 8)
    return TOPO_ERR_INVALID;
  for (int b = 0; b < n_designs; ++b) out[b] = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) return TOPO_ERR_INVALID;
  if ((long long)(nx + 1) * (ny + 1) * (nz + 1) >= (1LL << 31)) return TOPO_ERR_INVALID;
  if (bc < 0 || bc > 5 || load < 0 || load > 4) return TOPO_ERR_INVALID;
  if ((bc == TOPO_BC_MBB || bc == TOPO_BC_MBB_STRIP) && (ny % 2)) return TOPO_ERR_INVALID;
  if (prm && (!(prm->nu >= 0.0 && prm->nu < 0.5) || !(prm->penal >= 1.0) || !(prm->h > 0.0) ||
              !(prm->E0 > 0.0) || !(prm->Emin >= 0.0) || !(prm->Emin < prm->E0)))
    return TOPO_ERR_INVALID;
  const Dims d = make_dims(nx, ny, nz, bc, ny / 2);
  MeshGroup* G = new (std::nothrow) MeshGroup();
  if (!G) return TOPO_ERR_OOM;
  G->nb = n_designs;
  G->S = group_region_bytes(d, gmg_levels);
  G->gmg_levels = gmg_levels;
  G->gmg_degree = smooth_degree;
  if (prm)
    G->prm = *prm;
  else
    topo_default_params(&G->prm);
  auto fail = [&](topo_status st) {
    for (int b = 0; b < n_designs; ++b) out[b] = nullptr;
    const std::vector<topo_mesh*> made = G->meshes;
    if (made.empty()) {
      if (G->arena) cudaFree(G->arena);
      if (G->h_sc) cudaFreeHost(G->h_sc);
      if (G->h_flag) cudaFreeHost(G->h_flag);
      if (G->h_next) cudaFreeHost(G->h_next);
      if (G->h_ids) cudaFreeHost(G->h_ids);
      if (G->d_ids) cudaFree(G->d_ids);
      if (G->stage) cudaFree(G->stage);
      delete G;
    } else {
      for (topo_mesh* m : made) topo_free(m);  // the last one frees the group
    }
    return st;
  };
  if (cudaMalloc(&G->arena, (size_t)(G->nb * G->S)) != cudaSuccess) {
    cudaGetLastError();
    G->arena = nullptr;
    return fail(TOPO_ERR_OOM);
  }
  if (cudaMemset(G->arena, 0, (size_t)(G->nb * G->S)) != cudaSuccess) return fail(TOPO_ERR_CUDA);
  if (cudaMallocHost(&G->h_sc, sizeof(PcgScalars) * G->nb) != cudaSuccess ||
      cudaMallocHost(&G->h_flag, sizeof(int) * G->nb) != cudaSuccess ||
      cudaMallocHost(&G->h_next, sizeof(MeshGroup::Next) * G->nb) != cudaSuccess ||
      cudaMallocHost(&G->h_ids, sizeof(int) * G->nb) != cudaSuccess ||
      cudaMalloc(&G->d_ids, sizeof(int) * G->nb) != cudaSuccess) {
    cudaGetLastError();
    return fail(TOPO_ERR_OOM);
  }
  for (int b = 0; b < n_designs; ++b) {
    topo_mesh* m = new (std::nothrow) topo_mesh();
    if (!m) return fail(TOPO_ERR_OOM);
    m->group = G;
    m->gidx = b;
    m->region = G->arena + b * G->S;
    m->region_size = G->S;
    m->region_open = true;
    G->meshes.push_back(m);
    ++G->refs;
    topo_status st = create_impl(nx, ny, nz, bc, load, &G->prm, stream, m);
    if (st != TOPO_OK) return fail(st);
    GmgAlloc alloc{m, region_alloc};
    const cudaError_t e = gmg_create(m->gmg, m->d, gmg_levels, smooth_degree, m->lam_max,
                                     m->stream, &alloc);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? TOPO_ERR_OOM : TOPO_ERR_INVALID);
    }
    m->bytes += m->gmg.bytes;
    m->gmg_built = true;
    m->gmg_levels_req = gmg_levels;
    m->gmg_degree = smooth_degree;
    m->region_open = false;  // later (optional) buffers are ordinary allocations
    if (m->region_used != G->meshes[0]->region_used) return fail(TOPO_ERR_INVALID);
  }
  for (int b = 0; b < n_designs; ++b) out[b] = G->meshes[b];
  return TOPO_OK;
}

static topo_status set_density_impl(topo_mesh* m, const float* src_dev) {
  cudaStream_t s = m->stream;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if (src_dev != m->rho_in)
    CK(cudaMemcpyAsync(m->rho_in, src_dev, ne * sizeof(float), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(m->flags, 0, sizeof(int), s));
  LK(m, launch_simp(m->rho_in, m->rho_g, m->E32, m->E64, m->d, m->prm.E0, m->prm.Emin,
                    m->prm.penal, m->prm.h, m->flags, s));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, m->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  m->diag32 = m->diag64 = false;
  m->gmg.ready = false;
  m->solved = false;
  m->energy_fresh = false;
  m->e_positive = m->prm.Emin > 0.0;
  m->has_density = (bad == 0);
  return bad ? TOPO_ERR_NAN : TOPO_OK;
}

topo_status topo_set_density(topo_mesh* m, const float* rho, size_t n_elem, int on_device) {
  if (!m || !rho) return TOPO_ERR_INVALID;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if ((long long)n_elem != ne) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  if (!m->rho_in) CKS(dalloc(m, &m->rho_in, ne));
  if (!on_device) {
    CK(cudaMemcpyAsync(m->rho_in, rho, ne * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    return set_density_impl(m, m->rho_in);
  }
  return set_density_impl(m, rho);
}

topo_status topo_set_levelset(topo_mesh* m, const double* phi, size_t n_nodes, int on_device,
                              double eta, double eps0, double* volume) {
  if (!m || !(eta > 0.0) || !(eps0 >= 0.0 && eps0 <= 1.0)) return TOPO_ERR_INVALID;
  const long long nn = (long long)(m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
  if ((long long)n_nodes != nn) return TOPO_ERR_INVALID;
  if (!phi && !m->phi_in) return TOPO_ERR_INVALID;  // no current level set to reuse
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  cudaStream_t s = m->stream;
  if (!m->phi_in) CKS(dalloc(m, &m->phi_in, nn));
  if (phi && phi != m->phi_in)
    CK(cudaMemcpyAsync(m->phi_in, phi, nn * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  m->ls_eta = eta;
  m->ls_eps0 = eps0;
  CK(cudaMemsetAsync(m->flags, 0, sizeof(int), s));
  LK(m, launch_ersatz(m->phi_in, m->rho_g, m->E32, m->E64, m->d, m->prm.E0, eta, eps0, m->prm.h,
                      red_of(m, FIN_AUX), m->flags, s));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, m->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKS(sync_scalars(m));
  m->diag32 = m->diag64 = false;
  m->gmg.ready = false;
  m->solved = false;
  m->has_density = (bad == 0);
  m->ls_ready = (bad == 0);
  m->energy_fresh = false;
  m->e_positive = eps0 > 0.0;
  if (volume) *volume = m->h_sc->aux[0] * m->prm.h * m->prm.h * m->prm.h;
  return bad ? TOPO_ERR_NAN : TOPO_OK;
}

static long long node_count(const topo_mesh* m) {
  return (long long)(m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
}

topo_status topo_get_levelset(topo_mesh* m, double* phi, size_t n_nodes, int on_device) {
  if (!m || !phi) return TOPO_ERR_INVALID;
  const long long nn = node_count(m);
  if ((long long)n_nodes != nn || !m->phi_in) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CK(cudaMemcpyAsync(phi, m->phi_in, nn * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_shape_rhs(topo_mesh* m, double* bJ, double* bV, size_t n_nodes, int on_device) {
  if (!m || (!bJ && !bV)) return TOPO_ERR_INVALID;
  const long long nn = node_count(m), ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if ((long long)n_nodes != nn || !m->ls_ready) return TOPO_ERR_INVALID;
  if (!m->solved) return TOPO_ERR_NOT_SOLVED;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  cudaStream_t s = m->stream;
  if (!m->ls_part) CKS(dalloc(m, &m->ls_part, 16 * ne));
  if (!m->ls_bJ) CKS(dalloc(m, &m->ls_bJ, nn));
  if (!m->ls_bV) CKS(dalloc(m, &m->ls_bV, nn));
  LK(m, launch_shape_rhs(m->u64, m->phi_in, m->ls_part, m->ls_bJ, m->ls_bV, m->d, m->ls_eta,
                         m->prm.E0, m->prm.nu, m->prm.h, s));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (bJ) CK(cudaMemcpyAsync(bJ, m->ls_bJ, nn * sizeof(double), kind, s));
  if (bV) CK(cudaMemcpyAsync(bV, m->ls_bV, nn * sizeof(double), kind, s));
  if (!on_device) CK(cudaStreamSynchronize(s));
  return TOPO_OK;
}

topo_status topo_hilbertian_solve(topo_mesh* m, double ell, const double* b, double* v,
                                  size_t n_nodes, int on_device, double rtol, int max_iter,
                                  int* iters) {
  if (iters) *iters = 0;
  if (!m || !b || !v || !(ell >= 0.0) || !(rtol > 0.0) || max_iter < 1) return TOPO_ERR_INVALID;
  const long long nn = node_count(m);
  if ((long long)n_nodes != nn) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  cudaStream_t s = m->stream;
  const long long npad = (nn + 3) / 4 * 4;
  double** vecs[] = {&m->hx, &m->hr, &m->hz, &m->hp, &m->hq, &m->hdinv, &m->hb};
  for (double** q : vecs)
    if (!*q) CKS(dalloc(m, q, npad));
  if (!m->hdir) CKS(dalloc(m, &m->hdir, npad));
  const double ell2 = ell * ell;
  if (ell2 != m->h_ell2) {
    LK(m, launch_hilb_setup(m->f64, m->hdir, m->hdinv, m->d, ell2, m->prm.h, npad, s));
    m->h_ell2 = ell2;
  }
  const double* src = b;
  if (!on_device) {
    CK(cudaMemcpyAsync(m->hq, b, nn * sizeof(double), cudaMemcpyHostToDevice, s));
    src = m->hq;
  }
  LK(m, launch_hilb_rhs(src, m->hb, m->hdir, m->d, npad, s));  // b = 0 on Gamma_N
  // Jacobi-PCG (Eq. (20) is SPD and well conditioned): x0 = 0
  LK(m, launch_set_max_iter(m->sc, max_iter, s));
  LK(m, launch_pcg_init<double>(m->hb, m->hx, m->hr, m->hz, m->hp, m->hdinv, npad,
                                red_of(m, FIN_INIT, rtol * rtol), true, s));
  const int* done = &m->sc->done;
  for (int chunk = 0;; ++chunk) {
    for (int c = 0; c < 8; ++c) {
      LK(m, launch_hilb_apply(m->hp, m->hq, m->hdir, m->d, ell2, m->prm.h, red_of(m, FIN_ALPHA),
                              true, done, s));
      LK(m, launch_pcg_update<double>(m->hx, m->hr, m->hz, m->hp, m->hq, m->hdinv, npad,
                                      red_of(m, FIN_UPDATE), true, s));
      LK(m, launch_pcg_direction<double>(m->hp, m->hz, npad, m->sc, s));
    }
    CKS(sync_scalars(m));
    if (m->h_sc->done) break;
    if (chunk > max_iter) return TOPO_ERR_CUDA;  // the device never stopped: a bug
  }
  if (iters) *iters = m->h_sc->iter;
  CK(cudaMemcpyAsync(v, m->hx, nn * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (m->h_sc->status == 1) return TOPO_ERR_NOT_CONVERGED;
  if (m->h_sc->status != 0) return TOPO_ERR_NAN;
  return TOPO_OK;
}

topo_status topo_hj_evolve(topo_mesh* m, const double* v, size_t n_nodes, int on_device,
                           double gamma, int steps, double* dt) {
  if (dt) *dt = 0.0;
  if (!m || !v || !(gamma > 0.0) || steps < 0) return TOPO_ERR_INVALID;
  const long long nn = node_count(m);
  if ((long long)n_nodes != nn || !m->phi_in) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  cudaStream_t s = m->stream;
  if (!m->phi_tmp) CKS(dalloc(m, &m->phi_tmp, nn));
  if (!m->hq) CKS(dalloc(m, &m->hq, (nn + 3) / 4 * 4));
  if (!m->ls_scratch) CKS(dalloc(m, &m->ls_scratch, 1));
  if (!m->ls_dt) CKS(dalloc(m, &m->ls_dt, 1));
  const double* vd = v;
  if (!on_device) {
    CK(cudaMemcpyAsync(m->hq, v, nn * sizeof(double), cudaMemcpyHostToDevice, s));
    vd = m->hq;
  }
  LK(m, launch_hj_steps(m->phi_in, m->phi_tmp, vd, m->d, gamma, m->prm.h, steps, m->ls_scratch,
                        m->ls_dt, s));
  m->ls_ready = false;  // the moduli no longer match phi until topo_set_levelset
  if (dt) {
    CK(cudaMemcpyAsync(dt, m->ls_dt, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return TOPO_OK;
}

// nodal densities from the mesh's current element densities (Eqs. (25)-(27))
static topo_status nodal_density_impl(topo_mesh* m) {
  const long long nn = node_count(m);
  if (!m->rho_in) return TOPO_ERR_NO_DENSITY;
  if (!m->tr_rho_n) CKS(dalloc(m, &m->tr_rho_n, nn));
  LK(m, launch_nodal_density(m->rho_in, m->tr_rho_n, m->d, m->prm.h, m->stream));
  return TOPO_OK;
}

// iso-surface of a nodal field into tr_tris / tr_off / tr_n
static topo_status extract_impl(topo_mesh* m, const double* f, double level, bool above) {
  cudaStream_t s = m->stream;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if (!m->tr_counts) CKS(dalloc(m, &m->tr_counts, ne));
  if (!m->tr_off) CKS(dalloc(m, &m->tr_off, ne + 1));
  if (!m->tr_scratch) CKS(dalloc(m, &m->tr_scratch, scan_scratch_count(ne)));
  LK(m, launch_mt_count(f, m->tr_counts, m->tr_off, m->tr_scratch, m->d, level, above, m->prm.h,
                        s));
  long long n = 0;
  CK(cudaMemcpyAsync(&n, m->tr_off + ne, sizeof(n), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n > m->tr_cap) {
    if (m->tr_tris) CK(cudaFree(m->tr_tris));
    m->tr_tris = nullptr;
    m->tr_cap = 0;
    const long long cap = n + n / 4 + 64;
    CKS(dalloc(m, &m->tr_tris, 9 * cap));
    m->tr_cap = cap;
  }
  if (n > 0)
    LK(m, launch_mt_emit(f, m->tr_off, m->tr_tris, m->d, level, above, m->prm.h, s));
  m->tr_n = n;
  return TOPO_OK;
}

topo_status topo_nodal_density(topo_mesh* m, double* rho_n, size_t n_nodes, int on_device) {
  if (!m || !rho_n) return TOPO_ERR_INVALID;
  const long long nn = node_count(m);
  if ((long long)n_nodes != nn) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(nodal_density_impl(m));
  CK(cudaMemcpyAsync(rho_n, m->tr_rho_n, nn * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_levelset_from_density(topo_mesh* m, double rho_t, long long* n_triangles) {
  if (n_triangles) *n_triangles = 0;
  if (!m || !(rho_t > 0.0 && rho_t < 1.0)) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  const long long nn = node_count(m);
  CKS(nodal_density_impl(m));
  CKS(extract_impl(m, m->tr_rho_n, rho_t, true));
  if (n_triangles) *n_triangles = m->tr_n;
  if (m->tr_n == 0) return TOPO_ERR_INVALID;  // no boundary at rho_t: no distance to it
  if (!m->phi_in) CKS(dalloc(m, &m->phi_in, nn));
  LK(m, launch_sdf(m->tr_tris, m->tr_off, m->tr_rho_n, rho_t, m->phi_in, m->d, m->prm.h,
                   m->stream));
  CK(cudaStreamSynchronize(m->stream));
  m->ls_ready = false;  // moduli still come from the densities until topo_set_levelset
  return TOPO_OK;
}

topo_status topo_extract_levelset_surface(topo_mesh* m, long long* n_triangles) {
  if (n_triangles) *n_triangles = 0;
  if (!m || !m->phi_in) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(extract_impl(m, m->phi_in, 0.0, false));
  if (n_triangles) *n_triangles = m->tr_n;
  return TOPO_OK;
}

topo_status topo_get_surface(topo_mesh* m, double* tri, size_t max_triangles, int on_device,
                             long long* n_triangles) {
  if (!m || (!tri && max_triangles)) return TOPO_ERR_INVALID;
  if (n_triangles) *n_triangles = m->tr_n;
  if ((long long)max_triangles < m->tr_n) return TOPO_ERR_INVALID;
  if (m->tr_n == 0) return TOPO_OK;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CK(cudaMemcpyAsync(tri, m->tr_tris, 9 * m->tr_n * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_reinit(topo_mesh* m, double gamma, double tol, int max_steps, int* steps) {
  if (steps) *steps = 0;
  if (!m || !(gamma > 0.0 && gamma <= 1.0) || !(tol >= 0.0) || max_steps < 1)
    return TOPO_ERR_INVALID;
  if (!m->phi_in) return TOPO_ERR_INVALID;
  const long long nn = node_count(m);
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  cudaStream_t s = m->stream;
  if (!m->phi_tmp) CKS(dalloc(m, &m->phi_tmp, nn));
  if (!m->ls_scratch) CKS(dalloc(m, &m->ls_scratch, 1));
  const double h = m->prm.h, dt = gamma * h;
  double* a = m->phi_in;
  double* b = m->phi_tmp;
  int done = 0;
  unsigned long long bits = 0;
  while (done < max_steps) {
    const int chunk = std::min(8, max_steps - done);
    for (int c = 0; c < chunk; ++c) {
      if (c == chunk - 1) CK(cudaMemsetAsync(m->ls_scratch, 0, sizeof(unsigned long long), s));
      LK(m, launch_reinit_step(a, b, m->d, dt, h, m->ls_scratch, s));
      std::swap(a, b);
    }
    done += chunk;
    CK(cudaMemcpyAsync(&bits, m->ls_scratch, sizeof(bits), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double change;
    std::memcpy(&change, &bits, sizeof(change));
    if (change <= tol * h) break;
  }
  if (a != m->phi_in) CK(cudaMemcpyAsync(m->phi_in, a, nn * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  m->ls_ready = false;
  if (steps) *steps = done;
  return TOPO_OK;
}

topo_status topo_element_energy(topo_mesh* m, double* w, size_t n_elem, int on_device) {
  if (!m || !w) return TOPO_ERR_INVALID;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if ((long long)n_elem != ne) return TOPO_ERR_INVALID;
  if (!m->solved) return TOPO_ERR_NOT_SOLVED;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  if (!m->dc) CKS(dalloc(m, &m->dc, ne));
  // the Eq. (3) kernel with p = 1 and -(E0 - Emin) h replaced by h: w_e = u_e^T k0(h) u_e
  LK(m, launch_sensitivity(m->u64, m->rho_g, m->E64, m->dc, m->d, m->mcd, 1.0, -m->prm.h,
                           red_of(m, FIN_AUX), m->stream));
  CK(cudaMemcpyAsync(w, m->dc, ne * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_solve(topo_mesh* m, const topo_solve_opts* opts, topo_solve_info* info) {
  Timer t;
  if (info) std::memset(info, 0, sizeof(*info));
  if (!m) {
    if (info) info->status = TOPO_ERR_INVALID;
    return TOPO_ERR_INVALID;
  }
  topo_solve_opts o;
  if (opts)
    o = *opts;
  else
    topo_default_opts(&o);
  topo_status st;
  {
    Fence fence(m);
    st = fence.st != TOPO_OK ? fence.st : do_solve(m, &o, info);
  }
  if (info) {
    info->status = st;
    info->seconds = t.seconds();
  }
  return st;
}

// ---------------------------------------------------------------------------
// Batched solve of a whole mesh group: the FP32 GMG-PCG inner solves and the
// FP64 refinement steps of all designs run in lockstep, one launch per
// kernel for all designs (the design is a grid dimension).  A design whose
// true residual already meets rtol, or that has stopped, sits out later outer
// steps (its inner tolerance is 1: its inner solve ends at once, x = 0 adds
// nothing); inner CG chunks run until every design's inner solve is done,
// finished designs' kernels returning at once.
// ---------------------------------------------------------------------------
namespace {

topo_status group_read_scalars(MeshGroup* G) {
  topo_mesh* m = G->meshes[0];
  CK(cudaMemcpy2DAsync(G->h_sc, sizeof(PcgScalars), m->sc, (size_t)G->S, sizeof(PcgScalars),
                       G->nb, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaMemcpy2DAsync(G->h_flag, sizeof(int), m->flags + 1, (size_t)G->S, sizeof(int), G->nb,
                       cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

// profile: events around every CG apply (design 0's events; one launch covers
// every design still iterating)
// Launch width for n live designs of a group of nb: 1, 2, 3, 4, 6, 8, 12,
// 16, 24, ... (at most 50 % padding, few distinct graphs), capped at nb.
int live_bucket(int n, int nb) {
  int w = 1;
  for (int p = 1;; p *= 2) {
    if (p >= n) { w = p; break; }
    if (p >= 2 && p + p / 2 >= n) { w = p + p / 2; break; }
  }
  return std::min(w, nb);
}

// bt: the designs the chunk covers (all of them, or the compacted list);
// kind: IK_GMG32, IK_JAC32 or IK_JAC64 (the single-design iterations of
// enqueue_iters with the design as a grid dimension)
topo_status group_enqueue_iters(MeshGroup* G, int kind, int count, bool profile, const Bat& bt) {
  topo_mesh* m = G->meshes[0];
  cudaStream_t s = m->stream;
  const int* done = &m->sc->done;
  for (int c = 0; c < count; ++c) {
    if (profile) CK(cudaEventRecordWithFlags(m->ev[2 * c], s, cudaEventRecordExternal));
    if (kind == IK_JAC64)
      LK(m, launch_apply<double>(m->p64, m->q64, m->E64, nullptr, m->d, m->k0d, MCD(m),
                                 red_of(m, FIN_ALPHA), APPLY_DOT, done, m->flags + 1, s, bt));
    else
      LK(m, launch_apply<float>(m->p32, m->q32, m->E32, nullptr, m->d, m->k0f, MCF(m),
                                red_of(m, FIN_ALPHA), APPLY_DOT, done, m->flags + 1, s, bt));
    if (profile) CK(cudaEventRecordWithFlags(m->ev[2 * c + 1], s, cudaEventRecordExternal));
    if (kind == IK_JAC64) {
      LK(m, launch_pcg_update<double>(m->x64, m->s64, m->z64, m->p64, m->q64, m->dinv64,
                                      m->nvec, red_of(m, FIN_UPDATE), true, s, bt));
      LK(m, launch_pcg_direction<double>(m->p64, m->z64, m->nvec, m->sc, s, bt));
      continue;
    }
    if (kind == IK_JAC32) {
      LK(m, launch_pcg_update<float>(m->x32, m->r32, m->z32, m->p32, m->q32, m->dinv32, m->nvec,
                                     red_of(m, FIN_UPDATE), true, s, bt));
    } else {  // the update also forms the V-cycle's first direction; z = V(r), with
              // r . z (beta) fused into the V-cycle's last smoothing step
      float* d0 = nullptr;
      const float th = gmg_first_direction(m->gmg, &d0);
      LK(m, launch_pcg_update<float>(m->x32, m->r32, d0 ? d0 : m->z32, m->p32, m->q32,
                                     d0 ? m->dinv32 : nullptr, m->nvec, red_of(m, FIN_RR_ONLY),
                                     false, s, bt, th));
      const Red zr = red_of(m, FIN_RZ_BETA);
      GmgProf gp;
      GmgProf* gpp = cheb_prof(m, profile, c, gp);
      CK(gmg_vcycle(m->gmg, m->r32, m->z32, m->k0f, MCF(m), done, m->flags + 1, s, &m->launches,
                    bt, &zr, d0 != nullptr, gpp));
      cheb_prof_done(m, gpp);
    }
    LK(m, launch_pcg_direction<float>(m->p32, m->z32, m->nvec, m->sc, s, bt));
  }
  return TOPO_OK;
}

// One chunk of CG iterations over `n` designs: all of the group (n == nb)
// or the first n entries of G->d_ids (already on the device).  One graph per
// (chunk length, profiling, n), so n takes few values (live_bucket).
topo_status group_run_iters(MeshGroup* G, int kind, int count, bool profile, int n) {
  topo_mesh* m = G->meshes[0];
  const bool all = n >= G->nb;
  const Bat bt{all ? G->nb : n, G->S, all ? nullptr : G->d_ids, G->nb};
  const long long key = (long long)count | ((long long)profile << 16) | ((long long)bt.nb << 20) |
                        ((long long)kind << 40);
  auto it = G->graphs.find(key);
  if (it == G->graphs.end()) {
    const long long l0 = m->launches;
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    const topo_status st = group_enqueue_iters(G, kind, count, profile, bt);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (st != TOPO_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != TOPO_OK ? st : cuda_status(e);
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(ei);
    ChunkGraph cg;
    cg.exec = ex;
    cg.launches = m->launches - l0;
    m->launches = l0;
    it = G->graphs.emplace(key, cg).first;
  }
  CK(cudaGraphLaunch(it->second.exec, m->stream));
  m->launches += it->second.launches;
  return TOPO_OK;
}

// The FP64 inner-CG vectors of every design of the group in one arena at the
// group stride (x64, s64, z64, p64, q64, dinv64 of design b at arena64 +
// b * S + q * vb).  A design that already had its own (a single-design FP64
// solve) gives them up: its stream is drained and its captured graphs, which
// hold the old addresses, are dropped first.
topo_status ensure_group_fp64(MeshGroup* G) {
  if (G->arena64) return TOPO_OK;
  topo_mesh* m0 = G->meshes[0];
  const long long vb = (m0->nvec * (long long)sizeof(double) + 255) / 256 * 256;
  if (6 * vb > G->S) return TOPO_ERR_INVALID;  // cannot happen: the region holds more
  const long long bytes = (long long)(G->nb - 1) * G->S + 6 * vb;
  void* a = nullptr;
  if (cudaMalloc(&a, (size_t)bytes) != cudaSuccess) {
    cudaGetLastError();
    return TOPO_ERR_OOM;
  }
  G->arena64 = static_cast<char*>(a);
  G->arena64_bytes = bytes;
  CK(cudaMemsetAsync(a, 0, (size_t)bytes, m0->stream));
  for (int b = 0; b < G->nb; ++b) {
    topo_mesh* m = G->meshes[b];
    double** v[6] = {&m->x64, &m->s64, &m->z64, &m->p64, &m->q64, &m->dinv64};
    if (m->x64) {
      CK(cudaStreamSynchronize(m->stream));
      clear_graphs(m);
      for (double** q : v) {
        if (*q) cudaFree(*q);
        m->bytes -= m->nvec * (long long)sizeof(double);
      }
    }
    for (int q = 0; q < 6; ++q)
      *v[q] = reinterpret_cast<double*>(G->arena64 + (long long)b * G->S + q * vb);
    m->bytes += 6 * vb;
    m->diag64 = false;
  }
  // every design's stream after the fill (design 0's stream runs the batch)
  CK(cudaEventRecord(m0->ev_in, m0->stream));
  for (int b = 1; b < G->nb; ++b) CK(cudaStreamWaitEvent(G->meshes[b]->stream, m0->ev_in, 0));
  return TOPO_OK;
}

// Can these meshes (in any order) be solved as their group, with these options?
MeshGroup* batchable(topo_mesh* const* meshes, int n, const topo_solve_opts& o) {
  if (n < 2) return nullptr;
  MeshGroup* G = meshes[0]->group;
  if (!G || G->nb != n) return nullptr;
  const bool gmg = o.precond == TOPO_PRECOND_GMG;
  if (gmg ? o.precision != TOPO_PREC_FP32
          : (o.precond != TOPO_PRECOND_JACOBI ||
             (o.precision != TOPO_PREC_FP32 && o.precision != TOPO_PREC_FP64)))
    return nullptr;
  if (o.residual != TOPO_RESIDUAL_DWORD && o.residual != TOPO_RESIDUAL_FP64) return nullptr;
  if (gmg && (o.gmg_levels != G->gmg_levels || o.smooth_degree != G->gmg_degree)) return nullptr;
  if (!(o.rtol > 0.0) || o.max_iter < 1 || o.max_outer < 1 || o.check_every < 1 ||
      o.check_every > 1024)
    return nullptr;
  for (int a = 0; a < n; ++a) {
    topo_mesh* m = meshes[a];
    if (m->group != G || !m->use_modal || m->mcf.form != G->meshes[0]->mcf.form)
      return nullptr;
    if (gmg && (!m->gmg.arena || !m->gmg_built || m->gmg_levels_req != G->gmg_levels ||
                m->gmg_degree != G->gmg_degree))
      return nullptr;
  }
  for (topo_mesh* m : G->meshes)
    if (!m) return nullptr;
  return G;
}

// infos[b]: design b of the group
topo_status group_solve(MeshGroup* G, const topo_solve_opts& o, topo_solve_info* infos) {
  Timer timer;
  const int nb = G->nb;
  topo_mesh* m = G->meshes[0];
  cudaStream_t s = m->stream;
  const Bat bt{nb, G->S};
  for (topo_mesh* q : G->meshes)
    if (!q->has_density) return TOPO_ERR_NO_DENSITY;
  // design 0's stream (which runs the batch) after every design's earlier work
  for (int b = 1; b < nb; ++b) {
    CK(cudaEventRecord(G->meshes[b]->ev_in, G->meshes[b]->stream));
    CK(cudaStreamWaitEvent(s, G->meshes[b]->ev_in, 0));
  }
  const int kind = o.precond == TOPO_PRECOND_GMG      ? IK_GMG32
                   : o.precision == TOPO_PREC_FP64    ? IK_JAC64
                                                      : IK_JAC32;
  if (kind == IK_JAC64) CKS(ensure_group_fp64(G));
  // setup for the current moduli (all designs at once)
  bool need_diag = false, need_gmg = false;
  for (topo_mesh* q : G->meshes) {
    need_diag |= kind == IK_JAC64 ? !q->diag64 : !q->diag32;
    need_gmg |= kind == IK_GMG32 && !q->gmg.ready;
  }
  if (kind == IK_JAC64 && need_diag) {
    LK(m, launch_diag_inv<double>(m->dinv64, m->E64, m->d, m->k0d, s, bt));
    for (topo_mesh* q : G->meshes) q->diag64 = true;
  } else if (need_diag || need_gmg) {
    LK(m, launch_diag_inv<float>(m->dinv32, m->E32, m->d, m->k0f, s, bt));
    for (topo_mesh* q : G->meshes) q->diag32 = true;
    if (kind == IK_GMG32) {
      CK(gmg_setup(m->gmg, m->E32, m->dinv32, m->k0f, m->k0d, s, &m->launches, bt));
      for (topo_mesh* q : G->meshes) {
        q->gmg.ready = true;
        q->gmg.lv[0].E = q->E32;  // each design's own hierarchy now describes its moduli
        q->gmg.lv[0].dinv = q->dinv32;
      }
    }
  }
  for (topo_mesh* q : G->meshes) q->solved = false;
  // design 0 holds the batch's FP32 operator timing
  const bool prof = m->prof && kind != IK_JAC64;
  if (prof) CKS(ensure_profile_events(m, o.check_every));
  CK(cudaMemset2DAsync(m->flags + 1, (size_t)G->S, 0, sizeof(int), nb, s));
  if (o.warm_start) {
    CKS(enqueue_residual(m, false, nullptr, bt));  // a warm start may already be converged
    for (topo_mesh* q : G->meshes) q->energy_fresh = q->use_modal;
  } else {
    CK(cudaMemset2DAsync(m->u64, (size_t)G->S, 0, sizeof(double) * m->nvec, nb, s));
    for (topo_mesh* q : G->meshes) q->energy_fresh = false;
    CK(cudaMemcpy2DAsync(m->r64, (size_t)G->S, m->f64, (size_t)G->S, sizeof(double) * m->nvec,
                         nb, cudaMemcpyDeviceToDevice, s));
    LK(m, launch_dot<double>(m->r64, m->r64, m->nvec, red_of(m, FIN_AUX), s, bt));
  }
  CKS(group_read_scalars(G));
  std::vector<int> outer(nb, 0), total(nb, 0), detail(nb, TOPO_FAIL_NONE);
  std::vector<topo_status> st(nb, TOPO_OK);
  std::vector<char> running(nb, 1);
  std::vector<double> rel(nb, 0.0), expect(nb, 1.0);
  std::vector<char> last_dword(nb, 0);  // design b's last residual was double-word
  for (;;) {
    // decisions on the fresh FP64 residuals
    int live = 0;
    for (int b = 0; b < nb; ++b) {
      MeshGroup::Next& nx = G->h_next[b];
      nx.rtol2 = 4.0;  // sit out
      nx.max_iter = 1;
      nx.sat_out = 1;
      nx.skip_dword = 1;
      nx.skip_fp64 = 1;
      if (!running[b]) continue;
      const PcgScalars& h = G->h_sc[b];
      const double fn = std::sqrt(G->meshes[b]->fnorm2), rr = h.aux[0];
      if (G->h_flag[b]) {
        st[b] = TOPO_ERR_TIMEOUT;
        detail[b] = TOPO_FAIL_TIMEOUT;
        running[b] = 0;
        continue;
      }
      if (!std::isfinite(rr)) {
        st[b] = TOPO_ERR_NAN;
        detail[b] = TOPO_FAIL_RESIDUAL;
        running[b] = 0;
        continue;
      }
      rel[b] = fn > 0 ? std::sqrt(rr) / fn : 0.0;
      if (rel[b] <= o.rtol && !last_dword[b]) {  // only an FP64 residual certifies
        running[b] = 0;
        continue;
      }
      if (outer[b] >= o.max_outer || total[b] >= o.max_iter) {
        st[b] = TOPO_ERR_NOT_CONVERGED;
        detail[b] = TOPO_FAIL_LIMIT;
        running[b] = 0;
        continue;
      }
      // FP64 inner CG: the final tolerance directly, with margin
      const double inner =
          kind == IK_JAC64
              ? std::min(std::max(0.5 * o.rtol * fn / std::sqrt(rr), 1e-15), 0.5)
              : std::min(std::max(o.inner_rtol, kInnerMargin * o.rtol * fn / std::sqrt(rr)), 0.5);
      expect[b] = inner * rel[b];
      const bool dw = dword_residual(o, expect[b]);
      nx.skip_dword = dw ? 0 : 1;
      nx.skip_fp64 = dw ? 1 : 0;
      nx.rtol2 = inner * inner;
      nx.max_iter = o.max_iter - total[b];
      nx.sat_out = 0;
      ++live;
    }
    if (!live) break;
    static_assert(sizeof(MeshGroup::Next) == 3 * sizeof(double) &&
                      offsetof(PcgScalars, skip_fp64) - offsetof(PcgScalars, rtol2_next) ==
                          offsetof(MeshGroup::Next, skip_fp64) &&
                      sizeof(PcgScalars) - offsetof(PcgScalars, rtol2_next) ==
                          sizeof(MeshGroup::Next),
                  "Next mirrors the tail of PcgScalars");
    CK(cudaMemcpy2DAsync(&m->sc->rtol2_next, (size_t)G->S, G->h_next, sizeof(MeshGroup::Next),
                         sizeof(MeshGroup::Next), nb, cudaMemcpyHostToDevice, s));
    // inner start: b = r / ||r|| in FP32 (FP64: b = r), x = 0, z = M^-1 r, p = z
    const int* done = &m->sc->done;
    LK(m, launch_set_max_iter(m->sc, -1, s, bt));
    if (kind == IK_JAC64) {
      LK(m, launch_pcg_init<double>(m->r64, m->x64, m->s64, m->z64, m->p64, m->dinv64, m->nvec,
                                    red_of(m, FIN_INIT, -1.0), true, s, bt));
    } else {
      LK(m, launch_narrow_scaled(m->b32, m->r64, m->nvec, m->sc, s, bt));
      if (kind == IK_JAC32) {
        LK(m, launch_pcg_init<float>(m->b32, m->x32, m->r32, m->z32, m->p32, m->dinv32, m->nvec,
                                     red_of(m, FIN_INIT, -1.0), true, s, bt));
      } else {
        LK(m, launch_pcg_init<float>(m->b32, m->x32, m->r32, m->z32, m->p32, nullptr, m->nvec,
                                     red_of(m, FIN_INIT, -1.0), false, s, bt));
        const Red zr = red_of(m, FIN_SET_RZ);
        CK(gmg_vcycle(m->gmg, m->r32, m->z32, m->k0f, MCF(m), done, m->flags + 1, s,
                      &m->launches, bt, &zr));
        LK(m, launch_pcg_direction<float>(m->p32, m->z32, m->nvec, m->sc, s, bt));
      }
    }
    std::vector<int> before(nb, -1), at(nb, 0);
    std::vector<char> iterating(running);  // designs not done (first chunk: taking part)
    for (int chunk = 0;; ++chunk) {
      // compact the chunk's launches to the live designs, padded with a
      // finished design (its CTAs return at once) up to the launch width
      int n_live = 0, idle = -1;
      for (int b = 0; b < nb; ++b) {
        if (iterating[b])
          G->h_ids[n_live++] = b;
        else if (idle < 0)
          idle = b;
      }
      const int width = live_bucket(n_live, nb);
      if (width < nb) {
        for (int q = n_live; q < width; ++q) G->h_ids[q] = idle;
        CK(cudaMemcpyAsync(G->d_ids, G->h_ids, sizeof(int) * width, cudaMemcpyHostToDevice, s));
      }
      CKS(group_run_iters(G, kind, o.check_every, prof, width));
      CKS(group_read_scalars(G));
      bool all_done = true, progress = false;
      for (int b = 0; b < nb; ++b) {
        const PcgScalars& h = G->h_sc[b];
        if (!h.done) all_done = false;
        if (h.iter != before[b]) progress = true;
        before[b] = h.iter;
        iterating[b] = !h.done;
      }
      if (prof) {  // launch c of the chunk advanced the designs with more than c iterations
        for (int c = 0; c < o.check_every; ++c) {
          int active = 0;
          for (int b = 0; b < nb; ++b) active += (G->h_sc[b].iter - at[b]) > c;
          if (!active) break;
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, m->ev[2 * c], m->ev[2 * c + 1]));
          m->prof_ms += ms;
          m->prof_launches += active;
          if (kind == IK_GMG32) CKS(cheb_prof_collect(m, c, active));
        }
        for (int b = 0; b < nb; ++b) at[b] = G->h_sc[b].iter;
      }
      if (all_done) break;
      if (!progress) return TOPO_ERR_CUDA;  // no design moved without stopping: a bug
    }
    for (int b = 0; b < nb; ++b) {
      if (!running[b]) continue;
      const PcgScalars& h = G->h_sc[b];
      total[b] += h.iter;
      ++outer[b];
      if (h.status == 2) {
        st[b] = TOPO_ERR_NAN;
        detail[b] = TOPO_FAIL_BREAKDOWN;
        running[b] = 0;
      }
    }
    // u += ||r|| x, then the FP64 residual, for the designs that took part
    // (those that sat out keep u and their residual)
    if (kind == IK_JAC64)
      LK(m, launch_accumulate<double>(m->u64, m->x64, m->nvec, m->sc, false, s, bt));
    else
      LK(m, launch_accumulate<float>(m->u64, m->x32, m->nvec, m->sc, true, s, bt));
    // double-word for the designs whose residual cannot end their solve,
    // FP64 for the others: one launch each, skipping the designs of the other
    bool any_dw = false, any_64 = false;
    for (int b = 0; b < nb; ++b) {
      const MeshGroup::Next& nx = G->h_next[b];
      any_dw |= nx.skip_dword == 0;
      any_64 |= nx.skip_fp64 == 0;
      if (!nx.sat_out) last_dword[b] = nx.skip_dword == 0;
    }
    if (any_dw) CKS(enqueue_residual(m, true, &m->sc->skip_dword, bt));
    if (any_64) CKS(enqueue_residual(m, false, &m->sc->skip_fp64, bt));
    for (int b = 0; b < nb; ++b)  // designs that took part have a new u
      if (!G->h_next[b].sat_out)
        G->meshes[b]->energy_fresh = G->h_next[b].skip_fp64 == 0 && G->meshes[b]->use_modal;
    CKS(group_read_scalars(G));
  }
  // every design's stream after the batch
  CK(cudaEventRecord(m->ev_in, s));
  for (int b = 1; b < nb; ++b) CK(cudaStreamWaitEvent(G->meshes[b]->stream, m->ev_in, 0));
  topo_status first = TOPO_OK;
  for (int b = 0; b < nb; ++b) {
    topo_mesh* q = G->meshes[b];
    q->solved = (st[b] == TOPO_OK);
    if (infos) {
      infos[b].iters = total[b];
      infos[b].outer = outer[b];
      infos[b].status = st[b];
      infos[b].detail = detail[b];
      infos[b].rel_residual = rel[b];
      infos[b].seconds = timer.seconds();
    }
    if (st[b] != TOPO_OK && first == TOPO_OK) first = st[b];
  }
  return first;
}

}  // namespace

topo_status topo_solve_many(topo_mesh* const* meshes, int n, const topo_solve_opts* opts,
                            topo_solve_info* infos) {
  if (n < 0 || (n > 0 && !meshes)) return TOPO_ERR_INVALID;
  for (int a = 0; a < n; ++a) {
    if (!meshes[a]) return TOPO_ERR_INVALID;
    for (int b = 0; b < a; ++b)
      if (meshes[a] == meshes[b]) return TOPO_ERR_INVALID;  // one task per mesh
  }
  topo_solve_opts o;
  if (opts)
    o = *opts;
  else
    topo_default_opts(&o);
  if (MeshGroup* G = batchable(meshes, n, o)) {
    std::vector<std::unique_ptr<Fence>> fences;
    topo_status fst = TOPO_OK;
    for (int a = 0; a < n; ++a) {
      if (infos) std::memset(&infos[a], 0, sizeof(topo_solve_info));
      fences.emplace_back(new Fence(meshes[a]));
      if (fences.back()->st != TOPO_OK) fst = fences.back()->st;
    }
    if (fst != TOPO_OK) return fst;
    std::vector<topo_solve_info> by_design(G->nb);
    const topo_status st = group_solve(G, o, by_design.data());
    if (infos)
      for (int a = 0; a < n; ++a) {
        infos[a] = by_design[meshes[a]->gidx];
        if (st != TOPO_OK && infos[a].status == TOPO_OK && !meshes[a]->solved)
          infos[a].status = st;
      }
    return st;  // the fences order every caller stream after its design
  }
  std::vector<SolveTask> tasks(n);
  std::vector<std::unique_ptr<Fence>> fences;
  fences.reserve(n);
  for (int a = 0; a < n; ++a) {
    if (infos) std::memset(&infos[a], 0, sizeof(topo_solve_info));
    fences.emplace_back(new Fence(meshes[a]));
    SolveTask& t = tasks[a];
    t.m = meshes[a];
    t.o = o;
    t.info = infos ? &infos[a] : nullptr;
    const topo_status st = fences.back()->st != TOPO_OK ? fences.back()->st : task_start(t);
    if (st != TOPO_OK) task_finish(t, st);
  }
  // round-robin: advance every task whose scalars have arrived
  for (;;) {
    int active = 0, progressed = 0;
    for (SolveTask& t : tasks) {
      if (t.phase == SolveTask::P_FINISHED) continue;
      ++active;
      cudaSetDevice(t.m->dev);
      const cudaError_t q = cudaEventQuery(t.m->ev_poll);
      if (q == cudaSuccess) {
        task_advance(t);
        ++progressed;
      } else if (q != cudaErrorNotReady) {
        cudaGetLastError();
        task_finish(t, cuda_status(q));
      }
    }
    if (!active) break;
    if (!progressed) std::this_thread::yield();
  }
  fences.clear();  // make every caller stream wait for its mesh
  topo_status first = TOPO_OK;
  for (const SolveTask& t : tasks)
    if (t.st != TOPO_OK && first == TOPO_OK) first = t.st;
  return first;
}

// the element energies the last FP64 residual stored are those of u
static bool energies_usable(const topo_mesh* m) { return m->energy_fresh && m->e_positive; }

namespace {

// The meshes, in order, are a whole mesh group: its group, else nullptr.
MeshGroup* whole_group(topo_mesh* const* meshes, int n) {
  if (n < 2 || !meshes || !meshes[0]) return nullptr;
  MeshGroup* G = meshes[0]->group;
  if (!G || G->nb != n) return nullptr;
  for (int b = 0; b < n; ++b)
    if (meshes[b] != G->meshes[b]) return nullptr;
  return G;
}

// Orders one batched operation of a whole group on design 0's stream: after
// the callers' streams and every design's earlier work, and every design's
// stream (then its caller's) after it.
struct GroupScope {
  MeshGroup* G;
  std::vector<std::unique_ptr<Fence>> fences;
  topo_status st = TOPO_OK;
  explicit GroupScope(MeshGroup* g) : G(g) {
    for (topo_mesh* m : G->meshes) {
      fences.emplace_back(new Fence(m));
      if (fences.back()->st != TOPO_OK) st = fences.back()->st;
    }
    cudaStream_t s0 = G->meshes[0]->stream;
    for (int b = 1; b < G->nb && st == TOPO_OK; ++b)
      if (cudaEventRecord(G->meshes[b]->ev_in, G->meshes[b]->stream) != cudaSuccess ||
          cudaStreamWaitEvent(s0, G->meshes[b]->ev_in, 0) != cudaSuccess)
        st = TOPO_ERR_CUDA;
  }
  ~GroupScope() {
    topo_mesh* m0 = G->meshes[0];
    if (cudaEventRecord(m0->ev_in, m0->stream) == cudaSuccess)
      for (int b = 1; b < G->nb; ++b) cudaStreamWaitEvent(G->meshes[b]->stream, m0->ev_in, 0);
  }
  GroupScope(const GroupScope&) = delete;
  GroupScope& operator=(const GroupScope&) = delete;
};

topo_status ensure_stage(MeshGroup* G, size_t bytes) {
  if (G->stage_bytes >= bytes) return TOPO_OK;
  if (G->stage) cudaFree(G->stage);
  G->stage = nullptr;
  G->stage_bytes = 0;
  if (cudaMalloc(&G->stage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return TOPO_ERR_OOM;
  }
  G->stage_bytes = bytes;
  return TOPO_OK;
}

// Every mesh non-null, distinct, of the grid n_elem describes (0: any).
topo_status check_many(topo_mesh* const* meshes, int n, long long n_elem) {
  if (n < 1 || !meshes) return TOPO_ERR_INVALID;
  for (int a = 0; a < n; ++a) {
    if (!meshes[a]) return TOPO_ERR_INVALID;
    const Dims& d = meshes[a]->d;
    if (n_elem && (long long)d.nx * d.ny * d.nz != n_elem) return TOPO_ERR_INVALID;
    for (int b = 0; b < a; ++b)
      if (meshes[a] == meshes[b]) return TOPO_ERR_INVALID;
  }
  return TOPO_OK;
}

}  // namespace

topo_status topo_set_density_many(topo_mesh* const* meshes, int n, const float* rho,
                                  size_t n_elem, int on_device) {
  if (!rho) return TOPO_ERR_INVALID;
  CKS(check_many(meshes, n, (long long)n_elem));
  MeshGroup* G = whole_group(meshes, n);
  if (!G) {
    topo_status first = TOPO_OK;
    for (int b = 0; b < n; ++b) {
      const topo_status st = topo_set_density(meshes[b], rho + (size_t)b * n_elem, n_elem, on_device);
      if (st != TOPO_OK && first == TOPO_OK) first = st;
    }
    return first;
  }
  GroupScope scope(G);
  if (scope.st != TOPO_OK) return scope.st;
  topo_mesh* m0 = G->meshes[0];
  cudaStream_t s = m0->stream;
  const float* src = rho;
  if (!on_device) {
    CKS(ensure_stage(G, sizeof(float) * n_elem * n));
    CK(cudaMemcpyAsync(G->stage, rho, sizeof(float) * n_elem * n, cudaMemcpyHostToDevice, s));
    src = static_cast<const float*>(G->stage);
  }
  const Bat bt{G->nb, G->S};
  CK(cudaMemset2DAsync(m0->flags, (size_t)G->S, 0, sizeof(int), G->nb, s));
  LK(m0, launch_simp(src, m0->rho_g, m0->E32, m0->E64, m0->d, G->prm.E0, G->prm.Emin,
                     G->prm.penal, G->prm.h, m0->flags, s, m0->rho_in, (long long)n_elem, bt));
  CK(cudaMemcpy2DAsync(G->h_flag, sizeof(int), m0->flags, (size_t)G->S, sizeof(int), G->nb,
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  topo_status first = TOPO_OK;
  for (int b = 0; b < n; ++b) {
    topo_mesh* m = G->meshes[b];
    m->diag32 = m->diag64 = false;
    m->gmg.ready = false;
    m->solved = false;
    m->energy_fresh = false;
    m->e_positive = G->prm.Emin > 0.0;
    m->has_density = (G->h_flag[b] == 0);
    if (!m->has_density && first == TOPO_OK) first = TOPO_ERR_NAN;
  }
  return first;
}

topo_status topo_compliance_many(topo_mesh* const* meshes, int n, double* c) {
  if (!c) return TOPO_ERR_INVALID;
  CKS(check_many(meshes, n, 0));
  MeshGroup* G = whole_group(meshes, n);
  if (!G) {
    for (int b = 0; b < n; ++b) CKS(topo_compliance(meshes[b], &c[b]));
    return TOPO_OK;
  }
  for (int b = 0; b < n; ++b)
    if (!meshes[b]->solved) return TOPO_ERR_NOT_SOLVED;
  GroupScope scope(G);
  if (scope.st != TOPO_OK) return scope.st;
  topo_mesh* m0 = G->meshes[0];
  LK(m0, launch_dot<double>(m0->f64, m0->u64, m0->nvec, red_of(m0, FIN_AUX), m0->stream,
                            Bat{G->nb, G->S}));
  CKS(group_read_scalars(G));
  for (int b = 0; b < n; ++b) c[b] = G->h_sc[b].aux[0];
  return TOPO_OK;
}

topo_status topo_sensitivity_many(topo_mesh* const* meshes, int n, double* dc, size_t n_elem,
                                  int on_device) {
  if (!dc) return TOPO_ERR_INVALID;
  CKS(check_many(meshes, n, (long long)n_elem));
  MeshGroup* G = whole_group(meshes, n);
  if (!G) {
    for (int b = 0; b < n; ++b)
      CKS(topo_sensitivity(meshes[b], dc + (size_t)b * n_elem, n_elem, on_device));
    return TOPO_OK;
  }
  for (int b = 0; b < n; ++b)
    if (!meshes[b]->solved) return TOPO_ERR_NOT_SOLVED;
  GroupScope scope(G);
  if (scope.st != TOPO_OK) return scope.st;
  topo_mesh* m0 = G->meshes[0];
  cudaStream_t s = m0->stream;
  double* out = dc;
  if (!on_device) {
    CKS(ensure_stage(G, sizeof(double) * n_elem * n));
    out = static_cast<double*>(G->stage);
  }
  bool all_fresh = true;
  for (topo_mesh* q : G->meshes) all_fresh &= energies_usable(q);
  const double dE = (G->prm.E0 - G->prm.Emin) * G->prm.h;
  if (all_fresh)
    LK(m0, launch_sens_energy(m0->energy, m0->rho_g, m0->E64, out, m0->d, G->prm.penal, dE,
                              red_of(m0, FIN_AUX), s, (long long)n_elem, Bat{G->nb, G->S}));
  else
    LK(m0, launch_sensitivity(m0->u64, m0->rho_g, m0->E64, out, m0->d, m0->mcd, G->prm.penal,
                              dE, red_of(m0, FIN_AUX), s, (long long)n_elem, Bat{G->nb, G->S}));
  if (!on_device) {
    CK(cudaMemcpyAsync(dc, out, sizeof(double) * n_elem * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return TOPO_OK;
}

topo_status topo_compliance(topo_mesh* m, double* c) {
  if (!m || !c) return TOPO_ERR_INVALID;
  if (!m->solved) return TOPO_ERR_NOT_SOLVED;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  LK(m, launch_dot<double>(m->f64, m->u64, m->nvec, red_of(m, FIN_AUX), m->stream));
  CKS(sync_scalars(m));
  *c = m->h_sc->aux[0];
  return TOPO_OK;
}

static topo_status sens_impl(topo_mesh* m) {
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if (!m->dc) CKS(dalloc(m, &m->dc, ne));
  const double dE = (m->prm.E0 - m->prm.Emin) * m->prm.h;
  if (energies_usable(m))
    LK(m, launch_sens_energy(m->energy, m->rho_g, m->E64, m->dc, m->d, m->prm.penal, dE,
                             red_of(m, FIN_AUX), m->stream));
  else
    LK(m, launch_sensitivity(m->u64, m->rho_g, m->E64, m->dc, m->d, m->mcd, m->prm.penal, dE,
                             red_of(m, FIN_AUX), m->stream));
  return TOPO_OK;
}

topo_status topo_compliance_energy(topo_mesh* m, double* c) {
  if (!m || !c) return TOPO_ERR_INVALID;
  if (!m->solved) return TOPO_ERR_NOT_SOLVED;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(sens_impl(m));
  CKS(sync_scalars(m));
  *c = m->h_sc->aux[0];
  return TOPO_OK;
}

topo_status topo_sensitivity(topo_mesh* m, double* dc, size_t n_elem, int on_device) {
  if (!m || !dc) return TOPO_ERR_INVALID;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if ((long long)n_elem != ne) return TOPO_ERR_INVALID;
  if (!m->solved) return TOPO_ERR_NOT_SOLVED;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(sens_impl(m));
  CK(cudaMemcpyAsync(dc, m->dc, ne * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_get_displacement(topo_mesh* m, double* u, size_t n_dof, int on_device) {
  if (!m || !u) return TOPO_ERR_INVALID;
  const long long nd = 3LL * (m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
  if ((long long)n_dof != nd) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  double* dst = on_device ? u : m->aos;
  LK(m, launch_pack<double>(m->u64, dst, m->d, m->stream));
  if (!on_device) {
    CK(cudaMemcpyAsync(u, m->aos, nd * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
  }
  return TOPO_OK;
}

topo_status topo_jacobi_inverse(topo_mesh* m, double* dinv, size_t n_dof, int on_device) {
  if (!m || !dinv) return TOPO_ERR_INVALID;
  if (!m->has_density) return TOPO_ERR_NO_DENSITY;
  const long long nd = 3LL * (m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
  if ((long long)n_dof != nd) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(ensure_fp64_inner(m));
  if (!m->diag64) {
    LK(m, launch_diag_inv<double>(m->dinv64, m->E64, m->d, m->k0d, m->stream));
    m->diag64 = true;
  }
  double* dst = on_device ? dinv : m->aos;
  LK(m, launch_pack<double>(m->dinv64, dst, m->d, m->stream));
  if (!on_device) {
    CK(cudaMemcpyAsync(dinv, m->aos, nd * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
  }
  return TOPO_OK;
}

topo_status topo_set_displacement(topo_mesh* m, const double* u, size_t n_dof, int on_device) {
  if (!m || !u) return TOPO_ERR_INVALID;
  const long long nd = 3LL * (m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
  if ((long long)n_dof != nd) return TOPO_ERR_INVALID;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(upload_f64(m, u, m->u64, n_dof, on_device));
  m->solved = false;
  m->energy_fresh = false;
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_apply(topo_mesh* m, int precision, const double* x, double* y, size_t n_dof,
                       int on_device) {
  if (!m || !x || !y) return TOPO_ERR_INVALID;
  if (precision != TOPO_PREC_FP64 && precision != TOPO_PREC_FP32 && precision != TOPO_PREC_DWORD)
    return TOPO_ERR_INVALID;
  const long long nd = 3LL * (m->d.nx + 1) * (m->d.ny + 1) * (m->d.nz + 1);
  if ((long long)n_dof != nd) return TOPO_ERR_INVALID;
  if (!m->has_density) return TOPO_ERR_NO_DENSITY;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  cudaStream_t s = m->stream;
  const double* src = x;
  if (!on_device) {
    CK(cudaMemcpyAsync(m->aos, x, nd * sizeof(double), cudaMemcpyHostToDevice, s));
    src = m->aos;
  }
  if (precision == TOPO_PREC_FP64) {
    CKS(ensure_fp64_inner(m));
    LK(m, launch_unpack<double>(src, m->p64, m->d, s));
    LK(m, launch_apply<double>(m->p64, m->q64, m->E64, nullptr, m->d, m->k0d, MCD(m), red_of(m, FIN_NONE),
                            APPLY_PLAIN, nullptr, m->flags + 1, s));
    LK(m, launch_pack<double>(m->q64, on_device ? y : m->aos, m->d, s));
  } else if (precision == TOPO_PREC_DWORD) {
    CKS(ensure_fp64_inner(m));
    LK(m, launch_unpack<double>(src, m->p64, m->d, s));
    LK(m, launch_split_dw(m->p64, m->p32, m->q32, m->nvec, nullptr, s));
    LK(m, launch_apply_dw(m->p32, m->q32, m->q64, m->E64, nullptr, m->d, m->mcd,
                          red_of(m, FIN_NONE), APPLY_PLAIN, nullptr, s));
    LK(m, launch_pack<double>(m->q64, on_device ? y : m->aos, m->d, s));
  } else {
    LK(m, launch_unpack<float>(src, m->p32, m->d, s));
    LK(m, launch_apply<float>(m->p32, m->q32, m->E32, nullptr, m->d, m->k0f, MCF(m), red_of(m, FIN_NONE),
                           APPLY_PLAIN, nullptr, m->flags + 1, s));
    LK(m, launch_pack<float>(m->q32, on_device ? y : m->aos, m->d, s));
  }
  if (!on_device) {
    CK(cudaMemcpyAsync(y, m->aos, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return TOPO_OK;
}

topo_status topo_apply_internal(topo_mesh* m, int precision, int reps) {
  if (!m || reps < 0) return TOPO_ERR_INVALID;
  if (!m->has_density) return TOPO_ERR_NO_DENSITY;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  for (int r = 0; r < reps; ++r) {
    if (precision == TOPO_PREC_FP64) {
      CKS(ensure_fp64_inner(m));
      LK(m, launch_apply<double>(m->p64, m->q64, m->E64, nullptr, m->d, m->k0d, MCD(m),
                              red_of(m, FIN_NONE), APPLY_PLAIN, nullptr, m->flags + 1, m->stream));
    } else if (precision == TOPO_PREC_FP32) {
      LK(m, launch_apply<float>(m->p32, m->q32, m->E32, nullptr, m->d, m->k0f, MCF(m), red_of(m, FIN_NONE),
                             APPLY_PLAIN, nullptr, m->flags + 1, m->stream));
    } else if (precision == TOPO_PREC_DWORD) {
      CKS(ensure_fp64_inner(m));
      LK(m, launch_apply_dw(m->p32, m->q32, m->q64, m->E64, nullptr, m->d, m->mcd,
                            red_of(m, FIN_NONE), APPLY_PLAIN, nullptr, m->stream));
    } else {
      return TOPO_ERR_INVALID;
    }
  }
  return TOPO_OK;
}

topo_status topo_mesh_info(const topo_mesh* m, long long* n_nodes, long long* n_free_dof,
                           long long* device_bytes) {
  if (!m) return TOPO_ERR_INVALID;
  const Dims& d = m->d;
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  long long fixed = 0;
  const long long face = (long long)(d.ny + 1) * (d.nz + 1);
  if (d.bc == BC_CANTILEVER)
    fixed = 3 * face;
  else if (d.bc == BC_MBB)
    fixed = face + (d.ny + 1) + 1;
  else if (d.bc == BC_MBB_STRIP)
    fixed = face + 2 * (d.ny + 1) + 1;
  else if (d.bc == BC_NONE)
    fixed = 0;
  else if (d.bc == BC_CORNERS)  // supported rows x supported layers on x = 0, all components
    fixed = 3LL * std::min(2 * (d.corner_j + 1), d.ny + 1) *
            (long long)std::min(2 * (d.corner_k + 1), d.nz + 1);
  else
    fixed = face + (long long)(d.nx + 1) * (d.nz + 1) + (long long)(d.nx + 1) * (d.ny + 1);
  if (n_nodes) *n_nodes = nn;
  if (n_free_dof) *n_free_dof = 3 * nn - fixed;
  if (device_bytes) *device_bytes = m->bytes;
  return TOPO_OK;
}

long long topo_footprint_bytes(int nx, int ny, int nz, const topo_solve_opts* opts) {
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  Dims d = make_dims(nx, ny, nz, 0, ny / 2);
  const long long nvec = 3 * d.comp;
  long long b = d.ecount * (4 + 4 + 8 + 8);  // rho, E32, E64, element energies
  b += nvec * (3 * 8 + 7 * 4);                // f, u, r (FP64) + 7 FP32 CG vectors
  b += (long long)sizeof(PcgScalars) + 4LL * kMaxPartials * 8 + 16;
  b += 3LL * (nx + 1) * (ny + 1) * (nz + 1) * 8;  // ABI staging
  b += (long long)nx * ny * nz * (8 + 4);          // sensitivities + density staging
  if (opts && opts->precision == TOPO_PREC_FP64) b += nvec * 6 * 8;
  if (!opts || opts->precond == TOPO_PRECOND_GMG) b += gmg_footprint(d, opts ? opts->gmg_levels : 0);
  return b;
}

void topo_default_simp_opts(topo_simp_opts* o) {
  if (!o) return;
  o->volfrac = 0.4;
  o->filter_radius = 2.0;
  o->move = 0.2;
  o->eta = 0.5;
  o->rho_min = 1e-3;
}

static topo_status ensure_simp_buffers(topo_mesh* m) {
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if (!m->dc) CKS(dalloc(m, &m->dc, ne));
  if (!m->dcf) CKS(dalloc(m, &m->dcf, ne));
  if (!m->rho_next) CKS(dalloc(m, &m->rho_next, ne));
  if (!m->oc_state) {
    unsigned char* p = nullptr;
    CKS(dalloc(m, &p, (long long)oc_state_bytes()));
    m->oc_state = p;
  }
  if (!m->oc_part) CKS(dalloc(m, &m->oc_part, (long long)oc_partials_count()));
  if (!m->oc_host) CK(cudaMallocHost(&m->oc_host, oc_state_bytes()));
  return TOPO_OK;
}

topo_status topo_filter(topo_mesh* m, double radius, const double* dc, double* dcf, size_t n_elem,
                        int on_device) {
  if (!m || !dc || !dcf || !(radius > 0.0) || radius > 2.9) return TOPO_ERR_INVALID;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if ((long long)n_elem != ne) return TOPO_ERR_INVALID;
  if (!m->has_density) return TOPO_ERR_NO_DENSITY;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(ensure_simp_buffers(m));
  cudaStream_t s = m->stream;
  const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(m->dc, dc, ne * sizeof(double), in, s));
  LK(m, launch_filter(m->dc, m->rho_g, m->dcf, m->d, radius, 1e-3, s));
  CK(cudaMemcpyAsync(dcf, m->dcf, ne * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!on_device) CK(cudaStreamSynchronize(s));
  m->solved = false;  // the stored sensitivities were overwritten
  return TOPO_OK;
}

topo_status topo_simp_update(topo_mesh* m, const topo_simp_opts* opts, topo_simp_info* info) {
  if (!m) return TOPO_ERR_INVALID;
  topo_simp_opts o;
  if (opts)
    o = *opts;
  else
    topo_default_simp_opts(&o);
  if (!(o.volfrac > 0.0 && o.volfrac <= 1.0) || !(o.filter_radius > 0.0) ||
      o.filter_radius > 2.9 || !(o.move > 0.0) || !(o.eta > 0.0) || !(o.rho_min >= 0.0) ||
      o.rho_min >= o.volfrac)
    return TOPO_ERR_INVALID;
  if (!m->solved) return TOPO_ERR_NOT_SOLVED;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CKS(ensure_simp_buffers(m));
  cudaStream_t s = m->stream;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  // J = f^T u of the solved state, then Eq. (3) -> Eq. (4) -> OC
  LK(m, launch_dot<double>(m->f64, m->u64, m->nvec, red_of(m, FIN_AUX), s));
  CKS(sync_scalars(m));
  const double J = m->h_sc->aux[0];
  LK(m, launch_sensitivity(m->u64, m->rho_g, m->E64, m->dc, m->d, m->mcd, m->prm.penal,
                           (m->prm.E0 - m->prm.Emin) * m->prm.h, red_of(m, FIN_AUX), s));
  LK(m, launch_filter(m->dc, m->rho_g, m->dcf, m->d, o.filter_radius, 1e-3, s));
  const int passes = 8;
  CK(launch_oc(m->rho_in, m->dcf, m->rho_next, ne, o.volfrac, o.move, o.eta, o.rho_min, passes,
               m->oc_state, m->oc_part, s));
  m->launches += 2 + passes;
  CK(cudaMemcpyAsync(m->oc_host, m->oc_state, oc_state_bytes(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double sum = 0.0, change = 0.0, lam = 0.0;
  oc_results(m->oc_host, &sum, &change, &lam);
  // the new densities become the mesh's (E by Eq. (1)); u stays for a warm start
  CKS(set_density_impl(m, m->rho_next));
  if (info) {
    info->compliance = J;
    info->volume = sum / (double)ne;
    info->change = change;
    info->lambda = lam;
  }
  return TOPO_OK;
}

topo_status topo_get_density(topo_mesh* m, float* rho, size_t n_elem, int on_device) {
  if (!m || !rho) return TOPO_ERR_INVALID;
  const long long ne = (long long)m->d.nx * m->d.ny * m->d.nz;
  if ((long long)n_elem != ne) return TOPO_ERR_INVALID;
  if (!m->has_density) return TOPO_ERR_NO_DENSITY;
  Fence fence(m);
  if (fence.st != TOPO_OK) return fence.st;
  CK(cudaMemcpyAsync(rho, m->rho_in, ne * sizeof(float),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_set_operator(topo_mesh* m, int kind) {
  if (!m || kind < TOPO_OPERATOR_MODAL || kind > TOPO_OPERATOR_MODAL_CLUSTER)
    return TOPO_ERR_INVALID;
  const bool modal = (kind != TOPO_OPERATOR_GATHER);
  const int form = kind == TOPO_OPERATOR_MODAL_SINGLE    ? 1
                   : kind == TOPO_OPERATOR_MODAL_PAIR    ? 2
                   : kind == TOPO_OPERATOR_TENSOR        ? 3
                   : kind == TOPO_OPERATOR_MODAL_CLUSTER ? 4
                                                         : 0;
  if (modal != m->use_modal || form != m->mcf.form) {
    CK(cudaSetDevice(m->dev));
    CK(cudaStreamSynchronize(m->stream));
    clear_graphs(m);  // the captured chunks hold the old kernels
    if (m->group) {   // and so do the group's batched chunks
      for (topo_mesh* q : m->group->meshes)
        if (q) CK(cudaStreamSynchronize(q->stream));
      for (auto& kv : m->group->graphs) cudaGraphExecDestroy(kv.second.exec);
      m->group->graphs.clear();
    }
    m->use_modal = modal;
    m->mcf.form = form;
  }
  return TOPO_OK;
}

topo_status topo_set_stream(topo_mesh* m, void* stream) {
  if (!m) return TOPO_ERR_INVALID;
  m->user = static_cast<cudaStream_t>(stream);
  return TOPO_OK;
}

topo_status topo_profile_enable(topo_mesh* m, int enable) {
  if (!m) return TOPO_ERR_INVALID;
  m->prof = enable != 0;
  return TOPO_OK;
}

topo_status topo_set_throughput_mode(topo_mesh* m, int enable) {
  if (!m || (enable != 0 && enable != 1)) return TOPO_ERR_INVALID;
  if (m->group) return TOPO_ERR_INVALID;  // mesh groups run their coarse end batched anyway
  if ((enable != 0) == m->throughput) return TOPO_OK;
  CK(cudaSetDevice(m->dev));
  CK(cudaStreamSynchronize(m->stream));
  clear_graphs(m);  // the captured chunks hold the old hierarchy
  if (m->gmg_built) {
    m->bytes -= m->gmg.bytes;
    gmg_free(m->gmg);
    m->gmg = Gmg();
    m->gmg_built = false;
  }
  m->throughput = enable != 0;
  return TOPO_OK;
}

topo_status topo_debug_inject_timeout(topo_mesh* m, int count) {
  if (!m || count < 0 || count > 1) return TOPO_ERR_INVALID;
  Fence f(m);
  if (f.st != TOPO_OK) return f.st;
  CK(cudaMemcpyAsync(m->flags + 2, &count, sizeof(int), cudaMemcpyHostToDevice, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return TOPO_OK;
}

topo_status topo_profile_read_smoother(topo_mesh* m, double* total_ms, long long* launches,
                                       double* bytes, int reset) {
  if (!m) return TOPO_ERR_INVALID;
  if (total_ms) *total_ms = m->profc_ms;
  if (launches) *launches = m->profc_launches;
  if (bytes) *bytes = m->profc_bytes;
  if (reset) {
    m->profc_ms = 0.0;
    m->profc_bytes = 0.0;
    m->profc_launches = 0;
  }
  return TOPO_OK;
}

topo_status topo_profile_read(topo_mesh* m, double* total_ms, long long* launches,
                              long long* all_launches, int reset) {
  if (!m) return TOPO_ERR_INVALID;
  if (total_ms) *total_ms = m->prof_ms;
  if (launches) *launches = m->prof_launches;
  if (all_launches) *all_launches = m->launches;
  if (reset) {
    m->prof_ms = 0.0;
    m->prof_launches = 0;
    m->launches = 0;
  }
  return TOPO_OK;
}

topo_status topo_server_create(long long mem_budget_bytes, int max_active, const topo_params* prm,
                               const topo_solve_opts* opts, void* stream, topo_server** out) {
  if (!out || mem_budget_bytes <= 0 || max_active < 1) return TOPO_ERR_INVALID;
  topo_server* s = new (std::nothrow) topo_server();
  if (!s) return TOPO_ERR_OOM;
  s->budget = mem_budget_bytes;
  s->max_active = max_active;
  s->user = static_cast<cudaStream_t>(stream);
  if (prm)
    s->prm = *prm;
  else
    topo_default_params(&s->prm);
  if (opts)
    s->opts = *opts;
  else
    topo_default_opts(&s->opts);
  *out = s;
  return TOPO_OK;
}

topo_status topo_server_open(topo_server* s, int nx, int ny, int nz, int bc, int load,
                             int* design) {
  if (!s || !design) return TOPO_ERR_INVALID;
  if (nx < 1 || ny < 1 || nz < 1 || bc < 0 || bc > 5 || load < 0 || load > 4) return TOPO_ERR_INVALID;
  if ((bc == TOPO_BC_MBB || bc == TOPO_BC_MBB_STRIP) && (ny % 2)) return TOPO_ERR_INVALID;
  const long long fp = topo_footprint_bytes(nx, ny, nz, &s->opts);
  if (fp > s->budget) return TOPO_ERR_OOM;  // could never be admitted
  ServerDesign d;
  d.id = s->next_design++;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.bc = bc;
  d.load = load;
  d.footprint = fp;
  s->designs[d.id] = std::move(d);
  *design = s->designs.rbegin()->first;
  return TOPO_OK;
}

topo_status topo_server_submit(topo_server* s, int design, const float* rho, size_t n_elem,
                               int* job) {
  if (!s || !rho) return TOPO_ERR_INVALID;
  auto it = s->designs.find(design);
  if (it == s->designs.end() || it->second.closing) return TOPO_ERR_INVALID;
  ServerDesign& d = it->second;
  if ((long long)n_elem != (long long)d.nx * d.ny * d.nz) return TOPO_ERR_INVALID;
  ServerJob j;
  j.id = s->next_job++;
  j.rho.assign(rho, rho + n_elem);
  j.submit_s = s->clock.seconds();
  d.queue.push_back(std::move(j));
  if (!d.mesh && !d.waiting) {
    d.waiting = true;
    s->admit.push_back(d.id);
  }
  if (job) *job = s->next_job - 1;
  return TOPO_OK;
}

topo_status topo_server_poll(topo_server* s, int wait, topo_job_result* out, int max_out,
                             int* n_out) {
  if (!s || (max_out > 0 && !out) || max_out < 0) return TOPO_ERR_INVALID;
  for (;;) {
    const bool moved = server_step(s);
    if (!s->done.empty() || !wait || !server_busy(s)) break;
    if (!moved) std::this_thread::yield();
  }
  int n = 0;
  while (n < max_out && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  if (n_out) *n_out = n;
  return TOPO_OK;
}

static ServerDesign* idle_design(topo_server* s, int design) {
  auto it = s->designs.find(design);
  if (it == s->designs.end() || !it->second.mesh || it->second.running) return nullptr;
  return &it->second;
}

topo_status topo_server_sensitivity(topo_server* s, int design, double* dc, size_t n_elem,
                                    int on_device) {
  if (!s) return TOPO_ERR_INVALID;
  ServerDesign* d = idle_design(s, design);
  if (!d) return TOPO_ERR_INVALID;
  return topo_sensitivity(d->mesh, dc, n_elem, on_device);
}

topo_status topo_server_displacement(topo_server* s, int design, double* u, size_t n_dof,
                                     int on_device) {
  if (!s) return TOPO_ERR_INVALID;
  ServerDesign* d = idle_design(s, design);
  if (!d) return TOPO_ERR_INVALID;
  return topo_get_displacement(d->mesh, u, n_dof, on_device);
}

topo_status topo_server_close(topo_server* s, int design) {
  if (!s) return TOPO_ERR_INVALID;
  auto it = s->designs.find(design);
  if (it == s->designs.end()) return TOPO_ERR_INVALID;
  it->second.closing = true;
  if (!it->second.mesh) {  // never admitted: drop it and its queued jobs
    s->admit.erase(std::remove(s->admit.begin(), s->admit.end(), design), s->admit.end());
    s->designs.erase(it);
  }
  return TOPO_OK;
}

topo_status topo_server_stats(const topo_server* s, long long* bytes_in_use, long long* peak_bytes,
                              int* active, int* waiting) {
  if (!s) return TOPO_ERR_INVALID;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (peak_bytes) *peak_bytes = s->peak;
  if (active) *active = s->active;
  if (waiting) *waiting = (int)s->admit.size();
  return TOPO_OK;
}

void topo_server_free(topo_server* s) {
  if (!s) return;
  for (auto& kv : s->designs) {
    ServerDesign& d = kv.second;
    if (d.mesh) {
      cudaSetDevice(d.mesh->dev);
      cudaStreamSynchronize(d.mesh->stream);
    }
    server_release(s, d);
  }
  delete s;
}

}  // extern "C"
