// Geometric multigrid V-cycle preconditioner for the masked stiffness
// operator (the paper leaves the solver of Eq. (2) open; this is the
// library's choice).  Grids are vertex-nested 2:1 coarsenings of the
// structured hex grid (odd element counts round up, the extra half element
// having E = 0); coarse operators are rediscretised with the mean child
// modulus on elements of twice the edge; smoothing is Chebyshev-accelerated
// Jacobi; the coarsest grid is solved with an explicit FP64 inverse.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "modal.cuh"

namespace topo {

struct GmgLevel {
  Dims d{};
  long long nvec = 0;
  float* E = nullptr;     // owned for levels >= 1 (level 0 borrows the mesh's)
  float* dinv = nullptr;  // owned for levels >= 1
  float* b = nullptr;     // owned for levels >= 1
  float* x = nullptr;     // owned for levels >= 1
  float* r = nullptr;     // owned
  float* dv[2] = {nullptr, nullptr};  // owned, Chebyshev direction double buffer
};

struct Gmg {
  std::vector<GmgLevel> lv;
  int degree = 3;            // Chebyshev degree per pre/post smoothing
  double lam_max = 0.0;      // bound on lambda_max(D^-1 A) (from k0)
  double lam_ratio = 15.0;   // smoothing interval [lam_max / lam_ratio, lam_max]
  // coarsest level: explicit inverse
  int nc = 0;                // dense size (3 * nodes of the coarsest grid)
  double* Ainv = nullptr;    // nc * nc
  double* side = nullptr;    // 4 * nc (Gauss-Jordan pivot row/column, ping-pong)
  double* bd = nullptr;      // nc
  cudaGraphExec_t gj_exec = nullptr;  // captured Gauss-Jordan pivot chain
  int gj_nb = 0;             // ... for this many designs
  long long gj_S = 0;        // ... at this design stride
  long long bytes = 0;
  int tail_l0 = -1;          // levels tail_l0 .. coarsest run as one kernel per design (-1: none)
  bool ready = false;        // set up for the current densities
  bool arena = false;        // buffers come from a mesh group's arena (not freed here)
  // throughput form (many meshes sharing the GPU): the coarse end runs as one
  // kernel per V-cycle and the coarsest inverse is formed by one kernel
  bool throughput = false;
};

// Optional allocator for the hierarchy's buffers (a mesh group's arena).
struct GmgAlloc {
  void* ctx;
  cudaError_t (*fn)(void* ctx, void** p, size_t bytes);
};

// The level grids a fine grid coarsens to, and the bytes a hierarchy holds.
// max_dof: the coarsest grid's size limit (DOF, fixed ones included)
std::vector<Dims> gmg_plan(const Dims& fine, int max_levels, int max_dof = 400);
long long gmg_footprint(const Dims& fine, int max_levels);
// Choose levels for a fine grid and allocate them (fine-level E/dinv/b/x are
// bound later, per call).  max_levels <= 0: automatic.
// throughput: the throughput form (see Gmg::throughput); its coarsest grid
// is kept within the single-kernel inverse's size (222 DOF)
cudaError_t gmg_create(Gmg& g, const Dims& fine, int max_levels, int degree, double lam_max,
                       cudaStream_t s, const GmgAlloc* alloc = nullptr, bool throughput = false);
// Per-density setup: coarse moduli, Jacobi diagonals, coarsest inverse.
// bt: the designs of a mesh group (pointers are design 0's; each design's
// hierarchy sits at the group's design stride from design 0's).
cudaError_t gmg_setup(Gmg& g, const float* E0, const float* dinv0, const K0<float>& k0f,
                      const K0<double>& k0d, cudaStream_t s, long long* launches,
                      const Bat& bt = Bat{});
// Timing of the finest level's Chebyshev steps (the k_modal_*<EpiChebStep>
// launches of level 0): a V-cycle given one records an event pair around each
// of them (ev[2 q], ev[2 q + 1], q < cap, external events: also inside stream
// capture) and, per recorded launch, whether it stores x (kXStore) or adds to
// it (the two move different bytes).
struct GmgProf {
  cudaEvent_t* ev = nullptr;
  int cap = 0;
  int n = 0;                  // launches recorded
  unsigned char store[16] = {};
};

// x = V(b) on level 0 (x, b: fine-level vectors); every kernel returns at once
// when *done is set.
// mcf != nullptr: smoother passes use the modal operator kernel
// zdot (optional): the reduction b . x of the result (the CG's r . z), fused
// into the finest level's last smoothing step
// d0_ready: the finest level's first Chebyshev direction D^-1 b / theta is
// already in its buffer (gmg_first_direction)
cudaError_t gmg_vcycle(Gmg& g, const float* b, float* x, const K0<float>& k0f,
                       const ModalCoef<float>* mcf, const int* done, int* errflag,
                       cudaStream_t s, long long* launches, const Bat& bt = Bat{},
                       const Red* zdot = nullptr, bool d0_ready = false,
                       GmgProf* prof = nullptr);
// Where a V-cycle's first finest-level Chebyshev direction goes (*d0) and its
// scale 1/theta, for a caller that forms it (D^-1 of the finest level is the
// one the hierarchy was set up with); 0 when the finest level is not smoothed.
float gmg_first_direction(const Gmg& g, float** d0);
void gmg_free(Gmg& g);
// lambda_max of diag(k0)^-1 k0 (bounds lambda_max(D^-1 A) on every level)
double k0_jacobi_bound(const double* k0);

}  // namespace topo
