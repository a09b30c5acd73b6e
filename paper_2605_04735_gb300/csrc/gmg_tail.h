// The coarse end of the multigrid V-cycle in one kernel per design
// (gmg_tail.cu): levels l0 .. coarsest in shared memory.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace topo {

constexpr int kTailMaxLevels = 6;        // smoothed levels the kernel takes
constexpr int kTailMaxDeg = 8;           // Chebyshev degree
constexpr size_t kTailMaxSmem = 200 * 1024;
constexpr int kTailMaxNodes = 1024;      // nodes of the tail's finest level

struct TailPlan {
  int nt;                                // smoothed levels: l0 .. l0 + nt - 1; then the coarsest
  int degree;
  float inv_theta;
  float c1[kTailMaxDeg], c2[kTailMaxDeg];
  float kdiag;                           // every diagonal entry of k0 (D^-1 from the moduli)
  int nc;                                // coarsest dense size
  int off[kTailMaxLevels + 2];           // shared-memory float offsets: levels, then FP64 b
  Dims d[kTailMaxLevels + 1];
  const float* E[kTailMaxLevels];        // moduli of the smoothed levels (design 0)
  const float* b;                        // right-hand side of level l0 (design 0)
  float* x;                              // result at level l0 (design 0)
  const double* Ainv;                    // the coarsest inverse, nc x nc (design 0)
};

// Bytes of shared memory the tail from level l0 needs (offsets: the plan's
// off[] filled in when non-null).
size_t tail_plan_smem(const std::vector<Dims>& lv, int l0, int* offsets);
// First level the tail can start at (>= 1, at least one smoothed level, at
// most kTailMaxNodes nodes, the plan within kTailMaxSmem), -1 if none.
int tail_first_level(const std::vector<Dims>& lv, int degree);
cudaError_t launch_vcycle_tail(const TailPlan& p, size_t smem, const K0<float>& k0,
                               const int* done, cudaStream_t s, const Bat& bt = Bat{});

}  // namespace topo
