// The modal operator evaluated in double-word arithmetic (dword.cuh), for the
// FP64 refinement residual r = f - K u.
//
// Same work split and element arithmetic as the plain-load modal kernel
// (modal.cuh): one element column per thread, z march, x-y transform shared
// between layers, corner-0 shift.  The displacement arrives pre-split into
// two FP32 vectors (hi, lo: k_split_dw), the moduli and the K~ coefficients
// are split on the fly / on the host, and the node result is widened to
// FP64 for the epilogue (EpiResid<double>: r = f - K u and ||r||^2 in FP64;
// EpiApply<double>: y = K u).  Every FP64 operation of the element
// arithmetic becomes 7 to 11 FP32 operations, which GB300 issues 64 times as
// fast, so the residual costs a fraction of the FP64 kernel's time at
// 2^-48 instead of 2^-53 relative rounding per operation.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "dword.cuh"
#include "modal.cuh"

namespace topo {

inline ModalCoef<Dw> dw_coef(const ModalCoef<double>& k) {
  ModalCoef<Dw> c{};
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < 8; ++m) {
      c.D[a][m] = dw_from(k.D[a][m]);
      for (int b = 0; b < 3; ++b) c.C[a][b][m] = dw_from(k.C[a][b][m]);
    }
  c.kdiag = dw_from(k.kdiag);
  c.form = k.form;
  return c;
}

// Grid and z-chunks as k_modal_plain; Epi runs on FP64 values.
#ifndef TOPO_DW_MINB
#define TOPO_DW_MINB 2
#endif
template <class Epi>
__global__ void __launch_bounds__(kModalTX* kModalTY, TOPO_DW_MINB)
    k_modal_dw(const float* __restrict__ xh, const float* __restrict__ xl,
               const double* __restrict__ E, const Dims d,
               const __grid_constant__ ModalCoef<Dw> kc, const Epi epi0, const Red red0,
               const int zchunk, const int zc, const DSel S, const int* __restrict__ done) {
  pdl_start();
  const int slot = blockIdx.z / zc, chunk = blockIdx.z - slot * zc;
  const long long off = S.off(slot);
  done = bshift(done, off);
  if (done != nullptr && *done) return;
  xh = bshift(xh, off);
  xl = bshift(xl, off);
  E = bshift(E, off);
  const Epi epi = epi0.shifted(off);
  const Red red = red0.shifted(off);
  __shared__ Dw xch[2][kModalTY][kModalTX][3];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * kModalOwnX, y0 = blockIdx.y * kModalOwnY;
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const int kb = chunk * zchunk;
  const int ke = min(kb + zchunk, d.nz + 1);
  const bool own = tx > 0 && ty > 0 && ex <= d.nx && ey <= d.ny;
  const bool clean = !d.box_may_fix(x0, x0 + kModalOwnX - 1, y0, kb);
  auto node_val = [&](int i, int j, int k, int c) -> Dw {
    if (i > d.nx + 1 || j > d.ny + 1 || k > d.nz + 1) return Dw(0.0f);  // beyond the ghosts
    const long long o = c * d.comp + d.node(i, j, k);
    return Dw(__ldg(xh + o), __ldg(xl + o));
  };
  ModalColumn<Dw> col;
  {
    Dw raw[2][2][3];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) raw[dy][dx][c] = node_val(ex + dx, ey + dy, kb - 1, c);
    modal_seed<Dw>(col, raw);
  }
  double part = 0.0;
  for (int ez = kb - 1; ez < ke; ++ez) {
    Dw top[2][2][3];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx)
#pragma unroll
        for (int c = 0; c < 3; ++c) top[dy][dx][c] = node_val(ex + dx, ey + dy, ez + 1, c);
    const Dw Ee = (ex <= d.nx && ey <= d.ny && ez <= d.nz) ? dw_from(__ldg(E + d.elem(ex, ey, ez)))
                                                           : Dw(0.0f);
    Dw plane[3][4], ctr[3], res[3];
    modal_layer<Dw>(col, top, Ee, kc, plane, ctr);
    modal_exchange<Dw>(plane, xch[(ez - kb + 1) & 1], tx, ty, res);
    if (own && ez >= kb) {
      const double acc[3] = {dw_to(res[0]), dw_to(res[1]), dw_to(res[2])};
      const double cen[3] = {dw_to(ctr[0]), dw_to(ctr[1]), dw_to(ctr[2])};
      const long long o = d.node(ex, ey, ez);
      part += clean ? epi_one(epi, ex, ey, ez, o, acc, cen, FreeDims{d.comp})
                    : epi_one(epi, ex, ey, ez, o, acc, cen, d);
    }
  }
  if (Epi::kReduce) {
    double v[1] = {part};
    reduce_finalize<1>(v, red, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * chunk),
                       gridDim.x * gridDim.y * zc);
  }
}

template <class Epi>
cudaError_t launch_modal_dw(const float* xh, const float* xl, const double* E, const Dims& d,
                            const ModalCoef<double>& kc, const Epi& epi, const Red& red,
                            const int* done, cudaStream_t s, const Bat& bt) {
  const int z = modal_zchunk(d, bt.nb);
  const int zc = (d.nz + z) / z;
  dim3 block(kModalTX, kModalTY, 1);
  dim3 grid((d.nx + kModalOwnX) / kModalOwnX, (d.ny + kModalOwnY) / kModalOwnY, zc * bt.nb);
  return launch_pdl(k_modal_dw<Epi>, grid, block, 0, s, xh, xl, E, d, dw_coef(kc), epi, red, z,
                    zc, bt.sel(), done);
}

}  // namespace topo
