// Per-element and per-node data kernels: SIMP interpolation (Eq. (1)),
// the load vector, layout conversion at the ABI boundary, and the adjoint
// sensitivity of the compliance (Eq. (3)) with the element-energy form of
// the compliance (Eq. (2)) fused into the same pass.
#include <cuda_runtime.h>

#include <algorithm>

#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "modal.cuh"

namespace topo {

namespace {

// Eq. (1): E_e = Emin + rho_e^p (E0 - Emin), evaluated in FP64 and stored
// both in FP64 and rounded to FP32; each scaled by the element size h
// (k0 of an element of edge h is h times the unit-cube k0 in 3-D).
// blockIdx.y: the design slot; its input at id * src_stride floats from
// rho, its buffers at id * S bytes; rho_keep (optional) keeps the input
__global__ void k_simp(const float* __restrict__ rho, float* __restrict__ rho_g,
                       float* __restrict__ E32, double* __restrict__ E64,
                       float* __restrict__ rho_keep, const Dims d, double E0, double Emin,
                       double penal, double hscale, int* __restrict__ bad, long long src_stride,
                       const DSel S) {
  const long long off = S.off(blockIdx.y);
  rho += S.id(blockIdx.y) * src_stride;
  rho_g = bshift(rho_g, off);
  E32 = bshift(E32, off);
  E64 = bshift(E64, off);
  rho_keep = bshift(rho_keep, off);
  bad = bshift(bad, off);
  const long long n = (long long)d.nx * d.ny * d.nz;
  int nbad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(e, d.nx, d.ny, i, j, k);
    float r = rho[e];
    if (rho_keep) rho_keep[e] = r;
    if (!(r >= 0.0f && r <= 1.0f)) {  // catches NaN too
      ++nbad;
      r = 0.0f;
    }
    const double rp = (penal == 3.0) ? (double)r * r * r : pow((double)r, penal);
    const double Ee = (Emin + rp * (E0 - Emin)) * hscale;
    const long long o = d.elem(i, j, k);
    rho_g[o] = r;
    E64[o] = Ee;
    E32[o] = (float)Ee;
  }
  if (nbad) atomicAdd(bad, nbad);
}

// Is face quad (a, b) in the load region?  Disc (paper Sec. 4.2): quads of
// the x = L face, (a, b) = (j, k), centroid within 0.1 ny of the face centre.
// Half-disc (Sec. 4.3): quads of the top face, (a, b) = (i, j), centroid
// within 0.1 ny of (0, ny/2).
__host__ __device__ inline bool in_load_region(int load, int a, int b, const Dims& d) {
  const double rad = 0.1 * d.ny;
  if (load == 3) {
    const double y = a + 0.5 - d.ny / 2.0, z = b + 0.5 - d.nz / 2.0;
    return a >= 0 && a < d.ny && b >= 0 && b < d.nz && y * y + z * z <= rad * rad;
  }
  const double x = a + 0.5, y = b + 0.5 - d.ny / 2.0;
  return a >= 0 && a < d.nx && b >= 0 && b < d.ny && x * x + y * y <= rad * rad;
}

// Consistent nodal forces of the load cases (component-major ghosted layout).
__global__ void k_build_load(double* __restrict__ f, const Dims d, int load, double mag, double h,
                             int nquads) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (load == 0 || load == 1) {
    // total `mag` in -z along a line of ny segments: ends get half a share
    if (t > d.ny) return;
    const int i = (load == 0) ? d.nx : 0;
    const int k = (load == 0) ? 0 : d.nz;
    const double share = mag / d.ny;
    const double v = (t == 0 || t == d.ny) ? 0.5 * share : share;
    f[2 * d.comp + d.node(i, t, k)] = -v;
  } else if (load == 2) {
    // uniform +x traction `mag` per unit area on x = L: each face quad of
    // area h^2 sends a quarter of its force to each of its corners
    const int nyz = (d.ny + 1) * (d.nz + 1);
    if (t >= nyz) return;
    const int j = t % (d.ny + 1);
    const int k = t / (d.ny + 1);
    const int cj = (j == 0 || j == d.ny) ? 1 : 2;
    const int ck = (k == 0 || k == d.nz) ? 1 : 2;
    f[d.node(d.nx, j, k)] = mag * h * h * 0.25 * cj * ck;
  } else {
    // total `mag` in -z, uniform over the region's face quads; a face node
    // collects a quarter share from each adjacent quad in the region
    const int w = (load == 3) ? d.ny + 1 : d.nx + 1;
    const int hgt = (load == 3) ? d.nz + 1 : d.ny + 1;
    if (t >= w * hgt) return;
    const int a = t % w, b = t / w;
    int cnt = 0;
    for (int da = -1; da <= 0; ++da)
      for (int db = -1; db <= 0; ++db) cnt += in_load_region(load, a + da, b + db, d) ? 1 : 0;
    if (!cnt) return;
    const long long o = (load == 3) ? d.node(d.nx, a, b) : d.node(a, b, d.nz);
    f[2 * d.comp + o] = -mag * 0.25 * cnt / nquads;
  }
}

template <typename T>
__global__ void k_pack(const T* __restrict__ soa, double* __restrict__ aos, const Dims d) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(n, d.nx + 1, d.ny + 1, i, j, k);
    const long long o = d.node(i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) aos[3 * n + c] = (double)soa[c * d.comp + o];
  }
}

template <typename T>
__global__ void k_unpack(const double* __restrict__ aos, T* __restrict__ soa, const Dims d) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(n, d.nx + 1, d.ny + 1, i, j, k);
    const long long o = d.node(i, j, k);
#pragma unroll
    for (int c = 0; c < 3; ++c) soa[c * d.comp + o] = d.fixed(c, i, j, k) ? T(0) : (T)aos[3 * n + c];
  }
}

// Eq. (3): dc_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e, FP64 throughout.
// The quadratic form is evaluated in the modal basis of the brick (see
// modal.cuh): with u^ = H^T (u_e - u_0), u_e^T k0 u_e = u^T K~ u^ =
// sum_p,m D[p][m] u^_p[m]^2 + 2 sum_{p<q} couplings, about 105 FP64
// operations instead of 300 FMAs for the dense symmetric form.  Also reduces
// sum_e E_e u_e^T k0 u_e (Eq. (2), element form) -> aux[0].
__global__ void __launch_bounds__(256)
    k_sensitivity(const double* __restrict__ u, const float* __restrict__ rho_g,
                  const double* __restrict__ E64, double* __restrict__ dc, const Dims d,
                  const __grid_constant__ ModalCoef<double> kc, double penal, double dE,
                  const Red red0, long long dc_stride, const DSel S) {
  // blockIdx.y: the design slot; its output at id * dc_stride doubles from dc
  const long long off = S.off(blockIdx.y);
  u = bshift(u, off);
  rho_g = bshift(rho_g, off);
  E64 = bshift(E64, off);
  dc += S.id(blockIdx.y) * dc_stride;
  const Red red = red0.shifted(off);
  const long long n = (long long)d.nx * d.ny * d.nz;
  double part = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(e, d.nx, d.ny, i, j, k);
    double uh[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int b = 0; b < 8; ++b)
        uh[c][b] = __ldg(u + c * d.comp + d.node(i + (b & 1), j + ((b >> 1) & 1), k + (b >> 2)));
      const double u0 = uh[c][0];
      uh[c][0] = 0.0;
#pragma unroll
      for (int b = 1; b < 8; ++b) uh[c][b] -= u0;
      fwht8(uh[c]);
    }
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int m = 1; m < 8; ++m) {
        s = fma(kc.D[p][m] * uh[p][m], uh[p][m], s);
#pragma unroll
        for (int q = p + 1; q < 3; ++q) {
          if (((m >> p) & 1) == ((m >> q) & 1)) continue;
          s = fma(2.0 * kc.C[p][q][m] * uh[p][m], uh[q][m ^ (1 << p) ^ (1 << q)], s);
        }
      }
    const long long og = d.elem(i, j, k);
    const double r = (double)rho_g[og];
    const double rp1 = (penal == 3.0) ? r * r : pow(r, penal - 1.0);
    dc[e] = -penal * rp1 * dE * s;
    part = fma(E64[og], s, part);
  }
  double v[1] = {part};
  reduce_finalize<1>(v, red, blockIdx.x, gridDim.x);
}

// Eq. (3) from element energies the FP64 residual kernel stored
// (energy_e = (u_e - u_0)^T k0 (u_e - u_0) of the current u): dc_e =
// -p rho_e^(p-1) dE energy_e, and sum_e E_e energy_e -> red.  Batched as
// k_sensitivity.
__global__ void __launch_bounds__(256)
    k_sens_energy(const double* __restrict__ energy, const float* __restrict__ rho_g,
                  const double* __restrict__ E64, double* __restrict__ dc, const Dims d,
                  double penal, double dE, const Red red0, long long dc_stride, const DSel S) {
  const long long off = S.off(blockIdx.y);
  energy = bshift(energy, off);
  rho_g = bshift(rho_g, off);
  E64 = bshift(E64, off);
  dc += S.id(blockIdx.y) * dc_stride;
  const Red red = red0.shifted(off);
  const long long n = (long long)d.nx * d.ny * d.nz;
  double part = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(e, d.nx, d.ny, i, j, k);
    const long long og = d.elem(i, j, k);
    const double w = energy[og];
    const double r = (double)rho_g[og];
    const double rp1 = (penal == 3.0) ? r * r : pow(r, penal - 1.0);
    dc[e] = -penal * rp1 * dE * w;
    part = fma(E64[og], w, part);
  }
  double v[1] = {part};
  reduce_finalize<1>(v, red, blockIdx.x, gridDim.x);
}

// Ersatz material of the level-set stage (Sec. 2.2.2): phi at the element
// centroid (mean of the 8 corner values of the Q1 interpolant of the nodal
// level set, node n = i + (nx+1)(j + (ny+1)k)), H_eta of Eq. (8),
// I = (1 - H) + eps0 H of Eq. (7), E_e = E0 I(phi_e) (k_e(phi) = I k_e^0,
// Eq. (9)); rho_g receives 1 - H (the material fraction).  Reduces the
// volume sum_e (1 - H(phi_e)) of Eq. (10) (unit V_e) -> aux[0].
__global__ void __launch_bounds__(256)
    k_ersatz(const double* __restrict__ phi, float* __restrict__ rho_g, float* __restrict__ E32,
             double* __restrict__ E64, const Dims d, double E0, double eta, double eps0,
             double hscale, const Red red, int* __restrict__ bad) {
  const long long n = (long long)d.nx * d.ny * d.nz;
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  double part = 0.0;
  int nbad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(e, d.nx, d.ny, i, j, k);
    const long long n0 = i + sx * j + sxy * k;
    double pe = 0.0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
      pe += __ldg(phi + n0 + (b & 1) + sx * ((b >> 1) & 1) + sxy * (b >> 2));
    pe *= 0.125;
    if (!(pe == pe)) {  // NaN
      ++nbad;
      pe = 0.0;
    }
    double H;
    if (pe < -eta)
      H = 0.0;
    else if (pe > eta)
      H = 1.0;
    else
      H = 0.5 + pe / (2.0 * eta) + sin(M_PI * pe / eta) / (2.0 * M_PI);
    const double Ee = E0 * ((1.0 - H) + eps0 * H) * hscale;
    const long long o = d.elem(i, j, k);
    rho_g[o] = (float)(1.0 - H);
    E64[o] = Ee;
    E32[o] = (float)Ee;
    part += 1.0 - H;
  }
  if (nbad) atomicAdd(bad, nbad);
  double v[1] = {part};
  reduce_finalize<1>(v, red);
}

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_simp(const float* rho, float* rho_g, float* E32, double* E64, const Dims& d,
                        double E0, double Emin, double penal, double hscale, int* bad,
                        cudaStream_t s, float* rho_keep, long long src_stride, const Bat& bt) {
  const long long n = (long long)d.nx * d.ny * d.nz;
  const dim3 grid(std::max(1, grid_for(n, 256) / bt.nb), bt.nb);
  k_simp<<<grid, 256, 0, s>>>(rho, rho_g, E32, E64, rho_keep, d, E0, Emin, penal, hscale, bad,
                              src_stride, bt.sel());
  return cudaGetLastError();
}

cudaError_t launch_build_load(double* f, const Dims& d, int load, double magnitude, double h,
                              cudaStream_t s) {
  long long n = d.ny + 1;
  int nquads = 0;
  if (load == 2) n = (long long)(d.ny + 1) * (d.nz + 1);
  if (load == 3 || load == 4) {
    const int A = (load == 3) ? d.ny : d.nx, B = (load == 3) ? d.nz : d.ny;
    for (int b = 0; b < B; ++b)
      for (int a = 0; a < A; ++a) nquads += in_load_region(load, a, b, d) ? 1 : 0;
    if (!nquads) return cudaErrorInvalidValue;
    n = (long long)(A + 1) * (B + 1);
  }
  k_build_load<<<(int)((n + 255) / 256), 256, 0, s>>>(f, d, load, magnitude, h, nquads);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack(const T* soa, double* aos, const Dims& d, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_pack<T><<<grid_for(nn, 256), 256, 0, s>>>(soa, aos, d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack(const double* aos, T* soa, const Dims& d, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_unpack<T><<<grid_for(nn, 256), 256, 0, s>>>(aos, soa, d);
  return cudaGetLastError();
}

cudaError_t launch_sensitivity(const double* u, const float* rho_g, const double* E64, double* dc,
                               const Dims& d, const ModalCoef<double>& kc, double penal, double dE,
                               const Red& red, cudaStream_t s, long long dc_stride,
                               const Bat& bt) {
  const long long n = (long long)d.nx * d.ny * d.nz;
  const dim3 grid(std::min(std::max(1, grid_for(n, 256) / bt.nb), kMaxPartials), bt.nb);
  k_sensitivity<<<grid, 256, 0, s>>>(u, rho_g, E64, dc, d, kc, penal, dE, red, dc_stride,
                                     bt.sel());
  return cudaGetLastError();
}

cudaError_t launch_sens_energy(const double* energy, const float* rho_g, const double* E64,
                               double* dc, const Dims& d, double penal, double dE, const Red& red,
                               cudaStream_t s, long long dc_stride, const Bat& bt) {
  const long long n = (long long)d.nx * d.ny * d.nz;
  const dim3 grid(std::min(std::max(1, grid_for(n, 256) / bt.nb), kMaxPartials), bt.nb);
  k_sens_energy<<<grid, 256, 0, s>>>(energy, rho_g, E64, dc, d, penal, dE, red, dc_stride,
                                     bt.sel());
  return cudaGetLastError();
}

cudaError_t launch_ersatz(const double* phi, float* rho_g, float* E32, double* E64, const Dims& d,
                          double E0, double eta, double eps0, double hscale, const Red& red,
                          int* bad, cudaStream_t s) {
  const long long n = (long long)d.nx * d.ny * d.nz;
  k_ersatz<<<grid_for(n, 256), 256, 0, s>>>(phi, rho_g, E32, E64, d, E0, eta, eps0, hscale, red,
                                            bad);
  return cudaGetLastError();
}

template cudaError_t launch_pack<float>(const float*, double*, const Dims&, cudaStream_t);
template cudaError_t launch_pack<double>(const double*, double*, const Dims&, cudaStream_t);
template cudaError_t launch_unpack<float>(const double*, float*, const Dims&, cudaStream_t);
template cudaError_t launch_unpack<double>(const double*, double*, const Dims&, cudaStream_t);

}  // namespace topo
