// Device kernels of the level-set stage around the ersatz state solve
// (Sec. 2.2.5-2.2.8): the relaxed shape-derivative right-hand sides
// (Eqs. (14), (15)), the Hilbertian extension operator A_H of Eqs. (19),
// (20) for Jacobi-PCG, and the first-order Godunov upwind steps of the
// Hamilton-Jacobi evolution (Eqs. (21), (22)) and of reinitialisation
// (Eqs. (23), (24)).  All level-set quantities are FP64 nodal arrays in dense
// node order n = i + (nx+1)(j + (ny+1)k); the displacement is the library's
// ghosted SoA FP64 vector.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace topo {

namespace {

constexpr int kLsThreads = 256;

__device__ __forceinline__ double hprime(double p, double eta) {
  return (fabs(p) <= eta) ? (1.0 + cos(M_PI * p / eta)) / (2.0 * eta) : 0.0;
}

// Per element: the 8 corner shares of bJ and bV by 2x2x2 Gauss quadrature
// (corner b = dx + 2 dy + 4 dz); elements whose 8 corner values all lie on
// one side outside the band contribute 0 (phi at a Gauss point is a convex
// combination of the corners).  out[(q * 8 + b) * ne + e], q = 0 (J), 1 (V).
__global__ void __launch_bounds__(kLsThreads)
    k_shape_rhs_elem(const double* __restrict__ u, const double* __restrict__ phi,
                     double* __restrict__ out, const Dims d, double eta, double lam, double mu,
                     double h) {
  const long long ne = (long long)d.nx * d.ny * d.nz;
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(e, d.nx, d.ny, i, j, k);
    const long long n0 = i + sx * j + sxy * k;
    double pc[8];
    double lo = 1e300, hi = -1e300;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      pc[b] = __ldg(phi + n0 + (b & 1) + sx * ((b >> 1) & 1) + sxy * (b >> 2));
      lo = fmin(lo, pc[b]);
      hi = fmax(hi, pc[b]);
    }
    double cJ[8], cV[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) cJ[b] = cV[b] = 0.0;
    if (hi >= -eta && lo <= eta) {
      double ue[3][8];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 8; ++b)
          ue[c][b] = __ldg(u + c * d.comp + d.node(i + (b & 1), j + ((b >> 1) & 1), k + (b >> 2)));
      const double gp = 0.5773502691896257645;  // 1 / sqrt(3)
      const double jac = 0.5 * h, detJ = jac * jac * jac;
#pragma unroll 1
      for (int q = 0; q < 8; ++q) {
        const double xq[3] = {(q & 1) ? gp : -gp, (q & 2) ? gp : -gp, (q & 4) ? gp : -gp};
        double N[8], dN[8][3];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const double s0 = (b & 1) ? 1.0 : -1.0, s1 = (b & 2) ? 1.0 : -1.0,
                       s2 = (b & 4) ? 1.0 : -1.0;
          const double a0 = 1.0 + s0 * xq[0], a1 = 1.0 + s1 * xq[1], a2 = 1.0 + s2 * xq[2];
          N[b] = a0 * a1 * a2 * 0.125;
          dN[b][0] = s0 * a1 * a2 * 0.125 / jac;
          dN[b][1] = a0 * s1 * a2 * 0.125 / jac;
          dN[b][2] = a0 * a1 * s2 * 0.125 / jac;
        }
        double pq = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        double exx = 0.0, eyy = 0.0, ezz = 0.0, gyz = 0.0, gxz = 0.0, gxy = 0.0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          pq = fma(N[b], pc[b], pq);
          g0 = fma(dN[b][0], pc[b], g0);
          g1 = fma(dN[b][1], pc[b], g1);
          g2 = fma(dN[b][2], pc[b], g2);
          exx = fma(dN[b][0], ue[0][b], exx);
          eyy = fma(dN[b][1], ue[1][b], eyy);
          ezz = fma(dN[b][2], ue[2][b], ezz);
          gyz = fma(dN[b][2], ue[1][b], fma(dN[b][1], ue[2][b], gyz));
          gxz = fma(dN[b][2], ue[0][b], fma(dN[b][0], ue[2][b], gxz));
          gxy = fma(dN[b][1], ue[0][b], fma(dN[b][0], ue[1][b], gxy));
        }
        const double w = hprime(pq, eta) * sqrt(g0 * g0 + g1 * g1 + g2 * g2) * detJ;
        if (w == 0.0) continue;
        const double tr = exx + eyy + ezz;
        const double en = lam * tr * tr + 2.0 * mu * (exx * exx + eyy * eyy + ezz * ezz) +
                          mu * (gyz * gyz + gxz * gxz + gxy * gxy);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          cV[b] = fma(w, N[b], cV[b]);
          cJ[b] = fma(w * en, N[b], cJ[b]);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      out[(long long)b * ne + e] = cJ[b];
      out[(long long)(8 + b) * ne + e] = cV[b];
    }
  }
}

// Per node: sum the shares of its (up to 8) elements -> bJ[n], bV[n]
__global__ void __launch_bounds__(kLsThreads)
    k_shape_rhs_node(const double* __restrict__ part, double* __restrict__ bJ,
                     double* __restrict__ bV, const Dims d) {
  const long long ne = (long long)d.nx * d.ny * d.nz;
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(n, d.nx + 1, d.ny + 1, i, j, k);
    double sJ = 0.0, sV = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {  // element (i - 1 + ax, j - 1 + ay, k - 1 + az)
      const int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
      const int ei = i - 1 + ax, ej = j - 1 + ay, ek = k - 1 + az;
      if (ei < 0 || ej < 0 || ek < 0 || ei >= d.nx || ej >= d.ny || ek >= d.nz) continue;
      const long long e = ei + (long long)d.nx * (ej + (long long)d.ny * ek);
      const int b = (1 - ax) + 2 * (1 - ay) + 4 * (1 - az);  // this node's corner of e
      sJ += part[(long long)b * ne + e];
      sV += part[(long long)(8 + b) * ne + e];
    }
    bJ[n] = sJ;
    bV[n] = sV;
  }
}

// 1-D rows of the assembled Q1 stiffness (k) and mass (m) at index i of 0..n
__device__ __forceinline__ void q1_rows(int i, int n, double h, double (&k)[3], double (&m)[3]) {
  const double l = (i > 0) ? 1.0 : 0.0, r = (i < n) ? 1.0 : 0.0;
  k[0] = -l / h;
  k[1] = (l + r) / h;
  k[2] = -r / h;
  m[0] = l * h / 6.0;
  m[1] = (l + r) * h / 3.0;
  m[2] = r * h / 6.0;
}

// y = A_H x (Eq. (20)) on free nodes, y = x on Dirichlet nodes (x = 0 there);
// the global Q1 operator is the tensor product of the assembled 1-D rows:
// A = ell^2 (Kx My Mz + Mx Ky Mz + Mx My Kz) + Mx My Mz, applied by sum
// factorisation over the 27-node window.  DOT: reduces x . y -> red.
template <bool DOT>
__global__ void __launch_bounds__(kLsThreads)
    k_hilb_apply(const double* __restrict__ x, double* __restrict__ y,
                 const uint8_t* __restrict__ dir, const Dims d, double ell2, double h,
                 const Red red, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  double part = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % sx);
    const int j = (int)((n / sx) % (d.ny + 1));
    const int k = (int)(n / sxy);
    double out;
    if (dir[n]) {
      out = x[n];
    } else {
      double kx[3], mx[3], ky[3], my[3], kz[3], mz[3];
      q1_rows(i, d.nx, h, kx, mx);
      q1_rows(j, d.ny, h, ky, my);
      q1_rows(k, d.nz, h, kz, mz);
      double t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (mz[c] == 0.0) continue;  // the neighbour plane is outside
        double a_kxmy = 0.0, a_mxky = 0.0, a_mxmy = 0.0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (my[b] == 0.0) continue;
          double sk = 0.0, sm = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (mx[a] == 0.0) continue;
            const double v = x[n + (a - 1) + sx * (b - 1) + sxy * (c - 1)];
            sk = fma(kx[a], v, sk);
            sm = fma(mx[a], v, sm);
          }
          a_kxmy = fma(my[b], sk, a_kxmy);
          a_mxky = fma(ky[b], sm, a_mxky);
          a_mxmy = fma(my[b], sm, a_mxmy);
        }
        t1 = fma(mz[c], a_kxmy, t1);
        t2 = fma(mz[c], a_mxky, t2);
        t3 = fma(kz[c], a_mxmy, t3);
        t4 = fma(mz[c], a_mxmy, t4);
      }
      out = fma(ell2, t1 + t2 + t3, t4);
    }
    y[n] = out;
    if (DOT) part = fma(x[n], out, part);
  }
  if (DOT) {
    double v[1] = {part};
    reduce_finalize<1>(v, red);
  }
}

// Jacobi inverse diagonal of A_H (1 on Dirichlet nodes and on the padding)
__global__ void k_hilb_dinv(double* __restrict__ dinv, const uint8_t* __restrict__ dir,
                            const Dims d, double ell2, double h, long long npad) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < npad;
       n += (long long)gridDim.x * blockDim.x) {
    if (n >= nn || dir[n]) {
      dinv[n] = 1.0;
      continue;
    }
    const int i = (int)(n % sx), j = (int)((n / sx) % (d.ny + 1)), k = (int)(n / sxy);
    double kx[3], mx[3], ky[3], my[3], kz[3], mz[3];
    q1_rows(i, d.nx, h, kx, mx);
    q1_rows(j, d.ny, h, ky, my);
    q1_rows(k, d.nz, h, kz, mz);
    const double a = ell2 * (kx[1] * my[1] * mz[1] + mx[1] * ky[1] * mz[1] +
                             mx[1] * my[1] * kz[1]) + mx[1] * my[1] * mz[1];
    dinv[n] = 1.0 / a;
  }
}

// Dirichlet mask of the extension problem: the loaded nodes (Gamma_N)
__global__ void k_hilb_mask(const double* __restrict__ f, uint8_t* __restrict__ dir,
                            const Dims d) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % sx), j = (int)((n / sx) % (d.ny + 1)), k = (int)(n / sxy);
    const long long o = d.node(i, j, k);
    dir[n] = (f[o] != 0.0 || f[d.comp + o] != 0.0 || f[2 * d.comp + o] != 0.0) ? 1 : 0;
  }
}

// b := 0 on Dirichlet nodes and on the padding
__global__ void k_hilb_rhs(const double* __restrict__ src, double* __restrict__ b,
                           const uint8_t* __restrict__ dir, long long nn, long long npad) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < npad;
       n += (long long)gridDim.x * blockDim.x)
    b[n] = (n < nn && !dir[n]) ? src[n] : 0.0;
}

// one-sided differences of phi at node (i, j, k) along one axis: (backward,
// forward), 0 where the neighbour is outside the grid
__device__ __forceinline__ void diffs(const double* __restrict__ phi, long long n, int i, int ni,
                                      long long stride, double h, double& dm, double& dp) {
  const double c = phi[n];
  dm = (i > 0) ? (c - phi[n - stride]) / h : 0.0;
  dp = (i < ni) ? (phi[n + stride] - c) / h : 0.0;
}

// Godunov upwind gradient norms for a positive / negative speed
__device__ __forceinline__ void upwind(const double* __restrict__ phi, long long n, int i, int j,
                                       int k, const Dims& d, double h, double& gp, double& gm,
                                       double& gc2) {
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  double p2 = 0.0, m2 = 0.0, c2 = 0.0;
  double dm, dp;
  const int idx[3] = {i, j, k};
  const int lim[3] = {d.nx, d.ny, d.nz};
  const long long st[3] = {1, sx, sxy};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    diffs(phi, n, idx[a], lim[a], st[a], h, dm, dp);
    p2 += fmax(dm, 0.0) * fmax(dm, 0.0) + fmin(dp, 0.0) * fmin(dp, 0.0);
    m2 += fmin(dm, 0.0) * fmin(dm, 0.0) + fmax(dp, 0.0) * fmax(dp, 0.0);
    // central difference inside, one-sided on the boundary faces
    const double cd = (idx[a] > 0 && idx[a] < lim[a]) ? 0.5 * (dm + dp) : (idx[a] > 0 ? dm : dp);
    c2 += cd * cd;
  }
  gp = sqrt(p2);
  gm = sqrt(m2);
  gc2 = c2;
}

// Eq. (21): phi_out = phi - dt (max(v,0) grad+ + min(v,0) grad-)
__global__ void __launch_bounds__(kLsThreads)
    k_hj_step(const double* __restrict__ phi, double* __restrict__ out,
              const double* __restrict__ v, const Dims d, const double* __restrict__ dt_dev,
              double h) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  const double dt = *dt_dev;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % sx), j = (int)((n / sx) % (d.ny + 1)), k = (int)(n / sxy);
    double gp, gm, gc2;
    upwind(phi, n, i, j, k, d, h, gp, gm, gc2);
    const double s = v[n];
    out[n] = phi[n] - dt * (fmax(s, 0.0) * gp + fmin(s, 0.0) * gm);
  }
}

// Eqs. (23), (24): phi_out = phi - dt (S+ grad+ + S- grad- - S), S from the
// current phi with the central-difference gradient; max |phi_out - phi| is
// folded into *maxchange (bit pattern of a non-negative double)
__global__ void __launch_bounds__(kLsThreads)
    k_reinit_step(const double* __restrict__ phi, double* __restrict__ out, const Dims d,
                  double dt, double h, unsigned long long* __restrict__ maxchange) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
  double mx = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % sx), j = (int)((n / sx) % (d.ny + 1)), k = (int)(n / sxy);
    double gp, gm, gc2;
    upwind(phi, n, i, j, k, d, h, gp, gm, gc2);
    const double p = phi[n];
    const double den = sqrt(p * p + h * h * gc2);
    const double S = (den > 0.0) ? p / den : 0.0;
    const double o = p - dt * (fmax(S, 0.0) * gp + fmin(S, 0.0) * gm - S);
    out[n] = o;
    mx = fmax(mx, fabs(o - p));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx > 0.0)
    atomicMax(maxchange, (unsigned long long)__double_as_longlong(mx));
}

// max |v| over the nodes -> *out (bit pattern of a non-negative double)
__global__ void __launch_bounds__(kLsThreads)
    k_max_abs(const double* __restrict__ v, long long n, unsigned long long* __restrict__ out) {
  double mx = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(v[q]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx > 0.0)
    atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// dt = gamma h / max |v| (Eq. (22)); 0 when v vanishes
__global__ void k_cfl_dt(const unsigned long long* __restrict__ vmax, double gamma, double h,
                         double* __restrict__ dt) {
  const double m = __longlong_as_double((long long)*vmax);
  *dt = (m > 0.0) ? gamma * h / m : 0.0;
}

int ls_blocks(long long n) {
  long long b = (n + kLsThreads - 1) / kLsThreads;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_shape_rhs(const double* u, const double* phi, double* part, double* bJ,
                             double* bV, const Dims& d, double eta, double E0, double nu,
                             double h, cudaStream_t s) {
  const double lam = E0 * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E0 / (2.0 * (1.0 + nu));
  const long long ne = (long long)d.nx * d.ny * d.nz;
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_shape_rhs_elem<<<ls_blocks(ne), kLsThreads, 0, s>>>(u, phi, part, d, eta, lam, mu, h);
  k_shape_rhs_node<<<ls_blocks(nn), kLsThreads, 0, s>>>(part, bJ, bV, d);
  return cudaGetLastError();
}

cudaError_t launch_hilb_setup(const double* f, uint8_t* dir, double* dinv, const Dims& d,
                              double ell2, double h, long long npad, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_hilb_mask<<<ls_blocks(nn), kLsThreads, 0, s>>>(f, dir, d);
  k_hilb_dinv<<<ls_blocks(npad), kLsThreads, 0, s>>>(dinv, dir, d, ell2, h, npad);
  return cudaGetLastError();
}

cudaError_t launch_hilb_rhs(const double* src, double* b, const uint8_t* dir, const Dims& d,
                            long long npad, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_hilb_rhs<<<ls_blocks(npad), kLsThreads, 0, s>>>(src, b, dir, nn, npad);
  return cudaGetLastError();
}

cudaError_t launch_hilb_apply(const double* x, double* y, const uint8_t* dir, const Dims& d,
                              double ell2, double h, const Red& red, bool dot, const int* done,
                              cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  if (dot)
    k_hilb_apply<true><<<ls_blocks(nn), kLsThreads, 0, s>>>(x, y, dir, d, ell2, h, red, done);
  else
    k_hilb_apply<false><<<ls_blocks(nn), kLsThreads, 0, s>>>(x, y, dir, d, ell2, h, red, done);
  return cudaGetLastError();
}

cudaError_t launch_hj_steps(double* phi, double* tmp, const double* v, const Dims& d,
                            double gamma, double h, int steps, unsigned long long* scratch,
                            double* dt_dev, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_max_abs<<<ls_blocks(nn), kLsThreads, 0, s>>>(v, nn, scratch);
  k_cfl_dt<<<1, 1, 0, s>>>(scratch, gamma, h, dt_dev);
  for (int q = 0; q < steps; ++q) {
    k_hj_step<<<ls_blocks(nn), kLsThreads, 0, s>>>(phi, tmp, v, d, dt_dev, h);
    e = cudaMemcpyAsync(phi, tmp, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_reinit_step(const double* phi, double* out, const Dims& d, double dt, double h,
                               unsigned long long* maxchange, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_reinit_step<<<ls_blocks(nn), kLsThreads, 0, s>>>(phi, out, d, dt, h, maxchange);
  return cudaGetLastError();
}

}  // namespace topo
