// SIMP -> level-set geometry transfer on the device (Sec. 3.2-3.4):
//   * nodal densities by a local linear least-squares fit per node
//     (Eqs. (25)-(27)), distance-weighted averaging where the normal
//     equations are singular (m < 4 or coplanar centroids), the element's own
//     density for m = 1;
//   * the iso-surface of a nodal field as a triangle soup: linear
//     interpolation on the edges of the 6 tetrahedra of the Kuhn split of
//     every hexahedron (marching tetrahedra; the split along the 0-7 diagonal
//     makes neighbouring cells agree on shared faces, so the surface is
//     closed).  Count per cell, exclusive scan, emit: triangles are stored
//     grouped by cell in cell order, which doubles as the spatial index;
//   * the signed distance at the nodes (Eqs. (28)-(30)): closest point on
//     each candidate triangle (plane projection if its barycentric
//     coordinates are non-negative, else the nearest of the three clamped edge
//     projections), candidates taken ring by ring of cells around the node
//     until no unvisited cell can hold a closer point; sign from the nodal
//     density.
// All geometry is FP64, unit-free: node (i, j, k) sits at (i, j, k) h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace topo {

namespace {

constexpr int kTrThreads = 256;

int tr_blocks(long long n) {
  long long b = (n + kTrThreads - 1) / kTrThreads;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

// -------------------------------------------------------------- nodal densities
__global__ void __launch_bounds__(kTrThreads)
    k_nodal_density(const float* __restrict__ rho, double* __restrict__ out, const Dims d,
                    double h) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(n, d.nx + 1, d.ny + 1, i, j, k);
    double xs[8][3], v[8];
    int m = 0;
    for (int c = 0; c < 8; ++c) {
      const int ei = i - 1 + (c & 1), ej = j - 1 + ((c >> 1) & 1), ek = k - 1 + (c >> 2);
      if (ei < 0 || ej < 0 || ek < 0 || ei >= d.nx || ej >= d.ny || ek >= d.nz) continue;
      xs[m][0] = (ei + 0.5) * h;
      xs[m][1] = (ej + 0.5) * h;
      xs[m][2] = (ek + 0.5) * h;
      v[m] = (double)rho[ei + (long long)d.nx * (ej + (long long)d.ny * ek)];
      ++m;
    }
    const double xn[3] = {i * h, j * h, k * h};
    double value = 0.0;
    bool done = false;
    if (m >= 4) {
      // normal equations X^T X a = X^T rho, X rows [1 x_e^T]
      double A[4][5];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 5; ++c) A[r][c] = 0.0;
      for (int q = 0; q < m; ++q) {
        const double row[4] = {1.0, xs[q][0], xs[q][1], xs[q][2]};
        for (int r = 0; r < 4; ++r) {
          for (int c = 0; c < 4; ++c) A[r][c] += row[r] * row[c];
          A[r][4] += row[r] * v[q];
        }
      }
      double scale = 0.0;
      for (int r = 0; r < 4; ++r) scale = fmax(scale, fabs(A[r][r]));
      bool singular = false;
      for (int p = 0; p < 4 && !singular; ++p) {  // Gauss-Jordan, partial pivoting
        int piv = p;
        for (int r = p + 1; r < 4; ++r)
          if (fabs(A[r][p]) > fabs(A[piv][p])) piv = r;
        if (fabs(A[piv][p]) <= 1e-12 * scale) {
          singular = true;
          break;
        }
        if (piv != p)
          for (int c = 0; c < 5; ++c) {
            const double t = A[p][c];
            A[p][c] = A[piv][c];
            A[piv][c] = t;
          }
        for (int r = 0; r < 4; ++r) {
          if (r == p) continue;
          const double f = A[r][p] / A[p][p];
          for (int c = p; c < 5; ++c) A[r][c] -= f * A[p][c];
        }
      }
      if (!singular) {
        const double a0 = A[0][4] / A[0][0], a1 = A[1][4] / A[1][1], a2 = A[2][4] / A[2][2],
                     a3 = A[3][4] / A[3][3];
        value = a0 + xn[0] * a1 + xn[1] * a2 + xn[2] * a3;
        done = true;
      }
    }
    if (!done) {
      if (m == 1) {
        value = v[0];
      } else {
        double ws = 0.0, acc = 0.0;
        for (int q = 0; q < m; ++q) {
          const double dx = xs[q][0] - xn[0], dy = xs[q][1] - xn[1], dz = xs[q][2] - xn[2];
          const double w = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
          acc += w * v[q];
          ws += w;
        }
        value = acc / ws;
      }
    }
    out[n] = value;
  }
}

// ------------------------------------------------------- marching tetrahedra
// Kuhn split: tetrahedron t = (0, a_t, a_t + b_t, 7) for the 6 orders of the
// axis steps (1, 2, 4), in the order (1,2,4) (1,4,2) (2,1,4) (2,4,1) (4,1,2) (4,2,1)
__constant__ int kKuhn[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7},
                                {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

struct Cell {
  double g[8];     // field - level, signed so that inside is g >= 0
  double x[8][3];  // corner coordinates
};

__device__ __forceinline__ void load_cell(const double* __restrict__ f, long long c, const Dims& d,
                                          double level, bool above, double h, Cell& cl) {
  const int i = (int)(c % d.nx), j = (int)((c / d.nx) % d.ny),
            k = (int)(c / ((long long)d.nx * d.ny));
  const long long sx = d.nx + 1, sxy = (long long)(d.nx + 1) * (d.ny + 1);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int di = b & 1, dj = (b >> 1) & 1, dk = b >> 2;
    const double v = f[(i + di) + sx * (j + dj) + sxy * (k + dk)];
    cl.g[b] = above ? (v - level) : (level - v);
    cl.x[b][0] = (i + di) * h;
    cl.x[b][1] = (j + dj) * h;
    cl.x[b][2] = (k + dk) * h;
  }
}

__device__ __forceinline__ int tet_count(const Cell& cl, int t) {
  int cnt = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) cnt += (cl.g[kKuhn[t][v]] >= 0.0) ? 1 : 0;
  return (cnt == 0 || cnt == 4) ? 0 : (cnt == 2 ? 2 : 1);
}

__device__ __forceinline__ void cut(const Cell& cl, int a, int b, double* out) {
  const double t = cl.g[a] / (cl.g[a] - cl.g[b]);
#pragma unroll
  for (int q = 0; q < 3; ++q) out[q] = cl.x[a][q] + t * (cl.x[b][q] - cl.x[a][q]);
}

// writes the triangles of tetrahedron t (9 doubles each) and returns their number
__device__ int tet_emit(const Cell& cl, int t, double* __restrict__ dst) {
  int vtx[4];
  bool ins[4];
  int cnt = 0;
  for (int v = 0; v < 4; ++v) {
    vtx[v] = kKuhn[t][v];
    ins[v] = cl.g[vtx[v]] >= 0.0;
    cnt += ins[v] ? 1 : 0;
  }
  if (cnt == 0 || cnt == 4) return 0;
  if (cnt == 1 || cnt == 3) {
    int lone = 0;
    for (int v = 0; v < 4; ++v)
      if (ins[v] == (cnt == 1)) lone = v;
    int o = 0;
    for (int v = 0; v < 4; ++v)
      if (v != lone) cut(cl, vtx[lone], vtx[v], dst + 3 * (o++));
    return 1;
  }
  int in2[2], out2[2], a = 0, b = 0;
  for (int v = 0; v < 4; ++v) {
    if (ins[v])
      in2[a++] = vtx[v];
    else
      out2[b++] = vtx[v];
  }
  double q0[3], q1[3], q2[3], q3[3];
  cut(cl, in2[0], out2[0], q0);
  cut(cl, in2[0], out2[1], q1);
  cut(cl, in2[1], out2[1], q2);
  cut(cl, in2[1], out2[0], q3);
  for (int q = 0; q < 3; ++q) {
    dst[q] = q0[q];
    dst[3 + q] = q1[q];
    dst[6 + q] = q2[q];
    dst[9 + q] = q0[q];
    dst[12 + q] = q2[q];
    dst[15 + q] = q3[q];
  }
  return 2;
}

__global__ void __launch_bounds__(kTrThreads)
    k_mt_count(const double* __restrict__ f, long long* __restrict__ counts, const Dims d,
               double level, bool above, double h) {
  const long long ne = (long long)d.nx * d.ny * d.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ne;
       c += (long long)gridDim.x * blockDim.x) {
    Cell cl;
    load_cell(f, c, d, level, above, h, cl);
    int n = 0;
    for (int t = 0; t < 6; ++t) n += tet_count(cl, t);
    counts[c] = n;
  }
}

__global__ void __launch_bounds__(kTrThreads)
    k_mt_emit(const double* __restrict__ f, const long long* __restrict__ offsets,
              double* __restrict__ tris, const Dims d, double level, bool above, double h) {
  const long long ne = (long long)d.nx * d.ny * d.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ne;
       c += (long long)gridDim.x * blockDim.x) {
    const long long o = offsets[c];
    if (offsets[c + 1] == o) continue;
    Cell cl;
    load_cell(f, c, d, level, above, h, cl);
    long long w = o;
    for (int t = 0; t < 6; ++t) w += tet_emit(cl, t, tris + 9 * w);
  }
}

// ----------------------------------------------------------------- scan
// exclusive scan of n int64 counts into out[0..n] (out[n] = total), in three
// passes: block sums, one-block scan of the sums, block-local scans
constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(kScanBlock)
    k_scan_sums(const long long* __restrict__ in, long long n, long long* __restrict__ sums) {
  __shared__ long long ws[kScanBlock / 32];
  const long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
  long long v = (i < n) ? in[i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int q = 0; q < kScanBlock / 32; ++q) s += ws[q];
    sums[blockIdx.x] = s;
  }
}

// exclusive scan of `nb` block sums by one block (chunks of kScanBlock)
__global__ void __launch_bounds__(kScanBlock)
    k_scan_block_offsets(long long* __restrict__ sums, long long nb) {
  __shared__ long long buf[kScanBlock];
  long long carry = 0;
  for (long long base = 0; base < nb; base += kScanBlock) {
    const long long i = base + threadIdx.x;
    buf[threadIdx.x] = (i < nb) ? sums[i] : 0;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {  // inclusive Hillis-Steele
      const long long t = (threadIdx.x >= off) ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    const long long incl = buf[threadIdx.x];
    const long long excl = incl - ((i < nb) ? sums[i] : 0);
    __syncthreads();
    if (i < nb) sums[i] = carry + excl;
    carry += buf[kScanBlock - 1];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanBlock)
    k_scan_local(const long long* __restrict__ in, long long n,
                 const long long* __restrict__ block_off, long long* __restrict__ out) {
  __shared__ long long buf[kScanBlock];
  const long long i = blockIdx.x * (long long)kScanBlock + threadIdx.x;
  const long long v = (i < n) ? in[i] : 0;
  buf[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const long long t = (threadIdx.x >= off) ? buf[threadIdx.x - off] : 0;
    __syncthreads();
    buf[threadIdx.x] += t;
    __syncthreads();
  }
  const long long excl = block_off[blockIdx.x] + buf[threadIdx.x] - v;
  if (i < n) out[i] = excl;
  if (i == n - 1) out[n] = excl + v;
}

// ------------------------------------------------------------ signed distance
__device__ __forceinline__ void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ double seg_dist(const double* p, const double* a, const double* b) {
  double ab[3], ap[3];
  sub3(b, a, ab);
  sub3(p, a, ap);
  const double L2 = dot3(ab, ab);
  double q[3];
  if (L2 == 0.0) {
    sub3(p, a, q);
    return sqrt(dot3(q, q));
  }
  const double t = fmin(fmax(dot3(ap, ab) / L2, 0.0), 1.0);
  for (int c = 0; c < 3; ++c) q[c] = p[c] - (a[c] + t * ab[c]);
  return sqrt(dot3(q, q));
}

// Eq. (28): distance from p to the triangle (a, b, c)
__device__ double tri_dist(const double* p, const double* a, const double* b, const double* c) {
  const double de = fmin(fmin(seg_dist(p, a, b), seg_dist(p, b, c)), seg_dist(p, c, a));
  double ba[3], ca[3], n[3];
  sub3(b, a, ba);
  sub3(c, a, ca);
  cross3(ba, ca, n);
  const double nn = dot3(n, n);
  if (nn == 0.0) return de;
  double pa[3];
  sub3(p, a, pa);
  const double s = dot3(pa, n) / nn;
  double q[3];
  for (int k = 0; k < 3; ++k) q[k] = p[k] - s * n[k];
  double cb[3], qb[3], ac[3], qc[3], w[3];
  sub3(c, b, cb);
  sub3(q, b, qb);
  cross3(cb, qb, w);
  const double l1 = dot3(w, n) / nn;
  sub3(a, c, ac);
  sub3(q, c, qc);
  cross3(ac, qc, w);
  const double l2 = dot3(w, n) / nn;
  const double l3 = 1.0 - l1 - l2;
  return (l1 >= 0.0 && l2 >= 0.0 && l3 >= 0.0) ? fabs(s) * sqrt(nn) : de;
}

__device__ __forceinline__ void scan_cell(const double* __restrict__ tris,
                                          const long long* __restrict__ off, long long cell,
                                          const double* p, double& best) {
  const long long t0 = off[cell], t1 = off[cell + 1];
  for (long long t = t0; t < t1; ++t) {
    const double* T = tris + 9 * t;
    best = fmin(best, tri_dist(p, T, T + 3, T + 6));
  }
}

// Eqs. (29), (30) per node: rings r = 0, 1, ... of cells around the node's 2x2x2
// cell block; after ring r every unvisited cell is at least (r + 1) h away
__global__ void __launch_bounds__(kTrThreads)
    k_sdf(const double* __restrict__ tris, const long long* __restrict__ off,
          const double* __restrict__ rho_n, double rho_t, double* __restrict__ phi, const Dims d,
          double h) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  const int rmax = max(d.nx, max(d.ny, d.nz)) + 1;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    unflatten3(n, d.nx + 1, d.ny + 1, i, j, k);
    const double p[3] = {i * h, j * h, k * h};
    double best = INFINITY;
    for (int r = 0; r <= rmax; ++r) {
      // ring r: cells with ci in [i-1-r, i+r] (likewise j, k) not in ring r-1
      const int i0 = i - 1 - r, i1 = i + r, j0 = j - 1 - r, j1 = j + r, k0 = k - 1 - r,
                k1 = k + r;
      for (int ck = max(k0, 0); ck <= min(k1, d.nz - 1); ++ck) {
        const bool kface = (ck == k0 || ck == k1);
        for (int cj = max(j0, 0); cj <= min(j1, d.ny - 1); ++cj) {
          const bool jface = (cj == j0 || cj == j1);
          if (kface || jface) {
            for (int ci = max(i0, 0); ci <= min(i1, d.nx - 1); ++ci)
              scan_cell(tris, off, ci + (long long)d.nx * (cj + (long long)d.ny * ck), p, best);
          } else {
            if (i0 >= 0) scan_cell(tris, off, i0 + (long long)d.nx * (cj + (long long)d.ny * ck), p, best);
            if (i1 <= d.nx - 1 && i1 != i0)
              scan_cell(tris, off, i1 + (long long)d.nx * (cj + (long long)d.ny * ck), p, best);
          }
        }
      }
      if (best <= (r + 1) * h) break;
    }
    phi[n] = (rho_n[n] >= rho_t) ? -best : best;
  }
}

}  // namespace

cudaError_t launch_nodal_density(const float* rho, double* out, const Dims& d, double h,
                                 cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_nodal_density<<<tr_blocks(nn), kTrThreads, 0, s>>>(rho, out, d, h);
  return cudaGetLastError();
}

long long scan_scratch_count(long long n) { return (n + kScanBlock - 1) / kScanBlock; }

cudaError_t launch_mt_count(const double* f, long long* counts, long long* offsets,
                            long long* scratch, const Dims& d, double level, bool above, double h,
                            cudaStream_t s) {
  const long long ne = (long long)d.nx * d.ny * d.nz;
  k_mt_count<<<tr_blocks(ne), kTrThreads, 0, s>>>(f, counts, d, level, above, h);
  const long long nb = scan_scratch_count(ne);
  k_scan_sums<<<(unsigned)nb, kScanBlock, 0, s>>>(counts, ne, scratch);
  k_scan_block_offsets<<<1, kScanBlock, 0, s>>>(scratch, nb);
  k_scan_local<<<(unsigned)nb, kScanBlock, 0, s>>>(counts, ne, scratch, offsets);
  return cudaGetLastError();
}

cudaError_t launch_mt_emit(const double* f, const long long* offsets, double* tris, const Dims& d,
                           double level, bool above, double h, cudaStream_t s) {
  const long long ne = (long long)d.nx * d.ny * d.nz;
  k_mt_emit<<<tr_blocks(ne), kTrThreads, 0, s>>>(f, offsets, tris, d, level, above, h);
  return cudaGetLastError();
}

cudaError_t launch_sdf(const double* tris, const long long* offsets, const double* rho_n,
                       double rho_t, double* phi, const Dims& d, double h, cudaStream_t s) {
  const long long nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_sdf<<<tr_blocks(nn), kTrThreads, 0, s>>>(tris, offsets, rho_n, rho_t, phi, d, h);
  return cudaGetLastError();
}

}  // namespace topo
