/*
 * Plain FP64 CPU oracle pieces for grids too large to assemble (millions of
 * DOFs): the matrix-free product K(rho) u, the true residual f - K u, the
 * element energies u_e^T k0 u_e and a Jacobi-preconditioned conjugate
 * gradient solve of K_ff u_f = f_f.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/ and bench.py's CPU-baseline leg use
 * it (through oracle/fullsize.py); the CUDA library never links or calls it,
 * and it shares no code with it.
 *
 * What it computes (arXiv 2605.04735, Sec. 2.1.1, Eq. (2)):
 *   K(rho) = sum_e E_e k0 scattered by the element's 24 DOFs,
 * with E_e (Eq. (1)) and k0 (Sec. 2.1.2) given by the caller (the Python
 * oracle computes both), i.e. exactly the assembled matrix of oracle/fem.py
 * applied without forming it.  The element loop visits the elements in 8
 * classes by the parity of (i, j, k): two elements of one class share no
 * node, so a class may be summed by several threads at once without two of
 * them adding into one entry.  Within a class the order of the additions
 * into one node follows the class order, so results do not depend on the
 * thread count.
 *
 * Numbering as in oracle/fem.py: node n = i + (nx+1)(j + (ny+1)k), DOF 3n+c,
 * element e = i + nx(j + ny k), local nodes (0,0,0) (1,0,0) (1,1,0) (0,1,0)
 * (0,0,1) (1,0,1) (1,1,1) (0,1,1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int LX[8] = {0, 1, 1, 0, 0, 1, 1, 0};
static const int LY[8] = {0, 0, 1, 1, 0, 0, 1, 1};
static const int LZ[8] = {0, 0, 0, 0, 1, 1, 1, 1};

/* the 24 global DOFs of element (i, j, k) */
static void element_dofs(long nx, long ny, long i, long j, long k, long dof[24]) {
  for (int a = 0; a < 8; ++a) {
    const long n = (i + LX[a]) + (nx + 1) * ((j + LY[a]) + (ny + 1) * (k + LZ[a]));
    for (int c = 0; c < 3; ++c) dof[3 * a + c] = 3 * n + c;
  }
}

/* y = K(E) u over all DOFs (no boundary condition): y is overwritten. */
void oracle_apply(int nx, int ny, int nz, const double* E, const double* k0, const double* u,
                  double* y) {
  const long nn = (long)(nx + 1) * (ny + 1) * (nz + 1);
  memset(y, 0, sizeof(double) * 3 * nn);
  for (int cls = 0; cls < 8; ++cls) {
    const int pi = cls & 1, pj = (cls >> 1) & 1, pk = cls >> 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = pk; k < nz; k += 2)
      for (int j = pj; j < ny; j += 2)
        for (int i = pi; i < nx; i += 2) {
          long dof[24];
          double ue[24];
          element_dofs(nx, ny, i, j, k, dof);
          for (int a = 0; a < 24; ++a) ue[a] = u[dof[a]];
          const double Ee = E[i + (long)nx * (j + (long)ny * k)];
          for (int a = 0; a < 24; ++a) {
            double s = 0.0;
            for (int b = 0; b < 24; ++b) s += k0[24 * a + b] * ue[b];
            y[dof[a]] += Ee * s;
          }
        }
  }
}

/* r = f - K u on free DOFs, 0 on fixed ones; returns ||r||_2. */
double oracle_residual(int nx, int ny, int nz, const double* E, const double* k0,
                       const double* f, const uint8_t* fixed, const double* u, double* r) {
  const long nd = 3L * (nx + 1) * (ny + 1) * (nz + 1);
  oracle_apply(nx, ny, nz, E, k0, u, r);
  double rr = 0.0;
  for (long q = 0; q < nd; ++q) {
    r[q] = fixed[q] ? 0.0 : f[q] - r[q];
    rr += r[q] * r[q];
  }
  return sqrt(rr);
}

/* w_e = u_e^T k0 u_e for every element. */
void oracle_element_energies(int nx, int ny, int nz, const double* k0, const double* u,
                             double* w) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long dof[24];
        double ue[24];
        element_dofs(nx, ny, i, j, k, dof);
        for (int a = 0; a < 24; ++a) ue[a] = u[dof[a]];
        double s = 0.0;
        for (int a = 0; a < 24; ++a) {
          double t = 0.0;
          for (int b = 0; b < 24; ++b) t += k0[24 * a + b] * ue[b];
          s += ue[a] * t;
        }
        w[i + (long)nx * (j + (long)ny * k)] = s;
      }
}

static double dot(long n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long q = 0; q < n; ++q) s += a[q] * b[q];
  return s;
}

/*
 * Jacobi-preconditioned CG on K_ff x_f = f_f (fixed DOFs held at 0), from
 * x as given (x = 0 for a cold start).  D = diag K from the same element sum.
 * The recursive residual decides when to look at the true one; the solve
 * ends when the true relative residual ||f - K x|| / ||f|| is <= rtol, or
 * when `maxiter` iterations are spent, or when restarting from the true
 * residual no longer lowers it (the attainable floor of FP64).  Returns the
 * iterations used; *relres receives the final true relative residual.
 */
long oracle_cg(int nx, int ny, int nz, const double* E, const double* k0, const double* f,
               const uint8_t* fixed, double rtol, long maxiter, double* x, double* relres) {
  const long nd = 3L * (nx + 1) * (ny + 1) * (nz + 1);
  double* dinv = (double*)calloc(nd, sizeof(double));
  double* r = (double*)malloc(sizeof(double) * nd);
  double* z = (double*)malloc(sizeof(double) * nd);
  double* p = (double*)malloc(sizeof(double) * nd);
  double* q = (double*)malloc(sizeof(double) * nd);
  long it = 0;
  if (!dinv || !r || !z || !p || !q) {
    *relres = -1.0;
    goto out;
  }
  /* diagonal: sum over the elements of a DOF's node of E_e k0[l, l] */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long dof[24];
        element_dofs(nx, ny, i, j, k, dof);
        const double Ee = E[i + (long)nx * (j + (long)ny * k)];
        for (int a = 0; a < 24; ++a) dinv[dof[a]] += Ee * k0[24 * a + a];
      }
  for (long t = 0; t < nd; ++t) {
    dinv[t] = (fixed[t] || dinv[t] == 0.0) ? 0.0 : 1.0 / dinv[t];
    if (fixed[t]) x[t] = 0.0;
  }
  const double fn = sqrt(dot(nd, f, f));
  if (fn == 0.0) {
    memset(x, 0, sizeof(double) * nd);
    *relres = 0.0;
    goto out;
  }
  double best = INFINITY;
  for (;;) { /* one CG run from the true residual of the current x */
    const double tn = oracle_residual(nx, ny, nz, E, k0, f, fixed, x, r) / fn;
    *relres = tn;
    if (tn <= rtol || it >= maxiter || !(tn < 0.5 * best)) break;
    best = tn;
    for (long t = 0; t < nd; ++t) p[t] = z[t] = dinv[t] * r[t];
    double rz = dot(nd, r, z);
    while (it < maxiter) {
      oracle_apply(nx, ny, nz, E, k0, p, q);
      for (long t = 0; t < nd; ++t)
        if (fixed[t]) q[t] = 0.0;
      const double pq = dot(nd, p, q);
      if (!(pq > 0.0)) break;
      const double alpha = rz / pq;
      double rr = 0.0;
#pragma omp parallel for reduction(+ : rr) schedule(static)
      for (long t = 0; t < nd; ++t) {
        x[t] += alpha * p[t];
        r[t] -= alpha * q[t];
        z[t] = dinv[t] * r[t];
        rr += r[t] * r[t];
      }
      ++it;
      if (sqrt(rr) <= 0.5 * rtol * fn) break; /* look at the true residual */
      const double rz2 = dot(nd, r, z);
      const double beta = rz2 / rz;
      rz = rz2;
#pragma omp parallel for schedule(static)
      for (long t = 0; t < nd; ++t) p[t] = z[t] + beta * p[t];
    }
  }
out:
  free(dinv);
  free(r);
  free(z);
  free(p);
  free(q);
  return it;
}
