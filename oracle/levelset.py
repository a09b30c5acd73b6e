"""FP64 CPU oracle of the level-set stage's state quantities (Sec. 2.2).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline, never by the library.

Conventions: the level set phi is nodal, phi < 0 inside the material
(Sec. 2.2.1); node n = i + (nx+1)(j + (ny+1)k), unit element edge h = 1
unless a function takes h.  Element values are phi at the element
centroid; for the trilinear (Q1) interpolant that is the mean of the
eight corner values.

  heaviside(phi, eta)          regularised Heaviside H_eta, Eq. (8)
  heaviside_prime(phi, eta)    its derivative (zero outside |phi| <= eta)
  ersatz(phi, eta, eps0)       characteristic function I, Eq. (7)
  element_phi(...)             phi at the element centroids (Q1 interpolant)
  ersatz_modulus(...)          E_e = E0 I(phi_e): k_e(phi) = I(phi_e) k_e^0, Eq. (9)
  volume(...)                  V(phi) = sum_e V_e (1 - H_eta(phi_e)), Eq. (10)
  Problem(...)                 the ersatz state problem K(phi) U = F (Eq. (9)),
                               with J = sum_e I(phi_e) u_e^T k_e^0 u_e (Eq. (10))
"""
from __future__ import annotations

import numpy as np

from . import fem


def heaviside(phi, eta: float):
    """H_eta of Eq. (8): 0 below -eta, 1 above eta, and in between
    1/2 + phi/(2 eta) + sin(pi phi / eta) / (2 pi)."""
    phi = np.asarray(phi, dtype=np.float64)
    mid = 0.5 + phi / (2.0 * eta) + np.sin(np.pi * phi / eta) / (2.0 * np.pi)
    return np.where(phi < -eta, 0.0, np.where(phi > eta, 1.0, mid))


def heaviside_prime(phi, eta: float):
    """d H_eta / d phi: (1 + cos(pi phi / eta)) / (2 eta) on |phi| <= eta, else 0."""
    phi = np.asarray(phi, dtype=np.float64)
    mid = (1.0 + np.cos(np.pi * phi / eta)) / (2.0 * eta)
    return np.where(np.abs(phi) <= eta, mid, 0.0)


def ersatz(phi, eta: float, eps0: float):
    """I(phi) = (1 - H_eta(phi)) + eps0 H_eta(phi), Eq. (7): 1 in the solid
    (phi < -eta), eps0 in the void (phi > eta)."""
    H = heaviside(phi, eta)
    return (1.0 - H) + eps0 * H


def element_phi(phi_nodes, nx: int, ny: int, nz: int):
    """phi at the element centroids (element e = i + nx(j + ny k)): the Q1
    interpolant at the centre, i.e. the mean of the eight corner values."""
    p = np.asarray(phi_nodes, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1)
    s = np.zeros((nz, ny, nx))
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                s += p[dk:dk + nz, dj:dj + ny, di:di + nx]
    return (s / 8.0).reshape(-1)


def ersatz_modulus(phi_nodes, nx, ny, nz, eta, eps0, E0=1.0):
    """Element moduli of the ersatz material: k_e(phi) = I(phi_e) k_e^0 with
    k_e^0 the full-material (E0) element matrix, so E_e = E0 I(phi_e)."""
    return E0 * ersatz(element_phi(phi_nodes, nx, ny, nz), eta, eps0)


def volume(phi_nodes, nx, ny, nz, eta, h=1.0):
    """Material volume V(phi) = sum_e V_e (1 - H_eta(phi_e)), V_e = h^3."""
    return float(np.sum(1.0 - heaviside(element_phi(phi_nodes, nx, ny, nz), eta)) * h ** 3)


class Problem:
    """The ersatz state problem: the SIMP oracle's grid, supports, load,
    assembly and direct solve, with the element moduli taken from the level
    set (Eq. (9)) instead of the SIMP law (Eq. (1))."""

    def __init__(self, nx, ny, nz, bc, load, phi_nodes, eta, eps0, E0=1.0, nu=0.3, h=1.0,
                 load_magnitude=1.0):
        self.grid = fem.Grid(nx, ny, nz, h)
        self.phi = np.asarray(phi_nodes, dtype=np.float64)
        self.eta, self.eps0, self.E0 = float(eta), float(eps0), float(E0)
        self.phi_e = element_phi(self.phi, nx, ny, nz)
        self.k0 = fem.element_stiffness(h, nu)
        self.E = E0 * ersatz(self.phi_e, eta, eps0)
        self.K = fem.assemble(self.grid, self.E, self.k0)
        self.f = fem.load_vector(self.grid, load, load_magnitude)
        self.fixed = fem.fixed_dofs(self.grid, bc)
        self.f[self.fixed] = 0.0

    def solve(self):
        return fem.solve_direct(self.K, self.f, self.fixed, self.grid)

    def compliance(self, u):
        """J = F^T U (= U^T K(phi) U at equilibrium)."""
        return fem.compliance(self.f, u)

    def compliance_energy(self, u):
        """J = sum_e I(phi_e) u_e^T k_e^0 u_e, Eq. (10)."""
        return fem.compliance_energy(self.grid, u, self.E, self.k0)

    def element_energies_unit(self, u):
        """w_e = u_e^T k^0(E = 1) u_e per element."""
        return fem.element_energies(self.grid, u, self.k0)

    def dJ_dphi_e(self, u):
        """Derivative of J with respect to the element value phi_e (compliance
        is self-adjoint, so no adjoint solve): -E0 I'(phi_e) w_e =
        E0 (1 - eps0) H'(phi_e) w_e."""
        return self.E0 * (1.0 - self.eps0) * heaviside_prime(self.phi_e, self.eta) * \
            self.element_energies_unit(u)


# --------------------------------------------------------------------------
# Shape derivatives, Hilbertian extension, Hamilton-Jacobi, reinitialisation
# (Sec. 2.2.5-2.2.8, Eqs. (14)-(24)).  Unit element edge h unless given.
# --------------------------------------------------------------------------

def q1_values(xi: float, eta_: float, zeta: float) -> np.ndarray:
    """The 8 trilinear shape functions at (xi, eta, zeta) in [-1, 1]^3, in the
    oracle's local node order (fem.LOCAL_NODES)."""
    s = 2.0 * fem.LOCAL_NODES - 1.0
    return (1 + xi * s[:, 0]) * (1 + eta_ * s[:, 1]) * (1 + zeta * s[:, 2]) / 8.0


def _gauss2():
    p = 1.0 / np.sqrt(3.0)
    return [(a, b, c) for c in (-p, p) for b in (-p, p) for a in (-p, p)]  # unit weights


def shape_rhs(grid: fem.Grid, u: np.ndarray, phi_nodes, eta: float, E0: float = 1.0,
              nu: float = 0.3):
    """Nodal vectors of the relaxed shape derivatives, by 2x2x2 Gauss
    quadrature per element with phi and grad(phi) from the Q1 interpolant:

      bJ[n] = int_D sigma(u):eps(u) N_n H'_eta(phi) |grad phi| dx   (Eq. (14), w = N_n)
      bV[n] = int_D N_n H'_eta(phi) |grad phi| dx                  (Eq. (15) is -bV / V_D)

    sigma:eps = eps^T D(E0) eps, the strain energy density of the solid
    material (Voigt, engineering shear).  The augmented-Lagrangian right-hand
    side of Eqs. (16)-(17) is bJ + ((lambda - Lambda C) / V_D) bV."""
    h = grid.h
    jac = h / 2.0
    detJ = jac ** 3
    D = fem.constitutive_matrix(E0, nu)
    en = grid.element_nodes()                       # (ne, 8)
    ue = np.asarray(u, dtype=np.float64)[grid.element_dofs()]  # (ne, 24)
    pc = np.asarray(phi_nodes, dtype=np.float64)[en]           # (ne, 8)
    bJ = np.zeros(grid.n_nodes)
    bV = np.zeros(grid.n_nodes)
    for (a, b, c) in _gauss2():
        N = q1_values(a, b, c)                      # (8,)
        dN = fem.shape_gradients(a, b, c) / jac     # (8, 3)
        B = fem.strain_displacement(dN)             # (6, 24)
        phq = pc @ N
        gph = pc @ dN                               # (ne, 3)
        g = heaviside_prime(phq, eta) * np.linalg.norm(gph, axis=1) * detJ
        eps = ue @ B.T                              # (ne, 6)
        e = np.einsum("ei,ij,ej->e", eps, D, eps)
        np.add.at(bJ, en, (g * e)[:, None] * N[None, :])
        np.add.at(bV, en, g[:, None] * N[None, :])
    return bJ, bV


def q1_element_matrices(h: float = 1.0):
    """Element Laplacian int grad N_a . grad N_b and mass int N_a N_b of the
    Q1 brick of edge h (2x2x2 Gauss, exact for these integrands)."""
    jac = h / 2.0
    detJ = jac ** 3
    K = np.zeros((8, 8))
    M = np.zeros((8, 8))
    for (a, b, c) in _gauss2():
        N = q1_values(a, b, c)
        dN = fem.shape_gradients(a, b, c) / jac
        K += detJ * dN @ dN.T
        M += detJ * np.outer(N, N)
    return K, M


def hilbertian_matrix(grid: fem.Grid, ell: float):
    """A_H of Eq. (20): the Q1 discretisation of int (ell^2 grad v . grad w + v w)."""
    import scipy.sparse as sp
    Ke, Me = q1_element_matrices(grid.h)
    Ae = ell * ell * Ke + Me
    en = grid.element_nodes()
    rows = np.repeat(en, 8, axis=1).reshape(-1)
    cols = np.tile(en, (1, 8)).reshape(-1)
    vals = np.tile(Ae.reshape(-1), grid.n_elem)
    return sp.csr_matrix((vals, (rows, cols)), shape=(grid.n_nodes, grid.n_nodes))


def loaded_nodes(grid: fem.Grid, load: int) -> np.ndarray:
    """Gamma_N: the nodes that carry a share of the external load (mask)."""
    f = fem.load_vector(grid, load).reshape(-1, 3)
    return np.any(f != 0.0, axis=1)


def hilbertian_solve(grid: fem.Grid, ell: float, b: np.ndarray, dirichlet: np.ndarray):
    """Solve A_H v = b with v = 0 on the masked nodes (the traction boundary,
    Sec. 2.2.6), by a sparse direct solve on the free nodes."""
    import scipy.sparse.linalg as sla
    A = hilbertian_matrix(grid, ell)
    free = ~np.asarray(dirichlet, bool)
    v = np.zeros(grid.n_nodes)
    v[free] = sla.spsolve(A[free][:, free].tocsc(), np.asarray(b, np.float64)[free])
    return v


def _one_sided(phi, axis, h):
    """Backward and forward differences along `axis`; a difference that would
    reach outside the grid is 0 (the level set is extended by its boundary
    value)."""
    dm = np.zeros_like(phi)
    dp = np.zeros_like(phi)
    sl = [slice(None)] * phi.ndim
    lo, hi = list(sl), list(sl)
    lo[axis], hi[axis] = slice(1, None), slice(None, -1)
    d = (phi[tuple(lo)] - phi[tuple(hi)]) / h       # phi_{i+1} - phi_i at i
    dm[tuple(lo)] = d                                # backward difference at i+1
    dp[tuple(hi)] = d                                # forward difference at i
    return dm, dp


def _upwind_norms(phi, h):
    """First-order Godunov gradient norms for the two signs of the speed:
    (grad+ for speed > 0, grad- for speed < 0)."""
    gp = np.zeros_like(phi)
    gm = np.zeros_like(phi)
    for ax in range(3):
        dm, dp = _one_sided(phi, ax, h)
        gp += np.maximum(dm, 0.0) ** 2 + np.minimum(dp, 0.0) ** 2
        gm += np.minimum(dm, 0.0) ** 2 + np.maximum(dp, 0.0) ** 2
    return np.sqrt(gp), np.sqrt(gm)


def _grid3(a, grid):
    return np.asarray(a, dtype=np.float64).reshape(grid.nz + 1, grid.ny + 1, grid.nx + 1)


def hj_step(grid: fem.Grid, phi_nodes, v_nodes, dt: float):
    """One forward-Euler step of phi_t + v |grad phi| = 0 (Eq. (21)) with the
    first-order Godunov upwind stencil on the node grid."""
    phi = _grid3(phi_nodes, grid)
    v = _grid3(v_nodes, grid)
    gp, gm = _upwind_norms(phi, grid.h)
    out = phi - dt * (np.maximum(v, 0.0) * gp + np.minimum(v, 0.0) * gm)
    return out.reshape(-1)


def cfl_dt(grid: fem.Grid, v_nodes, gamma: float) -> float:
    """Eq. (22) with CFL number gamma: dt = gamma h / max |v|."""
    return gamma * grid.h / float(np.max(np.abs(v_nodes)))


def hj_evolve(grid: fem.Grid, phi_nodes, v_nodes, gamma: float, steps: int):
    dt = cfl_dt(grid, v_nodes, gamma)
    phi = np.asarray(phi_nodes, np.float64)
    for _ in range(steps):
        phi = hj_step(grid, phi, v_nodes, dt)
    return phi


def smeared_sign(grid: fem.Grid, phi_nodes):
    """S(phi) = phi / sqrt(phi^2 + h^2 |grad phi|^2) (Eq. (24)), |grad phi| by
    central differences (one-sided on the boundary faces)."""
    phi = _grid3(phi_nodes, grid)
    g2 = np.zeros_like(phi)
    for ax in range(3):
        g2 += np.gradient(phi, grid.h, axis=ax) ** 2
    return (phi / np.sqrt(phi * phi + grid.h * grid.h * g2)).reshape(-1)


def reinit_step(grid: fem.Grid, phi_nodes, dt: float):
    """One step of phi_t + S(phi)(|grad phi| - 1) = 0 (Eq. (23)), the sign
    recomputed from the current phi, the same upwind stencil as hj_step."""
    phi = _grid3(phi_nodes, grid)
    S = _grid3(smeared_sign(grid, phi_nodes), grid)
    gp, gm = _upwind_norms(phi, grid.h)
    out = phi - dt * (np.maximum(S, 0.0) * gp + np.minimum(S, 0.0) * gm - S)
    return out.reshape(-1)


def reinit(grid: fem.Grid, phi_nodes, gamma: float = 0.5, tol: float = 1e-4,
           max_steps: int = 500):
    """Iterate reinit_step with dt = gamma h (|S| <= 1) until the largest change
    of phi in a step is at most tol * h; returns (phi, steps)."""
    phi = np.asarray(phi_nodes, np.float64)
    dt = gamma * grid.h
    for s in range(1, max_steps + 1):
        new = reinit_step(grid, phi, dt)
        change = float(np.max(np.abs(new - phi)))
        phi = new
        if change <= tol * grid.h:
            return phi, s
    return phi, max_steps
