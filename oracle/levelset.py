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
