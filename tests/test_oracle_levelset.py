"""Pins of the level-set oracle (Eqs. (7)-(10)) against what the definitions
and the mathematics fix, independent of the oracle's own formulas."""
import numpy as np
import pytest

from oracle import fem, levelset as L
from paper_2605_04735_gb300 import inputs as I


def _nodes(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(float)


@pytest.mark.parametrize("eta", [0.5, 1.0, 2.5])
def test_heaviside_values_symmetry_and_continuity(eta):
    assert L.heaviside(-eta, eta) == pytest.approx(0.0, abs=1e-15)
    assert L.heaviside(eta, eta) == pytest.approx(1.0, abs=1e-15)
    assert L.heaviside(0.0, eta) == 0.5
    phi = np.random.default_rng(1).uniform(-3 * eta, 3 * eta, 1000)
    assert np.allclose(L.heaviside(phi, eta) + L.heaviside(-phi, eta), 1.0, atol=1e-15)
    # continuous at the band edges, monotone everywhere
    e = 1e-9
    for x in (-eta, eta):
        assert abs(L.heaviside(x - e, eta) - L.heaviside(x + e, eta)) < 1e-8
    xs = np.linspace(-2 * eta, 2 * eta, 4001)
    assert np.all(np.diff(L.heaviside(xs, eta)) >= -1e-16)


@pytest.mark.parametrize("eta", [0.5, 1.5])
def test_heaviside_derivative_by_differences_and_unit_mass(eta):
    xs = np.linspace(-1.5 * eta, 1.5 * eta, 301)
    d = 1e-6
    fd = (L.heaviside(xs + d, eta) - L.heaviside(xs - d, eta)) / (2 * d)
    assert np.allclose(L.heaviside_prime(xs, eta), fd, atol=1e-6)
    fine = np.linspace(-eta, eta, 200001)
    mass = np.trapezoid(L.heaviside_prime(fine, eta), fine)
    assert mass == pytest.approx(1.0, abs=1e-9)
    assert L.heaviside_prime(eta, eta) == pytest.approx(0.0, abs=1e-15)


def test_ersatz_limits():
    eta, eps0 = 1.0, 1e-3
    assert L.ersatz(-5.0, eta, eps0) == 1.0
    assert L.ersatz(5.0, eta, eps0) == eps0
    assert L.ersatz(0.0, eta, eps0) == pytest.approx((1 + eps0) / 2)
    phi = np.linspace(-3, 3, 101)
    v = L.ersatz(phi, eta, eps0)
    assert np.all((v >= eps0 - 1e-15) & (v <= 1 + 1e-15))


def test_element_phi_reproduces_linear_fields():
    nx, ny, nz = 5, 4, 3
    X = _nodes(nx, ny, nz)
    a, b = np.array([0.3, -1.1, 0.7]), 2.5
    pe = L.element_phi(X @ a + b, nx, ny, nz)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    C = np.stack([i.ravel(), j.ravel(), k.ravel()], 1) + 0.5
    assert np.allclose(pe, C @ a + b, atol=1e-13)


def test_volume_of_a_half_space_is_exact():
    nx, ny, nz = 12, 5, 4
    X = _nodes(nx, ny, nz)
    for c in (3, 7):
        phi = X[:, 0] - c  # solid for x < c; element centroids sit 0.5 off the plane
        assert L.volume(phi, nx, ny, nz, eta=0.4) == c * ny * nz


def test_volume_of_a_ball_approaches_the_exact_volume():
    n, r = 32, 9.0
    X = _nodes(n, n, n)
    phi = np.linalg.norm(X - n / 2, axis=1) - r  # signed distance, solid inside
    v = L.volume(phi, n, n, n, eta=1.0)
    assert v == pytest.approx(4.0 / 3.0 * np.pi * r ** 3, rel=0.02)


def test_all_solid_level_set_reduces_to_solid_simp_problem():
    nx, ny, nz = 6, 3, 3
    phi = -10.0 * np.ones((nx + 1) * (ny + 1) * (nz + 1))
    P = L.Problem(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, phi, 1.0, 1e-3)
    Q = fem.Problem(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, np.ones(nx * ny * nz))
    u, v = P.solve(), Q.solve()
    assert np.allclose(u, v, rtol=1e-12, atol=1e-14)
    assert P.compliance(u) == pytest.approx(Q.compliance(v), rel=1e-12)


def test_ersatz_compliance_energy_identity_and_element_derivative():
    nx, ny, nz, eta, eps0 = 6, 3, 3, 1.5, 1e-3
    X = _nodes(nx, ny, nz)
    # a void ball of radius 1.2 in the middle (phi > 0 inside it), the band straddles it
    phi = 1.2 - np.linalg.norm(X - np.array([3.0, 1.5, 1.5]), axis=1)
    P = L.Problem(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, phi, eta, eps0)
    u = P.solve()
    assert P.compliance(u) == pytest.approx(P.compliance_energy(u), rel=1e-11)
    g = P.dJ_dphi_e(u)
    band = np.flatnonzero(np.abs(P.phi_e) < eta)
    assert band.size > 0 and np.all(g >= 0)
    # central differences of J with respect to one element value, at fixed grid/load
    d = 1e-5
    for e in band[:4]:
        Js = []
        for s in (+1, -1):
            pe = P.phi_e.copy()
            pe[e] += s * d
            E = L.ersatz(pe, eta, eps0)
            K = fem.assemble(P.grid, E, P.k0)
            us = fem.solve_direct(K, P.f, P.fixed, P.grid)
            Js.append(fem.compliance(P.f, us))
        fd = (Js[0] - Js[1]) / (2 * d)
        assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-10 * abs(P.compliance(u)))


# ---- shape derivatives, Hilbertian extension, HJ, reinitialisation --------

def test_hilbertian_matrix_pins():
    g = fem.Grid(6, 4, 3)
    Klap = L.hilbertian_matrix(g, 1.0) - L.hilbertian_matrix(g, 0.0)
    M = L.hilbertian_matrix(g, 0.0)
    one = np.ones(g.n_nodes)
    assert np.abs(Klap @ one).max() < 1e-13          # constants are in the kernel
    assert one @ (M @ one) == pytest.approx(6 * 4 * 3, rel=1e-13)  # total volume
    X = g.node_ijk().astype(float)
    a = np.array([0.4, -1.3, 0.9])
    v = X @ a                                         # linear field: exact energy
    assert v @ (Klap @ v) == pytest.approx(a @ a * 6 * 4 * 3, rel=1e-12)
    # constant data extends to the same constant (natural boundary, no Dirichlet)
    b = 2.5 * (L.hilbertian_matrix(g, 0.0) @ one)
    vs = L.hilbertian_solve(g, 2.0, b, np.zeros(g.n_nodes, bool))
    assert np.allclose(vs, 2.5, atol=1e-12)


def test_hilbertian_solve_matches_the_1d_modal_solution():
    """-ell^2 v'' + v = cos(pi x / Lx) with natural boundaries has
    v = cos(pi x / Lx) / (1 + (ell pi / Lx)^2); the Q1 solution converges to it."""
    nx, ny, nz, ell = 32, 2, 2, 3.0
    g = fem.Grid(nx, ny, nz)
    X = g.node_ijk().astype(float)
    gx = np.cos(np.pi * X[:, 0] / nx)
    b = L.hilbertian_matrix(g, 0.0) @ gx              # int g N_n with g interpolated
    v = L.hilbertian_solve(g, ell, b, np.zeros(g.n_nodes, bool))
    exact = gx / (1.0 + (ell * np.pi / nx) ** 2)
    assert np.abs(v - exact).max() < 5e-3


@pytest.mark.parametrize("eta", [1.5, 2.0])
def test_shape_rhs_measures_the_interface_and_scales_with_uniform_energy(eta):
    nx, ny, nz = 16, 6, 5
    g = fem.Grid(nx, ny, nz)
    X = g.node_ijk().astype(float)
    phi = X[:, 0] - 7.3                              # plane x = 7.3, |grad phi| = 1
    t = 1e-3                                         # uniform strain eps_xx = t
    u = np.zeros(g.n_dof)
    u[0::3] = t * X[:, 0]
    bJ, bV = L.shape_rhs(g, u, phi, eta)
    # coarea: int H'(phi) |grad phi| = area of the zero level set = ny * nz
    assert bV.sum() == pytest.approx(ny * nz, rel=2e-3)
    lam, mu = fem.lame(1.0, 0.3)
    assert np.allclose(bJ, (lam + 2 * mu) * t * t * bV, rtol=1e-12, atol=1e-20)


def test_shape_rhs_measures_a_sphere():
    n, r = 24, 7.0
    g = fem.Grid(n, n, n)
    X = g.node_ijk().astype(float)
    phi = np.linalg.norm(X - n / 2, axis=1) - r
    _, bV = L.shape_rhs(g, np.zeros(g.n_dof), phi, 1.5)
    assert bV.sum() == pytest.approx(4 * np.pi * r * r, rel=0.03)


def test_hj_step_moves_a_plane_by_v_dt_and_follows_hopf_lax_at_a_kink():
    g = fem.Grid(12, 3, 3)
    X = g.node_ijk().astype(float)
    dt = 0.3
    for v in (1.0, -1.0):
        phi = X[:, 0] - 5.5
        out = L.hj_step(g, phi, v * np.ones(g.n_nodes), dt)
        inner = (X[:, 0] > 0) & (X[:, 0] < g.nx)
        assert np.allclose(out[inner], phi[inner] - v * dt, atol=1e-14)
    # phi0 = |x - 6|: phi(x, t) = min over |y - x| <= t of phi0 = max(|x - 6| - t, 0)
    phi = np.abs(X[:, 0] - 6.0)
    out = L.hj_step(g, phi, np.ones(g.n_nodes), dt)
    inner = (X[:, 0] > 0) & (X[:, 0] < g.nx)
    assert np.allclose(out[inner], np.maximum(phi[inner] - dt, 0.0), atol=1e-14)
    assert L.cfl_dt(g, np.array([0.5, -2.0]), 0.5) == 0.25


def test_reinit_keeps_a_distance_and_restores_one_from_a_scaled_field():
    g = fem.Grid(20, 4, 4)
    X = g.node_ijk().astype(float)
    sdf = X[:, 0] - 9.4
    out, steps = L.reinit(g, sdf, tol=1e-10, max_steps=5)
    inner = (X[:, 0] > 0) & (X[:, 0] < g.nx)
    assert np.allclose(out[inner], sdf[inner], atol=1e-12)
    out, steps = L.reinit(g, 3.0 * sdf, tol=1e-6, max_steps=400)
    near = inner & (np.abs(sdf) < 3.0)
    assert np.abs(out[near] - sdf[near]).max() < 0.1
    assert np.sign(out[np.abs(sdf) > 0.5]).tolist() == np.sign(sdf[np.abs(sdf) > 0.5]).tolist()
