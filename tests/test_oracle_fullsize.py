"""Pins of the matrix-free FP64 oracle (oracle/fullsize.c) used for the
full-size workloads: its K u must be the assembled K of oracle.fem (itself
pinned by the mechanics tests) applied to u, its CG must reach the direct
Cholesky solution, its energies must be the assembled quadratic forms.
Grids are ragged (odd counts in every direction, so every parity class of
the element loop is uneven)."""
import numpy as np
import pytest

from oracle import fem
from oracle import fullsize as FS
from paper_2605_04735_gb300 import inputs as I

GRIDS = [(1, 1, 1), (3, 2, 2), (5, 3, 4), (7, 4, 3), (2, 5, 7)]


@pytest.mark.parametrize("n", GRIDS)
def test_apply_is_the_assembled_matrix(n):
    g = fem.Grid(*n)
    rng = np.random.default_rng(sum(n))
    E = rng.uniform(1e-3, 1.0, g.n_elem)
    k0 = fem.element_stiffness(1.0, 0.3)
    u = rng.normal(size=g.n_dof)
    K = fem.assemble(g, E, k0)
    ref = K @ u
    y = FS.apply(g, E, k0, u)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_apply_of_a_rigid_motion_is_zero_and_of_a_unit_vector_is_a_column():
    g = fem.Grid(4, 3, 3)
    E = np.random.default_rng(1).uniform(0.1, 1.0, g.n_elem)
    k0 = fem.element_stiffness(1.0, 0.3)
    X = g.node_ijk().astype(float)
    rot = np.stack([-X[:, 1], X[:, 0], np.zeros(len(X))], 1).reshape(-1)  # rotation about z
    assert np.abs(FS.apply(g, E, k0, rot)).max() <= 1e-12
    K = fem.assemble(g, E, k0)
    e = np.zeros(g.n_dof)
    e[3 * g.node(2, 1, 1) + 1] = 1.0
    assert np.abs(FS.apply(g, E, k0, e) - K[:, 3 * g.node(2, 1, 1) + 1].toarray().ravel()).max() \
        <= 1e-15


@pytest.mark.parametrize("n,bc,load", [((6, 4, 4), fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM),
                                       ((8, 4, 2), fem.BC_MBB, fem.LOAD_EDGE_X0_TOP)])
def test_residual_and_energies_match_the_assembled_forms(n, bc, load):
    rho = I.density_uniform(*n, 0.01, 1.0, 4)
    P = fem.Problem(*n, bc, load, rho)
    u = np.random.default_rng(3).normal(size=P.grid.n_dof)
    u[P.fixed] = 0.0
    r, nr = FS.residual(P.grid, P.E, P.k0, P.f, P.fixed, u)
    ref = fem.residual(P.K, P.f, u, P.fixed)
    assert np.abs(r - ref).max() <= 1e-13 * np.abs(ref).max()
    assert nr == pytest.approx(np.linalg.norm(ref), rel=1e-13)
    w = FS.element_energies(P.grid, P.k0, u)
    assert np.allclose(w, fem.element_energies(P.grid, u, P.k0), rtol=1e-13, atol=0)


@pytest.mark.parametrize("n,bc,load,lo", [((12, 4, 4), fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM, 0.01),
                                          ((10, 6, 4), fem.BC_MBB, fem.LOAD_EDGE_X0_TOP, 1e-3)])
def test_cg_reaches_the_direct_solution(n, bc, load, lo):
    rho = I.density_uniform(*n, lo, 1.0, 6)
    P = fem.Problem(*n, bc, load, rho)
    u_ref = P.solve()
    u, it, rel = FS.cg(P.grid, P.E, P.k0, P.f, P.fixed, rtol=1e-12)
    assert rel <= 1e-12 and it > 0
    # the assembled residual of the same u (another summation order: near the
    # FP64 floor the two differ by rounding, not by more)
    assert P.rel_residual(u) <= 2e-12
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    assert np.all(u[P.fixed] == 0.0)
    assert P.compliance(u) == pytest.approx(P.compliance(u_ref), rel=1e-11)


def test_cg_reports_an_unreached_tolerance():
    n = (6, 3, 3)
    P = fem.Problem(*n, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM,
                    I.density_uniform(*n, 0.01, 1.0, 2))
    u, it, rel = FS.cg(P.grid, P.E, P.k0, P.f, P.fixed, rtol=1e-12, maxiter=5)
    assert it == 5 and rel > 1e-12
    assert P.rel_residual(u) == pytest.approx(rel, rel=1e-10)
