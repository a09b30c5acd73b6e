"""The operator in double-word arithmetic (two FP32 words per value, ~48
significand bits), the kernel of the refinement residuals that cannot end a
solve, against the FP64 oracle's assembled K and against the FP64 path.

Tolerances: a double-word operation rounds at ~2^-48 = 3.6e-15 relative
(FP64: 1.1e-16); an element's result takes ~100 such operations on values of
the size of the element's terms, so the 2-norm error of K x relative to the
oracle stays below 1e-12 for random x (1e-11 is asserted).  Under a rigid
translation 1e5 times larger than the strain-carrying part, the corner-0
shift keeps the error relative to K x near the same level (1e-9 asserted;
the FP32 kernel reaches only 2e-2 there).  Solves certify convergence with
an FP64 residual whatever the residual option, so the two options must give
the same displacement to the solve tolerance.
"""
import numpy as np
import pytest

from oracle import fem
from paper_2605_04735_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def topo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04735_gb300 import build
    build.build()
    from paper_2605_04735_gb300 import topo as t
    t.lib()
    return t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    (40, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (33, 10, 12, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (5, 17, 3, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION),
    (1, 1, 1, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (70, 12, 9, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (40, 20, 20, I.BC_CORNERS, I.LOAD_DISC_XL),
]


@pytest.mark.parametrize("case", CASES)
def test_dword_operator_matches_assembled_K(topo, case):
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 17)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    x = np.random.default_rng(5).normal(size=P.grid.n_dof)
    xm = x.copy()
    xm[P.fixed] = 0.0
    y_ref = P.K @ xm
    y_ref[P.fixed] = 0.0
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_density(rho)
        y = m.apply(x, precision=topo.PREC_DWORD)
        y64 = m.apply(x, precision=topo.PREC_FP64)
    assert _rel(y, y_ref) <= 1e-11
    assert _rel(y, y64) <= 1e-11
    assert np.all(y[P.fixed] == 0.0)


@pytest.mark.parametrize("nx", [40, 70])
def test_dword_operator_under_rigid_translation(topo, nx):
    ny, nz = 9, 7
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 19)
    P = fem.Problem(nx, ny, nz, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION, rho)
    g = P.grid
    X = g.node_ijk().astype(float)
    x = 0.01 * np.sin(X @ np.array([0.3, 0.5, 0.7]))[:, None] * np.ones((1, 3))
    x = (x + np.array([1e3, -2e3, 5e2])).reshape(-1)
    xm = x.copy()
    xm[P.fixed] = 0.0
    y_ref = P.K @ xm
    y_ref[P.fixed] = 0.0
    ijk = g.node_ijk()
    interior = (ijk[:, 0] > 1) & (ijk[:, 1] > 1) & (ijk[:, 2] > 1)  # away from the masked planes
    mask = np.repeat(interior, 3)
    with topo.Mesh(nx, ny, nz, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION) as m:
        m.set_density(rho)
        y = m.apply(x, precision=topo.PREC_DWORD)
    assert _rel(y[mask], y_ref[mask]) <= 1e-9


@pytest.mark.parametrize("case", [CASES[1], CASES[5]])
def test_solve_with_dword_residual_matches_fp64_residual(topo, case):
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.05, 1.0, 23)
    res = {}
    for r in (topo.RESIDUAL_DWORD, topo.RESIDUAL_FP64):
        with topo.Mesh(nx, ny, nz, bc, load) as m:
            m.set_density(rho)
            info = m.solve(topo.default_opts(rtol=1e-10, residual=r))
            res[r] = (info, m.displacement(), m.compliance())
    (i_dw, u_dw, c_dw), (i_64, u_64, c_64) = res[topo.RESIDUAL_DWORD], res[topo.RESIDUAL_FP64]
    assert i_dw.status == 0 and i_64.status == 0
    assert i_dw.rel_residual <= 1e-10 and i_64.rel_residual <= 1e-10
    assert i_dw.outer == i_64.outer
    assert _rel(u_dw, u_64) <= 1e-8
    assert c_dw == pytest.approx(c_64, rel=1e-9)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    assert _rel(u_dw, P.solve()) <= 1e-8


def test_residual_option_is_validated(topo):
    with topo.Mesh(8, 4, 4) as m:
        m.set_density(np.ones(8 * 4 * 4, np.float32))
        with pytest.raises(RuntimeError):
            m.solve(topo.default_opts(residual=7))


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]])
def test_sensitivity_from_residual_energies(topo, case):
    """After a solve the sensitivities come from the element energies the
    certifying FP64 residual kernel stored.  Reference: the energies of the
    same displacement in numpy FP64, each element's u shifted by its corner 0
    (k0 annihilates translations, so the shift changes the energy only by
    rounding, and keeps a large displacement from swamping a small strain
    energy); tolerance 1e-11 of the max |dc| (FP64 rounding of ~50-term sums
    of the element's terms)."""
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 37)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_density(rho)
        m.solve(topo.default_opts())
        u = m.displacement()
        dc = m.sensitivity()
        ce = m.compliance_energy()
        c = m.compliance()
    ue = u[P.grid.element_dofs()].reshape(-1, 8, 3)
    ue = (ue - ue[:, :1, :]).reshape(-1, 24)
    w = np.einsum("ea,ab,eb->e", ue, P.k0, ue)
    ref = -3.0 * rho.astype(np.float64) ** 2 * (1.0 - 1e-9) * w
    assert np.abs(dc - ref).max() <= 1e-11 * np.abs(ref).max()
    assert ce == pytest.approx(c, rel=1e-9)
