"""The ersatz-material state (level-set stage, Eqs. (7)-(10)) on the device
against the FP64 oracle, through the C ABI.

Tolerances as in test_gpu_parity: solves to a true FP64 relative residual of
1e-10 match the direct solution to 1e-8 (2-norm) and the compliance to 1e-8;
element moduli and volume are FP64 on both sides (1e-12); element energies of
the same u agree to FP64 rounding of the modal quadratic form (1e-10 of the
largest)."""
import numpy as np
import pytest

from oracle import levelset as L
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
    (24, 12, 12, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, 6, 1.0),
    (33, 10, 12, I.BC_MBB, I.LOAD_EDGE_X0_TOP, 5, 1.5),
    (40, 20, 20, I.BC_CORNERS, I.LOAD_DISC_XL, 10, 1.0),
]


@pytest.mark.parametrize("nx,ny,nz,bc,load,nvoid,eta", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_ersatz_state_matches_oracle(topo, nx, ny, nz, bc, load, nvoid, eta, prec):
    eps0 = 1e-3
    phi = I.levelset_voids(nx, ny, nz, nvoid, seed=31 + nx)
    P = L.Problem(nx, ny, nz, bc, load, phi, eta, eps0)
    u_ref = P.solve()
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        vol = m.set_levelset(phi, eta=eta, eps0=eps0)
        info = m.solve(topo.default_opts(precision=prec, rtol=1e-10,
                                         precond=topo.PRECOND_JACOBI if prec == 0
                                         else topo.PRECOND_GMG))
        u = m.displacement()
        c = m.compliance()
        ce = m.compliance_energy()
        w = m.element_energy()
    assert vol == pytest.approx(L.volume(phi, nx, ny, nz, eta), rel=1e-12)
    assert info.rel_residual <= 1e-10
    assert _rel(u, u_ref) <= 1e-8
    assert c == pytest.approx(P.compliance(u_ref), rel=1e-8)
    assert ce == pytest.approx(c, rel=1e-8)
    w_ref = P.element_energies_unit(u)  # the same u on both sides
    assert np.abs(w - w_ref).max() <= 1e-10 * np.abs(w_ref).max()


def test_levelset_then_density_restores_simp_state(topo):
    """set_density after set_levelset gives exactly the SIMP state again."""
    nx, ny, nz = 20, 8, 8
    rho = I.density_uniform(nx, ny, nz, 0.1, 1.0, 3)
    phi = I.levelset_voids(nx, ny, nz, 3, seed=5)
    with topo.Mesh(nx, ny, nz) as m:
        m.set_density(rho)
        m.solve(topo.default_opts(rtol=1e-10))
        c0 = m.compliance()
        m.set_levelset(phi)
        m.solve(topo.default_opts(rtol=1e-10))
        c1 = m.compliance()
        m.set_density(rho)
        m.solve(topo.default_opts(rtol=1e-10))
        c2 = m.compliance()
    assert c1 != pytest.approx(c0, rel=1e-3)
    assert c2 == pytest.approx(c0, rel=1e-9)


def test_levelset_rejects_bad_input(topo):
    nx, ny, nz = 6, 3, 3
    with topo.Mesh(nx, ny, nz) as m:
        phi = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
        with pytest.raises(RuntimeError):
            m.set_levelset(phi[:-1])
        with pytest.raises(RuntimeError):
            m.set_levelset(phi, eta=0.0)
        phi[5] = np.nan
        with pytest.raises(RuntimeError):
            m.set_levelset(phi)
        with pytest.raises(RuntimeError):
            m.element_energy()  # no solve yet
