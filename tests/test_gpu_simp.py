"""The device SIMP update (filter Eq. (4) + OC) against the CPU oracle."""
import numpy as np
import pytest

from oracle import fem, simp
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


@pytest.mark.parametrize("R", [2.0, 1.5, 2.5])
def test_filter_matches_oracle(topo, R):
    nx, ny, nz = 37, 10, 9
    rho = I.density_uniform(nx, ny, nz, 0.001, 1.0, 3)
    dc = -I.rng(4).uniform(0, 2, nx * ny * nz)
    with topo.Mesh(nx, ny, nz) as m:
        m.set_density(rho)
        got = m.filter(dc, radius=R)
    ref = simp.sensitivity_filter(nx, ny, nz, rho, dc, R)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("bc,load", [(I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
                                     (I.BC_MBB, I.LOAD_EDGE_X0_TOP)])
def test_simp_update_matches_oracle(topo, bc, load):
    nx, ny, nz = 40, 12, 10
    rho = I.density_cone_smoothed(nx, ny, nz, 9)
    so = topo.default_simp_opts(volfrac=0.35)
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_density(rho)
        m.solve(topo.default_opts(rtol=1e-10))
        u = m.displacement()
        info = m.simp_update(so)
        new = m.density()
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    dc = P.sensitivity(u)
    dcf = simp.sensitivity_filter(nx, ny, nz, rho, dc, 2.0)
    ref, lam = simp.oc_update(rho, dcf, 0.35)
    assert abs(info.compliance - P.compliance(u)) <= 1e-12 * info.compliance
    assert abs(info.volume - 0.35) <= 1e-5 and abs(new.mean() - 0.35) <= 1e-5
    assert abs(info.lambda_ / lam - 1) <= 1e-4
    assert np.abs(new - ref).max() <= 2e-5
    assert abs(info.change - np.abs(ref - rho).max()) <= 2e-5


def test_simp_loop_follows_oracle(topo):
    """Four SIMP iterations from a uniform start: the device loop (FP32 GMG
    solves + FP64 refinement to 1e-10) follows the oracle's loop (direct
    solves), and the volume stays at V_f."""
    nx, ny, nz, vf = 24, 12, 12, 0.4
    rho0 = np.full(nx * ny * nz, vf, np.float32)
    iters = 4
    with topo.Mesh(nx, ny, nz) as m:
        hist = topo.simp_optimize(m, rho0, topo.default_simp_opts(volfrac=vf),
                                  topo.default_opts(rtol=1e-10), max_iter=iters, tol=0.0)
        rho_gpu = m.density()
    r = rho0.astype(np.float64)
    href = []
    for _ in range(iters):
        P = fem.Problem(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, r.astype(np.float32))
        u = P.solve()
        dcf = simp.sensitivity_filter(nx, ny, nz, P.rho, P.sensitivity(u), 2.0)
        new, _ = simp.oc_update(P.rho, dcf, vf)
        href.append((P.compliance(u), new.mean(), np.abs(new - P.rho).max()))
        r = new.astype(np.float32).astype(np.float64)
    for (c, v, ch), (cr, vr, chr_) in zip(hist, href):
        assert abs(c - cr) <= 1e-5 * cr
        assert abs(v - vf) <= 1e-5 and abs(ch - chr_) <= 1e-4
    assert np.abs(rho_gpu - r).max() <= 1e-3
    assert hist[-1][0] < hist[0][0]  # the design improves
