"""The device side of the x-slab decomposition on one GPU: every rank's slab
operator (the library's FP64 and FP32 kernels on a mesh of the slab's
element layers with no support) against the oracle's operator on the whole
grid, on the rank's owned node planes, for 2- and 3-way splits; the slab
Jacobi inverse likewise; and the slab Jacobi-PCG driver with the device
operator (one rank) against the direct solution.  The exchange between ranks
is covered by the gloo tests (tests/test_multirank_slab.py); several GPUs
are not available here."""
import numpy as np
import pytest

from oracle import fem
from oracle import fullsize as FS
from paper_2605_04735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NX, NY, NZ = 41, 8, 6


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


def _problem():
    rho = I.density_cone_smoothed(NX, NY, NZ, 55)
    return fem.Problem(NX, NY, NZ, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, rho), rho


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
def test_slab_operators_reproduce_the_whole_grid_rows(topo, world, prec, tol):
    from paper_2605_04735_gb300 import slab as SL
    P, rho = _problem()
    u = np.random.default_rng(9).normal(size=P.grid.n_dof)
    y_ref = FS.apply(P.grid, P.E, P.k0, u)
    diag = fem.assemble(P.grid, P.E, P.k0).diagonal()
    for rank in range(world):
        s = SL.Slab.make(NX, NY, NZ, world, rank)
        op = SL.DeviceSlabOperator(s, rho, precision=prec)
        try:
            y = op.apply_local(s.to_local(u))
            dinv = op.dinv_local()
        finally:
            op.close()
        got = s.from_local(y)
        own = s.from_local(np.ones(s.to_local(u).shape)) > 0
        assert np.linalg.norm((got - y_ref)[own]) <= tol * np.linalg.norm(y_ref[own])
        dref = s.to_local(1.0 / diag)
        o = s.owned
        assert np.allclose(dinv[o], dref[o], rtol=1e-14, atol=0)


def test_slab_cg_with_the_device_operator_reaches_the_direct_solution(topo):
    from paper_2605_04735_gb300 import slab as SL
    P, rho = _problem()
    s = SL.Slab.make(NX, NY, NZ, 1, 0)
    op = SL.DeviceSlabOperator(s, rho, precision=0)
    try:
        fixed = s.to_local(P.fixed.astype(np.float64)) > 0.5
        dinv = np.where(fixed, 0.0, op.dinv_local())
        x, it, rel = SL.jacobi_pcg(s, SL.LocalComm(s), op.apply_local, dinv, s.to_local(P.f),
                                   fixed, rtol=1e-11)
    finally:
        op.close()
    u_ref = P.solve()
    assert rel <= 1e-11
    assert np.linalg.norm(s.from_local(x) - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
