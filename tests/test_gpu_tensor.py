"""The tensor-core operator (TOPO_OPERATOR_TENSOR: k_tc_tma, the element
products K0 U_e as TF32 GEMMs on tcgen05 with the accumulator in TMEM)
against the FP64 oracle, through the C ABI.

Tolerances, from the arithmetic:
  * the CG operator runs three TF32 passes (hi*hi + hi*lo + lo*hi, both
    operands split into a TF32 part and an FP32 remainder that the MMA
    truncates to TF32): each product carries ~2^-21 relative error, the
    24-term FP32 sums ~2^-24 each; on random x (no cancellation beyond a
    factor ~10) the relative 2-norm error of K x is <= 5e-6;
  * solves (the smoother's operator in one TF32 pass, 2^-11: a fixed
    approximation inside the preconditioner) stop on the library's true FP64
    residual, so at rtol = 1e-10 u and c match the direct solution to 1e-8
    and dc to 1e-6 of its max-norm, as for the SIMT kernels.
Grids need ny >= 6 for the 8-row tiles; smaller ones fall back to the SIMT
kernels (checked too)."""
import numpy as np
import pytest

from oracle import fem
from paper_2605_04735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TENSOR = 4


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
    (40, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),     # ragged x tiles of 15, y tiles of 7
    (33, 10, 12, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (17, 6, 5, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION),   # the smallest ny the tiles take
    (40, 20, 20, I.BC_CORNERS, I.LOAD_DISC_XL),
    (70, 12, 9, I.BC_MBB_STRIP, I.LOAD_HALFDISC_X0_TOP),
    (5, 3, 3, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),      # falls back to the SIMT kernels
]


@pytest.mark.parametrize("case", CASES)
def test_tensor_operator_matches_assembled_K(topo, case):
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 23)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    x = np.random.default_rng(6).normal(size=P.grid.n_dof)
    xm = x.copy()
    xm[P.fixed] = 0.0
    y_ref = P.K @ xm
    y_ref[P.fixed] = 0.0
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_operator(TENSOR)
        m.set_density(rho)
        y = m.apply(x, precision=topo.PREC_FP32)
        y2 = m.apply(x, precision=topo.PREC_FP32)
    assert _rel(y, y_ref) <= 5e-6
    assert np.all(y[P.fixed] == 0.0)
    assert np.array_equal(y, y2)  # deterministic


def test_tensor_operator_keeps_accuracy_under_rigid_translation(topo):
    """Each element row is shifted by its corner 0 before the MMA, so a rigid
    translation 1e5 times the strain-carrying part does not swamp K x: away
    from the masked planes (whose elements hold the translation's jump) the
    result matches the exact product of the FP32-rounded input to the
    arithmetic's own error."""
    nx, ny, nz = 40, 9, 7
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 19)
    P = fem.Problem(nx, ny, nz, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION, rho)
    X = P.grid.node_ijk().astype(float)
    x = 0.01 * np.sin(X @ np.array([0.3, 0.5, 0.7]))[:, None] * np.ones((1, 3))
    x = (x + np.array([1e3, -2e3, 5e2])).reshape(-1)
    x32 = x.astype(np.float32).astype(np.float64)  # what an FP32 kernel receives
    x32[P.fixed] = 0.0
    y_ref = P.K @ x32
    y_ref[P.fixed] = 0.0
    with topo.Mesh(nx, ny, nz, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION) as m:
        m.set_operator(TENSOR)
        m.set_density(rho)
        y = m.apply(x, precision=topo.PREC_FP32)
    ijk = P.grid.node_ijk()
    inner = np.repeat((ijk[:, 0] > 1) & (ijk[:, 1] > 1) & (ijk[:, 2] > 1), 3)
    assert _rel(y[inner], y_ref[inner]) <= 2e-6


@pytest.mark.parametrize("case", CASES[:5])
def test_tensor_solve_matches_direct_oracle(topo, case):
    nx, ny, nz, bc, load = case
    if bc == I.BC_ROLLER_BOX:
        load = I.LOAD_FACE_XL_TRACTION
    rho = I.density_cone_smoothed(nx, ny, nz, 41)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    u_ref = P.solve()
    opts = topo.default_opts(rtol=1e-10)
    out = {}
    for op in (0, TENSOR):
        with topo.Mesh(nx, ny, nz, bc, load) as m:
            m.set_operator(op)
            m.set_density(rho)
            info = m.solve(opts)
            out[op] = (m.displacement(), m.compliance(), m.sensitivity(), info)
    u, c, dc, info = out[TENSOR]
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert _rel(u, u_ref) <= 1e-8
    assert c == pytest.approx(P.compliance(u_ref), rel=1e-8)
    dc_ref = P.sensitivity(u_ref)
    assert np.abs(dc - dc_ref).max() <= 1e-6 * np.abs(dc_ref).max()
    # the TF32 smoother costs at most a few iterations more than the FP32 one
    assert info.iters <= out[0][3].iters * 1.3 + 3


def test_tensor_batch_matches_single_solves(topo):
    nx, ny, nz, nb = 48, 16, 12, 4
    opts = topo.default_opts(rtol=1e-10)
    rhos = [I.density_cone_smoothed(nx, ny, nz, 60 + b) for b in range(nb)]
    group = topo.create_batch(nb, nx, ny, nz, I.BC_MBB, I.LOAD_EDGE_X0_TOP, opts=opts)
    try:
        for m in group:
            m.set_operator(TENSOR)
        topo.set_density_many(group, np.stack(rhos))
        infos = topo.solve_many(group, opts)
        res = [(m.displacement(), m.compliance()) for m in group]
    finally:
        for m in group:
            m.close()
    for b in range(nb):
        with topo.Mesh(nx, ny, nz, I.BC_MBB, I.LOAD_EDGE_X0_TOP) as m:
            m.set_density(rhos[b])
            m.solve(opts)
            u1, c1 = m.displacement(), m.compliance()
        assert infos[b].status == 0 and infos[b].rel_residual <= 1e-10
        assert _rel(res[b][0], u1) <= 1e-8
        assert res[b][1] == pytest.approx(c1, rel=1e-8)
