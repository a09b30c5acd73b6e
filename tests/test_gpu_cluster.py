"""The cluster form of the one-column modal operator (TOPO_OPERATOR_MODAL_CLUSTER:
the x tiles of a grid row run as one thread-block cluster and pass the halo
column's corner sums through distributed shared memory).  Its K x against the
oracle's assembled K (Eq. (2)'s stiffness, k_e = E_e k0 of Eq. (3)) on grids
whose x extent is a multiple of 16 (the last CTA's extra node column) and not,
from one CTA to the eight of a portable cluster; solves with the form against
the direct oracle; and batched solves (the multigrid's 18- and 10-row tiles
on its coarse levels) against the same designs in the tiled form."""
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
    # (nx, ny, nz, bc, load): 1, 2, 3, 6 and 8 CTAs per cluster; nx = 16 k
    # gives the last CTA the node column nx on its lane 15
    (16, 12, 6, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (32, 12, 7, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (47, 13, 9, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION),
    (48, 16, 16, I.BC_CORNERS, I.LOAD_DISC_XL),
    (96, 12, 5, I.BC_MBB_STRIP, I.LOAD_HALFDISC_X0_TOP),
    (128, 12, 4, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (113, 12, 6, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
]


@pytest.mark.parametrize("case", CASES)
def test_cluster_operator_matches_assembled_K(topo, case):
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 29)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    x = np.random.default_rng(7).normal(size=P.grid.n_dof)
    xm = x.copy()
    xm[P.fixed] = 0.0
    y_ref = P.K @ xm
    y_ref[P.fixed] = 0.0
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_operator(topo.OPERATOR_MODAL_CLUSTER)
        m.set_density(rho)
        y = m.apply(x, precision=topo.PREC_FP32)
        m.set_operator(topo.OPERATOR_MODAL_SINGLE)
        y1 = m.apply(x, precision=topo.PREC_FP32)
    assert _rel(y, y_ref) <= 2e-6
    assert np.all(y[P.fixed] == 0.0)
    # the same arithmetic per element and node as the tiled form: only the
    # order of the x-neighbour sum differs at tile edges
    assert _rel(y, y1) <= 1e-6


@pytest.mark.parametrize("case", [CASES[1], CASES[3], (128, 12, 8, I.BC_MBB, I.LOAD_EDGE_X0_TOP)])
def test_cluster_solve_matches_direct_oracle(topo, case):
    """FP32 GMG-PCG with FP64 refinement on the cluster form: every smoother
    epilogue (Chebyshev steps with the on-the-fly Jacobi diagonal, the
    residual forms, the CG apply with its p.Ap) runs through it."""
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.05, 1.0, 31)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    u_ref = P.solve()
    c_ref = P.compliance(u_ref)
    dc_ref = P.sensitivity(u_ref)
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_operator(topo.OPERATOR_MODAL_CLUSTER)
        m.set_density(rho)
        info = m.solve(topo.default_opts(rtol=1e-10))
        u, c, dc = m.displacement(), m.compliance(), m.sensitivity()
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert _rel(u, u_ref) <= 1e-8
    assert abs(c - c_ref) <= 1e-8 * abs(c_ref)
    assert np.abs(dc - dc_ref).max() <= 1e-6 * np.abs(dc_ref).max()


def test_cluster_batch_matches_tiled_batch(topo):
    """A 96x32x32 mesh group (the benchmark's grid: 12-row tiles on the
    finest level, 18 and 10 rows on the coarser ones) solved with the
    cluster form and with the tiled form: the same designs to the stopping
    tolerance."""
    nx, ny, nz, nb = 96, 32, 32, 3
    opts = topo.default_opts(rtol=1e-10)
    rhos = [I.density_cone_smoothed(nx, ny, nz, 50 + b) for b in range(nb)]
    out = {}
    for op in (topo.OPERATOR_MODAL_SINGLE, topo.OPERATOR_MODAL_CLUSTER):
        meshes = topo.create_batch(nb, nx, ny, nz, I.BC_MBB, I.LOAD_EDGE_X0_TOP, opts=opts)
        try:
            for m, r in zip(meshes, rhos):
                m.set_operator(op)
                m.set_density(r)
            infos = topo.solve_many(meshes, opts)
            out[op] = [(i, m.displacement(), m.compliance()) for i, m in zip(infos, meshes)]
        finally:
            for m in meshes:
                m.close()
    for (i1, u1, c1), (i2, u2, c2) in zip(out[topo.OPERATOR_MODAL_SINGLE],
                                          out[topo.OPERATOR_MODAL_CLUSTER]):
        assert i1.status == 0 and i2.status == 0
        assert i2.rel_residual <= 1e-10
        assert _rel(u2, u1) <= 1e-8
        assert c2 == pytest.approx(c1, rel=1e-8)


def test_cluster_batch_designs_sit_out_after_converging(topo):
    """Designs of a group that converge at different outer steps: the ones
    done early sit out the later launches (whole clusters return at once) and
    keep their results; each design matches its own solve alone."""
    nx, ny, nz, nb = 48, 12, 12, 4
    opts = topo.default_opts(rtol=1e-10)
    rhos = [np.ones(nx * ny * nz, np.float32)] + \
           [I.density_voids(nx, ny, nz, 8, seed=s, rmin=2.0, rmax=4.0) for s in range(nb - 1)]
    meshes = topo.create_batch(nb, nx, ny, nz, opts=opts)
    try:
        for m, r in zip(meshes, rhos):
            m.set_operator(topo.OPERATOR_MODAL_CLUSTER)
            m.set_density(r)
        infos = topo.solve_many(meshes, opts)
        us = [m.displacement() for m in meshes]
    finally:
        for m in meshes:
            m.close()
    assert len({i.outer for i in infos}) > 1  # they do finish at different steps
    for b in range(nb):
        with topo.Mesh(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM) as m:
            m.set_operator(topo.OPERATOR_MODAL_CLUSTER)
            m.set_density(rhos[b])
            info1 = m.solve(opts)
            u1 = m.displacement()
        assert infos[b].status == 0 and infos[b].rel_residual <= 1e-10
        assert infos[b].outer == info1.outer
        assert _rel(us[b], u1) <= 1e-8
