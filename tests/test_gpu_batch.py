"""Batched solves of a mesh group (topo_create_batch + topo_solve_many): every
design's result against the same design solved alone and against the FP64
oracle.

Both paths stop on the true FP64 relative residual (1e-10 here), so their
displacements agree with the direct solution to ~1e-8 and with each other to
the same order; compliances to 1e-8 relative."""
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


def _alone(topo, nx, ny, nz, bc, load, rho, opts):
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_density(rho)
        info = m.solve(opts)
        return m.displacement(), m.compliance(), m.sensitivity(), info


@pytest.mark.parametrize("nx,ny,nz,bc,load,nb", [
    (40, 12, 10, I.BC_MBB, I.LOAD_EDGE_X0_TOP, 5),
    (33, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, 3),
    (160, 8, 8, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, 3),   # the paired operator kernel
    (40, 20, 20, I.BC_CORNERS, I.LOAD_DISC_XL, 4),
])
def test_batch_matches_single_solves(topo, nx, ny, nz, bc, load, nb):
    opts = topo.default_opts(rtol=1e-10)
    rhos = [I.density_cone_smoothed(nx, ny, nz, 40 + b) for b in range(nb)]
    meshes = topo.create_batch(nb, nx, ny, nz, bc, load, opts=opts)
    try:
        for m, r in zip(meshes, rhos):
            m.set_density(r)
        infos = topo.solve_many(meshes, opts)
        res = [(m.displacement(), m.compliance(), m.sensitivity()) for m in meshes]
    finally:
        for m in meshes:
            m.close()
    for b in range(nb):
        u, c, dc = res[b]
        u1, c1, dc1, info1 = _alone(topo, nx, ny, nz, bc, load, rhos[b], opts)
        assert infos[b].status == 0 and infos[b].rel_residual <= 1e-10
        assert _rel(u, u1) <= 1e-8
        assert c == pytest.approx(c1, rel=1e-8)
        assert np.abs(dc - dc1).max() <= 1e-7 * np.abs(dc1).max()
    if nx * ny * nz <= 6000:  # one design against the direct solution
        P = fem.Problem(nx, ny, nz, bc, load, rhos[0])
        ref = P.solve()
        assert _rel(res[0][0], ref) <= 1e-8


@pytest.mark.parametrize("nx,ny,nz,degree,levels", [
    (40, 12, 10, 1, 0),    # two smoothed levels in the one-kernel coarse end
    (40, 12, 10, 3, 0),
    (33, 9, 7, 6, 0),      # odd extents at every level
    (96, 32, 32, 2, 0),
    (40, 12, 10, 2, 3),    # three levels: one smoothed level and the coarsest in the kernel
    (48, 12, 12, 2, 0),
])
def test_batch_coarse_levels_match_single_solves(topo, nx, ny, nz, degree, levels):
    """Batched V-cycles run the levels of <= 1024 nodes in one kernel per
    design; single designs run them level by level.  Same smoothing degree and
    level count on both sides: the solves agree to the stopping tolerance and
    take the same number of outer steps (inner counts may differ by the FP32
    rounding of the two operator evaluations; convergence is checked after
    every iteration so the counts are comparable)."""
    opts = topo.default_opts(rtol=1e-10, smooth_degree=degree, gmg_levels=levels, check_every=1)
    nb = 3
    rhos = [I.density_cone_smoothed(nx, ny, nz, 70 + b) for b in range(nb)]
    meshes = topo.create_batch(nb, nx, ny, nz, opts=opts)
    try:
        for m, r in zip(meshes, rhos):
            m.set_density(r)
        infos = topo.solve_many(meshes, opts)
        us = [m.displacement() for m in meshes]
    finally:
        for m in meshes:
            m.close()
    for b in range(nb):
        u1, _, _, info1 = _alone(topo, nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM,
                                 rhos[b], opts)
        assert infos[b].status == 0 and infos[b].rel_residual <= 1e-10
        assert infos[b].outer == info1.outer
        assert abs(infos[b].iters - info1.iters) <= max(2, info1.iters // 10)
        assert _rel(us[b], u1) <= 1e-8


def test_batch_designs_converge_at_different_outer_steps(topo):
    """A solid design converges in fewer outer steps than near-binary void
    designs; it sits out the later steps and its result is unchanged."""
    nx, ny, nz, nb = 48, 12, 12, 4
    opts = topo.default_opts(rtol=1e-10)
    rhos = [np.ones(nx * ny * nz, np.float32)] + \
           [I.density_voids(nx, ny, nz, 8, seed=s, rmin=2.0, rmax=4.0) for s in range(nb - 1)]
    meshes = topo.create_batch(nb, nx, ny, nz, opts=opts)
    try:
        for m, r in zip(meshes, rhos):
            m.set_density(r)
        infos = topo.solve_many(meshes, opts)
        us = [m.displacement() for m in meshes]
    finally:
        for m in meshes:
            m.close()
    for b in range(nb):
        u1, _, _, info1 = _alone(topo, nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM,
                                 rhos[b], opts)
        assert infos[b].status == 0
        assert infos[b].outer == info1.outer
        assert _rel(us[b], u1) <= 1e-8


def test_batch_warm_start_and_repeated_solves(topo):
    nx, ny, nz, nb = 36, 10, 10, 3
    opts = topo.default_opts(rtol=1e-9)
    warm = topo.default_opts(rtol=1e-9, warm_start=1)
    meshes = topo.create_batch(nb, nx, ny, nz, I.BC_MBB, I.LOAD_EDGE_X0_TOP, opts=opts)
    try:
        base = [I.density_cone_smoothed(nx, ny, nz, 70 + b) for b in range(nb)]
        for m, r in zip(meshes, base):
            m.set_density(r)
        topo.solve_many(meshes, opts)
        g = np.random.default_rng(3)
        new = [I.perturb(r, g.uniform(0.95, 1.05, r.size)) for r in base]
        for m, r in zip(meshes, new):
            m.set_density(r)
        infos = topo.solve_many(meshes, warm)
        us = [m.displacement() for m in meshes]
        cs = [m.compliance() for m in meshes]
    finally:
        for m in meshes:
            m.close()
    for b in range(nb):
        u1, c1, _, _ = _alone(topo, nx, ny, nz, I.BC_MBB, I.LOAD_EDGE_X0_TOP, new[b], opts)
        assert infos[b].status == 0
        assert _rel(us[b], u1) <= 1e-7
        assert cs[b] == pytest.approx(c1, rel=1e-8)


def test_batch_falls_back_when_not_a_whole_group(topo):
    """Part of a group, a different operator, or freed designs: the designs are
    solved one by one, with the same results."""
    nx, ny, nz, nb = 30, 8, 8, 4
    opts = topo.default_opts(rtol=1e-10)
    rhos = [I.density_uniform(nx, ny, nz, 0.1, 1.0, 90 + b) for b in range(nb)]
    meshes = topo.create_batch(nb, nx, ny, nz, opts=opts)
    try:
        for m, r in zip(meshes, rhos):
            m.set_density(r)
        part = topo.solve_many(meshes[1:3], opts)            # a subset
        meshes[3].set_operator(topo.OPERATOR_GATHER)
        whole = topo.solve_many(meshes, opts)                 # one design differs
        meshes[3].set_operator(topo.OPERATOR_MODAL)
        meshes[0].close()                                     # design 0 freed first
        rest = topo.solve_many(meshes[1:], opts)
        us = [m.displacement() for m in meshes[1:]]
        single = meshes[2].solve(opts)
    finally:
        for m in meshes:
            m.close()
    assert all(i.status == 0 for i in part + whole + rest) and single.status == 0
    for b in range(1, nb):
        u1, _, _, _ = _alone(topo, nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM,
                             rhos[b], opts)
        assert _rel(us[b - 1], u1) <= 1e-8


def test_batch_rejects_bad_arguments(topo):
    with pytest.raises(RuntimeError):
        topo.create_batch(0, 8, 4, 4)
    with pytest.raises(RuntimeError):
        topo.create_batch(2, 8, 5, 4, I.BC_MBB, I.LOAD_EDGE_X0_TOP)  # MBB needs an even ny


def test_batched_density_compliance_sensitivity_match_per_mesh_calls(topo):
    """topo_set_density_many / compliance_many / sensitivity_many on a whole
    group (one launch each) against the per-mesh calls on the same designs:
    densities from host and from device, sensitivities to host and device.
    The batched reductions sum in another block order, so compliances agree
    to rounding (1e-12 relative); sensitivities are elementwise identical."""
    import torch
    nx, ny, nz, nb = 36, 10, 10, 4
    opts = topo.default_opts(rtol=1e-9)
    rhos = np.stack([I.density_cone_smoothed(nx, ny, nz, 120 + b) for b in range(nb)])
    meshes = topo.create_batch(nb, nx, ny, nz, I.BC_MBB, I.LOAD_EDGE_X0_TOP, opts=opts)
    try:
        for src in (rhos, torch.from_numpy(rhos).cuda()):
            topo.set_density_many(meshes, src)
            topo.solve_many(meshes, opts)
            c = topo.compliance_many(meshes)
            dc = topo.sensitivity_many(meshes)
            dc_dev = topo.sensitivity_many(meshes, torch.empty((nb, nx * ny * nz),
                                                               dtype=torch.float64, device="cuda"))
            for b, m in enumerate(meshes):
                assert c[b] == pytest.approx(m.compliance(), rel=1e-12)
                ref = m.sensitivity()
                assert np.array_equal(dc[b], ref)
                assert np.array_equal(dc_dev[b].cpu().numpy(), ref)
                assert np.array_equal(m.density(), rhos[b])
    finally:
        for m in meshes:
            m.close()


def test_batched_io_on_separate_meshes_and_bad_input(topo):
    nx, ny, nz, nb = 12, 6, 6, 3
    rhos = np.stack([I.density_uniform(nx, ny, nz, 0.1, 1.0, 130 + b) for b in range(nb)])
    meshes = [topo.Mesh(nx, ny, nz) for _ in range(nb)]  # not a group: per-mesh calls
    try:
        topo.set_density_many(meshes, rhos)
        topo.solve_many(meshes, topo.default_opts())
        c = topo.compliance_many(meshes)
        dc = topo.sensitivity_many(meshes)
        for b, m in enumerate(meshes):
            assert c[b] == m.compliance()
            assert np.array_equal(dc[b], m.sensitivity())
        with pytest.raises(RuntimeError):
            topo.sensitivity_many(meshes, np.empty((nb, nx * ny * nz + 1), np.float64))
    finally:
        for m in meshes:
            m.close()
    group = topo.create_batch(nb, nx, ny, nz)
    try:
        bad = rhos.copy()
        bad[1, 5] = np.nan  # design 1 gets no density; the others do
        with pytest.raises(RuntimeError):
            topo.set_density_many(group, bad)
        with pytest.raises(RuntimeError):
            group[1].solve()
        assert group[0].solve().status == 0
    finally:
        for m in group:
            m.close()


@pytest.mark.parametrize("precision", [1, 0])  # FP32 Jacobi-PCG + FP64 refinement; plain FP64
@pytest.mark.parametrize("nx,ny,nz,bc,load", [
    (40, 12, 10, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (33, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
])
def test_batched_jacobi_matches_single_solves_and_the_oracle(topo, precision, nx, ny, nz, bc,
                                                             load):
    """Jacobi-preconditioned solves of a whole mesh group run as one batch
    (design 0 launches every kernel, the others none) and give each design's
    single-solve result; the FP64 batch also after design 0 had solved alone
    in FP64 with vectors of its own (they move into the group's FP64 arena)."""
    opts = topo.default_opts(precision=precision, precond=topo.PRECOND_JACOBI, rtol=1e-10)
    nb = 3
    rhos = [I.density_cone_smoothed(nx, ny, nz, 90 + b) for b in range(nb)]
    meshes = topo.create_batch(nb, nx, ny, nz, bc, load)
    try:
        for m, r in zip(meshes, rhos):
            m.set_density(r)
        if precision == 0:  # design 0 first alone: its own FP64 vectors and graphs
            meshes[0].solve(opts)
            u_first = meshes[0].displacement()
        for m in meshes:
            m.profile_read(reset=True)
        infos = topo.solve_many(meshes, opts)
        launches = [m.profile_read(reset=True)[2] for m in meshes]
        res = [(m.displacement(), m.compliance(), m.sensitivity()) for m in meshes]
    finally:
        for m in meshes:
            m.close()
    assert launches[0] > 0 and launches[1] == 0 and launches[2] == 0
    for b in range(nb):
        u, c, dc = res[b]
        u1, c1, dc1, info1 = _alone(topo, nx, ny, nz, bc, load, rhos[b], opts)
        assert infos[b].status == 0 and infos[b].rel_residual <= 1e-10
        assert _rel(u, u1) <= 1e-8
        assert c == pytest.approx(c1, rel=1e-9)
        assert np.abs(dc - dc1).max() <= 1e-7 * np.abs(dc1).max()
    if precision == 0:
        assert _rel(res[0][0], u_first) <= 1e-8
    P = fem.Problem(nx, ny, nz, bc, load, rhos[1])
    assert _rel(res[1][0], P.solve()) <= 1e-8
