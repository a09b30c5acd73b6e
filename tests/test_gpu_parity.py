"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic, stated per test):
  * operator, FP64 kernel: relative 2-norm error <= 1e-13 (FP64 rounding of
    576-term sums); FP32 kernel: <= 2e-6 (FP32 rounding of x, E, k0 and the
    sums, random x so no cancellation beyond a factor ~10);
  * solves: the library stops on the true FP64 relative residual; at
    rtol = 1e-10 (FP64 itself attains only ~1e-11 on slender beams, the
    direct solver included) the displacement and compliance must match the direct
    Cholesky solution to <= 1e-8 relative (2-norm over all DOFs), and the
    sensitivities to <= 1e-6 relative to their max-norm.
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
    # (nx, ny, nz, bc, load): ragged sizes spanning several 32x8 thread tiles
    (40, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (33, 10, 12, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (5, 17, 3, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION),
    (1, 1, 1, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (2, 2, 1, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    # the paper's problems (Sec. 4.2 corner-supported cantilever, Sec. 4.3 MBB)
    (40, 20, 20, I.BC_CORNERS, I.LOAD_DISC_XL),
    (40, 20, 20, I.BC_MBB_STRIP, I.LOAD_HALFDISC_X0_TOP),
]


# grids with nx >= 65 run the column-paired FP32 kernel (63 x 7 node tiles):
# several x tiles with a ragged last one, every support type, tiles with and
# without fixed DOFs
PAIR_CASES = [
    (70, 12, 9, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (130, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (66, 17, 13, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION),
    (80, 12, 12, I.BC_CORNERS, I.LOAD_DISC_XL),
    (128, 16, 9, I.BC_MBB_STRIP, I.LOAD_HALFDISC_X0_TOP),
]
# modal (automatic form), node-centric gather, modal one column, modal paired,
# modal one column with the x tiles as one thread-block cluster
OPS = [0, 1, 2, 3, 5]


@pytest.mark.parametrize("case", CASES + PAIR_CASES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
@pytest.mark.parametrize("op", OPS)
def test_operator_matches_assembled_K(topo, case, prec, tol, op):
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 17)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    x = np.random.default_rng(5).normal(size=P.grid.n_dof)
    xm = x.copy()
    xm[P.fixed] = 0.0
    y_ref = P.K @ xm
    y_ref[P.fixed] = 0.0
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_operator(op)
        m.set_density(rho)
        y = m.apply(x, precision=prec)
    assert _rel(y, y_ref) <= tol
    assert np.all(y[P.fixed] == 0.0)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("nx", [40, 70])
def test_operator_fp32_keeps_accuracy_under_rigid_translation(topo, op, nx):
    """The FP32 kernels subtract a reference displacement before the element
    arithmetic, so a large rigid translation added to x does not swamp K x."""
    ny, nz = 9, 7
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 19)
    P = fem.Problem(nx, ny, nz, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION, rho)
    g = P.grid
    X = g.node_ijk().astype(float)
    x = 0.01 * np.sin(X @ np.array([0.3, 0.5, 0.7]))[:, None] * np.ones((1, 3))
    x = x + np.array([1e3, -2e3, 5e2])  # rigid translation, 1e5 times the strain-carrying part
    x = x.reshape(-1)
    xm = x.copy()
    xm[P.fixed] = 0.0
    y_ref = P.K @ xm
    y_ref[P.fixed] = 0.0
    interior = np.ones(g.n_nodes, bool)
    ijk = g.node_ijk()
    interior &= (ijk[:, 0] > 1) & (ijk[:, 1] > 1) & (ijk[:, 2] > 1)  # away from the masked planes
    mask = np.repeat(interior, 3)
    with topo.Mesh(nx, ny, nz, I.BC_ROLLER_BOX, I.LOAD_FACE_XL_TRACTION) as m:
        m.set_operator(op)
        m.set_density(rho)
        y = m.apply(x, precision=1)
    # FP32 rounding of x itself (~6e-8 * 2e3) bounds what any FP32 kernel can reach
    assert _rel(y[mask], y_ref[mask]) <= 2e-2


def _solve_case(topo, nx, ny, nz, bc, load, rho, prec, rtol, **kw):
    kw.setdefault("precond", topo.PRECOND_JACOBI if prec == 0 else topo.PRECOND_GMG)
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_density(rho)
        info = m.solve(topo.default_opts(precision=prec, rtol=rtol, **kw))
        return (info, m.displacement(), m.compliance(), m.compliance_energy(), m.sensitivity())


SOLVERS = [(0, 0), (1, 0), (1, 1)]  # (precision, preconditioner): FP64 Jacobi, FP32 Jacobi, FP32 GMG


@pytest.mark.parametrize("prec,pc", SOLVERS)
@pytest.mark.parametrize("case", CASES)
def test_solve_matches_direct_oracle(topo, case, prec, pc):
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.05, 1.0, 23)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    u_ref = P.solve()
    c_ref = P.compliance(u_ref)
    dc_ref = P.sensitivity(u_ref)
    info, u, c, ce, dc = _solve_case(topo, nx, ny, nz, bc, load, rho, prec, 1e-10, precond=pc)
    assert info.rel_residual <= 1e-10
    assert _rel(u, u_ref) <= 1e-8
    assert abs(c - c_ref) <= 1e-8 * abs(c_ref)
    assert abs(ce - c) <= 1e-9 * abs(c)
    assert np.abs(dc - dc_ref).max() <= 1e-6 * np.abs(dc_ref).max()


def test_cantilever_24x12x12_all_paths(topo):
    """The small cantilever workload (uniform rho in [0.01, 1]): plain FP64
    and FP32+refinement both reach rtol 1e-8; at rtol 1e-10 both match the
    direct solve to 1e-8 (u, c) and 1e-6 (dc)."""
    w = I.WORKLOADS["cantilever_24x12x12"]
    rho = w.density()
    P = fem.Problem(w.nx, w.ny, w.nz, w.bc, w.load, rho)
    u_ref = P.solve()
    c_ref = P.compliance(u_ref)
    dc_ref = P.sensitivity(u_ref)
    for prec, pc in SOLVERS:
        info, u, c, ce, dc = _solve_case(topo, w.nx, w.ny, w.nz, w.bc, w.load, rho, prec, 1e-8,
                                         precond=pc)
        assert info.rel_residual <= 1e-8
        # the oracle's own FP64 residual of the GPU displacement
        assert P.rel_residual(u) <= 1.05e-8
        info, u, c, ce, dc = _solve_case(topo, w.nx, w.ny, w.nz, w.bc, w.load, rho, prec, 1e-10,
                                         precond=pc)
        assert _rel(u, u_ref) <= 1e-8
        assert abs(c - c_ref) <= 1e-8 * c_ref
        assert np.abs(dc - dc_ref).max() <= 1e-6 * np.abs(dc_ref).max()
        big = np.abs(dc_ref) > 1e-3 * np.abs(dc_ref).max()
        assert np.all(np.abs(dc - dc_ref)[big] <= 1e-6 * np.abs(dc_ref)[big])


def test_uniaxial_tension_closed_form(topo):
    nx, ny, nz, h, t = 6, 4, 3, 0.5, 1.7
    prm = topo.default_params(Emin=0.0, h=h, load=t)
    with topo.Mesh(nx, ny, nz, topo.BC_ROLLER_BOX, topo.LOAD_FACE_XL_TRACTION, prm) as m:
        m.set_density(np.ones(nx * ny * nz, np.float32))
        m.solve(topo.default_opts(precision=1, rtol=1e-12))
        u = m.displacement().reshape(-1, 3)
        c = m.compliance()
    g = fem.Grid(nx, ny, nz, h)
    X = g.node_ijk() * h
    exact = np.stack([t * X[:, 0], -0.3 * t * X[:, 1], -0.3 * t * X[:, 2]], axis=1)
    assert np.abs(u - exact).max() <= 1e-11 * np.abs(exact).max()
    V = nx * ny * nz * h ** 3
    assert abs(c - t * t * V) <= 1e-11 * t * t * V


@pytest.mark.parametrize("pc", [0, 1])
def test_mbb_96x32x32_full_size_properties(topo, pc):
    """Full-size MBB workload in the bench's configuration: the oracle
    assembles K in FP64 and checks the GPU displacement's true residual, the
    energy identity, and sampled sensitivities computed one by one."""
    w = I.WORKLOADS["mbb_96x32x32"]
    rho = w.density()
    P = fem.Problem(w.nx, w.ny, w.nz, w.bc, w.load, rho)
    info, u, c, ce, dc = _solve_case(topo, w.nx, w.ny, w.nz, w.bc, w.load, rho, 1, 1e-8,
                                     precond=pc)
    assert info.rel_residual <= 1e-8
    if pc == 1:
        assert info.iters <= 200  # multigrid keeps CG short
    assert P.rel_residual(u) <= 1.05e-8
    assert abs(c - P.compliance(u)) <= 1e-12 * c
    assert abs(c - float(u @ (P.K @ u))) <= 1e-7 * c
    assert abs(ce - c) <= 1e-7 * c
    elems = I.fd_elements(rho, 50, 99)
    en = fem.element_energies_at(P.grid, u, P.k0, elems)
    ref = -3.0 * rho[elems].astype(np.float64) ** 2 * (1 - 1e-9) * en
    # FP64 on both sides, different summation order: 1e-8 relative + 1e-12 of the largest
    # both FP64, different formulas: soft elements carry a cancellation floor ~1e-11 of max|dc|
    assert np.all(np.abs(dc[elems] - ref) <= 1e-8 * np.abs(ref) + 1e-9 * np.abs(ref).max())


def test_deterministic_bitwise(topo):
    w = I.WORKLOADS["cantilever_24x12x12"]
    rho = w.density()
    a = _solve_case(topo, w.nx, w.ny, w.nz, w.bc, w.load, rho, 1, 1e-8)
    b = _solve_case(topo, w.nx, w.ny, w.nz, w.bc, w.load, rho, 1, 1e-8)
    assert a[0].iters == b[0].iters
    assert np.array_equal(a[1], b[1]) and a[2] == b[2] and np.array_equal(a[4], b[4])


def test_warm_start_after_density_step(topo):
    w = I.WORKLOADS["cantilever_24x12x12"]
    rho = w.density()
    rho2 = I.perturb(rho, I.rng(3).uniform(0.95, 1.05, rho.size))
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load) as m:
        m.set_density(rho)
        m.solve(topo.default_opts(precision=1))
        m.set_density(rho2)
        warm = m.solve(topo.default_opts(precision=1, warm_start=1))
        u_warm = m.displacement()
    cold, u_cold = None, None
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load) as m:
        m.set_density(rho2)
        cold = m.solve(topo.default_opts(precision=1))
        u_cold = m.displacement()
    assert warm.rel_residual <= 1e-8 and cold.rel_residual <= 1e-8
    assert warm.iters < cold.iters
    P = fem.Problem(w.nx, w.ny, w.nz, w.bc, w.load, rho2)
    assert P.rel_residual(u_warm) <= 1.05e-8
    assert _rel(u_warm, u_cold) < 1e-4


def test_errors_are_reported_not_raised_in_the_library(topo):
    with pytest.raises(topo.TopoError) as e:
        topo.Mesh(4, 3, 2, topo.BC_MBB, topo.LOAD_EDGE_X0_TOP)   # odd ny for MBB
    assert e.value.status == topo.ERR_INVALID
    with topo.Mesh(4, 2, 2) as m:
        with pytest.raises(topo.TopoError) as e:
            m.solve()
        assert e.value.status == topo.ERR_NO_DENSITY
        with pytest.raises(topo.TopoError) as e:
            m.compliance()
        assert e.value.status == topo.ERR_NOT_SOLVED
        with pytest.raises(topo.TopoError) as e:
            m.set_density(np.ones(5, np.float32))
        assert e.value.status == topo.ERR_INVALID
        bad = np.ones(16, np.float32)
        bad[3] = np.nan
        with pytest.raises(topo.TopoError) as e:
            m.set_density(bad)
        assert e.value.status == topo.ERR_NAN
        bad[3] = 1.5
        with pytest.raises(topo.TopoError) as e:
            m.set_density(bad)
        assert e.value.status == topo.ERR_NAN
        m.set_density(np.full(16, 0.5, np.float32))
        info = m.solve(topo.default_opts(max_iter=1, rtol=1e-14, precond=0), check=False)
        assert info.status == topo.ERR_NOT_CONVERGED and info.iters <= 1
        info = m.solve(topo.default_opts(precision=0, precond=1), check=False)
        assert info.status == topo.ERR_INVALID
        info = m.solve(topo.default_opts(precision=7), check=False)
        assert info.status == topo.ERR_INVALID


def test_autograd_backward_matches_oracle_gradient_and_fd(topo):
    """Compliance as a torch.autograd.Function: the backward (the adjoint
    sensitivity kernel, no second solve) matches the oracle's gradient and
    central finite differences of the oracle's compliance."""
    import torch
    from paper_2605_04735_gb300.autograd import compliance
    nx, ny, nz = 6, 4, 4
    rho_np = I.density_uniform(nx, ny, nz, 0.2, 1.0, 41)
    rho = torch.from_numpy(rho_np).cuda().requires_grad_(True)
    with topo.Mesh(nx, ny, nz, topo.BC_CANTILEVER, topo.LOAD_EDGE_XL_BOTTOM) as m:
        c = compliance(rho, m, topo.default_opts(rtol=1e-11))
        c.backward()
    g = rho.grad.double().cpu().numpy()
    P = fem.Problem(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, rho_np)
    u = P.solve()
    assert abs(c.item() - P.compliance(u)) <= 1e-8 * P.compliance(u)
    ref = P.sensitivity(u)
    # rho.grad is float32: compare at float32 resolution
    assert np.abs(g - ref).max() <= 2e-6 * np.abs(ref).max()
    for e in (0, 17, 50, 95):
        cs = []
        for s in (1, -1):
            r2 = rho_np.astype(np.float64)
            r2[e] += s * 1e-4
            Q = fem.Problem(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, r2)
            cs.append(Q.compliance(Q.solve()))
        fd = (cs[0] - cs[1]) / 2e-4
        assert abs(fd - g[e]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(ref).max()


def test_stream_ordering_with_torch_default_stream(topo):
    """Device outputs are ordered before later work on the caller's stream
    (here torch's default stream), without a host synchronisation."""
    import torch
    w = I.WORKLOADS["cantilever_24x12x12"]
    rho = torch.from_numpy(w.density()).cuda()
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load) as m:
        m.set_density(rho)
        m.solve()
        dc = torch.zeros(w.n_elem, dtype=torch.float64, device="cuda")
        m.sensitivity(dc)
        s1 = float(dc.sum().item())  # torch reads dc on the default stream
        ref = m.sensitivity()
    assert abs(s1 - ref.sum()) <= 1e-12 * abs(ref.sum())


def test_solve_many_same_alone_and_in_the_mix(topo):
    """Designs of different sizes and BCs solved concurrently (one stream
    each, one host thread) give bitwise the same displacements, compliances
    and sensitivities as when each is solved alone (all reductions are in a
    fixed order), and each meets the FP64 residual target."""
    specs = [(24, 12, 12, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, 1),
             (32, 16, 16, I.BC_MBB, I.LOAD_EDGE_X0_TOP, 2),
             (40, 20, 20, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, 3),
             (16, 8, 8, I.BC_MBB, I.LOAD_EDGE_X0_TOP, 4)]
    alone = []
    for nx, ny, nz, bc, load, seed in specs:
        rho = I.density_cone_smoothed(nx, ny, nz, seed)
        with topo.Mesh(nx, ny, nz, bc, load) as m:
            m.set_density(rho)
            info = m.solve()
            alone.append((info.iters, m.displacement(), m.compliance(), m.sensitivity()))
    meshes = []
    for nx, ny, nz, bc, load, seed in specs:
        m = topo.Mesh(nx, ny, nz, bc, load)
        m.set_density(I.density_cone_smoothed(nx, ny, nz, seed))
        meshes.append(m)
    try:
        infos = topo.solve_many(meshes)
        for (it, u, c, dc), m, info in zip(alone, meshes, infos):
            assert info.status == 0 and info.rel_residual <= 1e-8
            assert info.iters == it
            assert np.array_equal(m.displacement(), u)
            assert m.compliance() == c
            assert np.array_equal(m.sensitivity(), dc)
    finally:
        for m in meshes:
            m.close()
    with pytest.raises(topo.TopoError):
        m2 = topo.Mesh(4, 2, 2)
        try:
            m2.set_density(np.full(16, 0.5, np.float32))
            topo.solve_many([m2, m2])
        finally:
            m2.close()
