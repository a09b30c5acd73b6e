"""The continuous-batching solve server: every request gives the same result
alone and in the mix (bitwise: all reductions are in a fixed order and each
design's sequence of warm-started solves is the same), admission never
exceeds the memory budget, and requests that arrive while others are on the
GPU are admitted and finish."""
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


def _alone(topo, r, steps):
    """The request's solves on its own mesh, one after the other (in the
    multigrid's throughput form, which the server uses for its designs)."""
    out = []
    with topo.Mesh(r.nx, r.ny, r.nz, r.bc, r.load) as m:
        m.set_throughput_mode(True)
        rho = r.rho0
        for s in range(steps):
            if s:
                rho = I.perturb(rho, r.factor(s))
            m.set_density(rho)
            info = m.solve(topo.default_opts(warm_start=1 if s else 0))
            out.append((info.iters, m.compliance()))
        u = m.displacement()
        dc = m.sensitivity()
    return out, u, dc


def test_server_same_alone_and_in_the_mix(topo):
    steps = 3
    reqs = I.serving_stream(n_requests=6, n_steps=steps, rate=0.0, max_ny=16, seed=77)
    alone = {r.rid: _alone(topo, r, steps) for r in reqs}
    fp = [topo.footprint_bytes(r.nx, r.ny, r.nz) for r in reqs]
    budget = int(max(fp) * 2.5)  # not everyone fits at once: admission must queue
    srv = topo.Server(budget, max_active=8)
    try:
        design, state, got = {}, {}, {r.rid: [] for r in reqs}
        first, rest = reqs[:3], reqs[3:]
        for r in first:
            d = srv.open(r.nx, r.ny, r.nz, r.bc, r.load)
            srv.submit(d, r.rho0)
            design[d], state[d] = r, (0, r.rho0)
        finished = 0
        late_admitted = False
        while finished < len(reqs):
            for res in srv.poll(wait=True):
                r = design[res.design]
                step, rho = state[res.design]
                assert res.status == 0 and res.rel_residual <= 1e-8
                got[r.rid].append((res.iters, res.compliance))
                if rest and not late_admitted:  # arrivals while others are on the GPU
                    for r2 in rest:
                        d2 = srv.open(r2.nx, r2.ny, r2.nz, r2.bc, r2.load)
                        srv.submit(d2, r2.rho0)
                        design[d2], state[d2] = r2, (0, r2.rho0)
                    late_admitted = True
                step += 1
                if step < steps:
                    rho = I.perturb(rho, r.factor(step))
                    srv.submit(res.design, rho)
                    state[res.design] = (step, rho)
                else:
                    a_steps, a_u, a_dc = alone[r.rid]
                    assert np.array_equal(srv.displacement(res.design), a_u)
                    assert np.array_equal(srv.sensitivity(res.design), a_dc)
                    srv.retire(res.design)
                    finished += 1
            st = srv.stats()
            assert st["bytes_in_use"] <= budget
        assert srv.stats()["peak_bytes"] <= budget
        for r in reqs:
            assert got[r.rid] == alone[r.rid][0], r.rid
    finally:
        srv.close()


def test_server_results_match_oracle_and_reject_oversize(topo):
    r = I.serving_stream(n_requests=1, n_steps=1, rate=0.0, max_ny=12, seed=5)[0]
    P = fem.Problem(r.nx, r.ny, r.nz, r.bc, r.load, r.rho0)
    c_ref = P.compliance(P.solve())
    with topo.Server(2**34, max_active=2) as srv:
        d = srv.open(r.nx, r.ny, r.nz, r.bc, r.load)
        srv.submit(d, r.rho0)
        res = srv.poll(wait=True)
        assert len(res) == 1 and res[0].status == 0
        assert abs(res[0].compliance - c_ref) <= 1e-6 * c_ref
    with topo.Server(1 << 20, max_active=2) as srv:  # 1 MiB: nothing fits
        with pytest.raises(topo.TopoError) as e:
            srv.open(24, 12, 12, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM)
        assert e.value.status == topo.ERR_OOM


def test_server_many_concurrent_setups_match_alone(topo):
    """Two dozen designs admitted at once set up their multigrid hierarchies
    and solve concurrently on their own streams; every compliance equals the
    one computed alone (bitwise)."""
    reqs = I.serving_stream(n_requests=24, n_steps=1, rate=0.0, max_ny=20, seed=123)
    alone = {}
    for r in reqs:
        with topo.Mesh(r.nx, r.ny, r.nz, r.bc, r.load) as m:
            m.set_throughput_mode(True)  # the server's form of the hierarchy
            m.set_density(r.rho0)
            info = m.solve()
            alone[r.rid] = (info.iters, m.compliance())
    with topo.Server(1 << 36, max_active=64) as srv:
        ds = {}
        for r in reqs:
            d = srv.open(r.nx, r.ny, r.nz, r.bc, r.load)
            srv.submit(d, r.rho0)
            ds[d] = r.rid
        got = []
        while len(got) < len(reqs):
            got += srv.poll(wait=True)
    for res in got:
        assert res.status == 0, (ds[res.design], res.status)
        assert (res.iters, res.compliance) == alone[ds[res.design]]


def test_server_staggered_admission_matches_alone(topo):
    """Designs admitted one by one while others are mid-solve (at most four
    resident), over several re-solves each: every job succeeds and matches
    the design's solves alone.  (A setup step ordered on the wrong stream
    used to corrupt a newly admitted design in exactly this pattern.)"""
    steps = 3
    reqs = I.serving_stream(n_requests=16, n_steps=steps, rate=0.0, max_ny=24, seed=321)
    alone = {r.rid: _alone(topo, r, steps)[0] for r in reqs}
    with topo.Server(1 << 36, max_active=4) as srv:
        design, state = {}, {}
        queue = list(reqs)
        got = {r.rid: [] for r in reqs}

        def admit_one():
            r = queue.pop(0)
            d = srv.open(r.nx, r.ny, r.nz, r.bc, r.load)
            srv.submit(d, r.rho0)
            design[d], state[d] = r, (0, r.rho0)

        for _ in range(4):
            admit_one()
        finished = 0
        while finished < len(reqs):
            for res in srv.poll(wait=True):
                r = design[res.design]
                step, rho = state[res.design]
                assert res.status == 0, (r.rid, step, res.status, res.detail)
                got[r.rid].append((res.iters, res.compliance))
                if queue:
                    admit_one()  # a new design arrives while the others keep solving
                step += 1
                if step < steps:
                    rho = I.perturb(rho, r.factor(step))
                    srv.submit(res.design, rho)
                    state[res.design] = (step, rho)
                else:
                    srv.retire(res.design)
                    finished += 1
    for r in reqs:
        assert got[r.rid] == alone[r.rid], r.rid


def test_server_rejects_invalid_densities_per_job_and_recovers(topo):
    """A job whose densities hold a NaN or a value above 1 fails with
    TOPO_ERR_NAN, detail 1 (the density check, which the server reads with
    the solve's first scalars instead of waiting on the host), and the same
    design's next valid job solves as on a fresh mesh."""
    nx, ny, nz = 24, 12, 12
    rho = I.density_cone_smoothed(nx, ny, nz, 5)
    with topo.Mesh(nx, ny, nz) as m:
        m.set_throughput_mode(True)
        m.set_density(rho)
        m.solve(topo.default_opts())
        c_ref = m.compliance()
    srv = topo.Server(1 << 32, max_active=4)
    try:
        d = srv.open(nx, ny, nz, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM)
        bad_nan = rho.copy()
        bad_nan[17] = np.nan
        bad_big = rho.copy()
        bad_big[3] = 1.5
        for bad in (bad_nan, bad_big):
            srv.submit(d, bad)
            res = [r for r in srv.poll(wait=True)]
            assert len(res) == 1 and res[0].status == topo.ERR_NAN and res[0].detail == 1
        srv.submit(d, rho)
        res = [r for r in srv.poll(wait=True)]
        assert len(res) == 1 and res[0].status == 0
        assert res[0].compliance == pytest.approx(c_ref, rel=1e-8)
    finally:
        srv.close()


@pytest.mark.parametrize("nx,ny,nz,bc,load", [
    (24, 12, 12, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),   # coarsest 3x2x2 instead of 6x3x3
    (48, 24, 24, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
    (33, 9, 7, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
])
def test_throughput_form_matches_the_direct_oracle(topo, nx, ny, nz, bc, load):
    """The server's form of the multigrid hierarchy (coarse end in one kernel,
    coarsest inverse in one kernel) solves to the same true residual and
    matches the direct solution like the default form."""
    rho = I.density_cone_smoothed(nx, ny, nz, 31)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    u_ref = P.solve()
    opts = topo.default_opts(rtol=1e-10)
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_throughput_mode(True)
        m.set_density(rho)
        info = m.solve(opts)
        u, c = m.displacement(), m.compliance()
        m.set_throughput_mode(False)  # back to the default form: rebuilt, same answer
        info0 = m.solve(opts)
        u0 = m.displacement()
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    assert c == pytest.approx(P.compliance(u_ref), rel=1e-8)
    assert np.linalg.norm(u0 - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    assert info.iters <= 1.3 * info0.iters + 3
