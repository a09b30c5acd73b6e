"""The failure path of a bounded device-side wait, made to run out on
purpose without faulting or hanging anything: topo_debug_inject_timeout arms
one bounded wait (64 polls) on a barrier that nothing completes, inside the
next launch of the TMA-staged operator kernel; the kernel's own transfers
are untouched.  The timeout must reach topo_solve_info (status
TOPO_ERR_TIMEOUT, detail TOPO_FAIL_TIMEOUT), mark only the affected design of
a mesh group, and leave the mesh usable: the next solve gives the result an
untouched mesh gives."""
import numpy as np
import pytest

from paper_2605_04735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FAIL_TIMEOUT = 5


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


NX, NY, NZ = 40, 12, 10


def _reference(topo, rho, opts):
    with topo.Mesh(NX, NY, NZ, I.BC_MBB, I.LOAD_EDGE_X0_TOP) as m:
        m.set_density(rho)
        m.solve(opts)
        return m.displacement()


def test_timeout_reaches_the_solve_info_and_the_mesh_recovers(topo):
    opts = topo.default_opts()
    rho = I.density_cone_smoothed(NX, NY, NZ, 501)
    with topo.Mesh(NX, NY, NZ, I.BC_MBB, I.LOAD_EDGE_X0_TOP) as m:
        m.set_density(rho)
        m.debug_inject_timeout(1)
        info = m.solve(opts, check=False)
        assert info.status == topo.ERR_TIMEOUT and info.detail == FAIL_TIMEOUT
        with pytest.raises(topo.TopoError) as e:  # not solved: no compliance
            m.compliance()
        assert e.value.status == topo.ERR_NOT_SOLVED
        info = m.solve(opts)  # armed once only: this solve runs clean
        assert info.status == 0 and info.rel_residual <= 1e-8
        u = m.displacement()
    ref = _reference(topo, rho, opts)
    assert np.linalg.norm(u - ref) <= 1e-6 * np.linalg.norm(ref)


def test_timeout_in_a_mesh_group_marks_only_its_design(topo):
    opts = topo.default_opts()
    nb = 3
    rhos = [I.density_cone_smoothed(NX, NY, NZ, 510 + b) for b in range(nb)]
    group = topo.create_batch(nb, NX, NY, NZ, I.BC_MBB, I.LOAD_EDGE_X0_TOP, opts=opts)
    try:
        topo.set_density_many(group, np.stack(rhos))
        group[1].debug_inject_timeout(1)
        infos = topo.solve_many(group, opts, check=False)
        assert infos[1].status == topo.ERR_TIMEOUT and infos[1].detail == FAIL_TIMEOUT
        for b in (0, 2):
            assert infos[b].status == 0 and infos[b].rel_residual <= 1e-8
        first = [group[b].displacement() for b in (0, 2)]
        infos = topo.solve_many(group, opts)  # the group recovers as a whole
        assert all(i.status == 0 and i.rel_residual <= 1e-8 for i in infos)
        us = [m.displacement() for m in group]
    finally:
        for m in group:
            m.close()
    for b in range(nb):
        ref = _reference(topo, rhos[b], opts)
        assert np.linalg.norm(us[b] - ref) <= 1e-6 * np.linalg.norm(ref)
    for u, b in zip(first, (0, 2)):
        assert np.linalg.norm(u - us[b]) <= 1e-6 * np.linalg.norm(us[b])


def test_inject_timeout_rejects_other_counts(topo):
    with topo.Mesh(8, 4, 4) as m:
        for bad in (-1, 2):
            with pytest.raises(topo.TopoError):
                m.debug_inject_timeout(bad)
