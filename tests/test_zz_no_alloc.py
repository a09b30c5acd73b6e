"""topo_sensitivity_noalloc: the entry point for callers that cannot allocate
GPU memory (their own allocator owns the device memory, or the budget is
fixed up front).  Its results must
match the mesh-based entry points (topo_sensitivity, topo_compliance_energy)
on the same displacement, on two calls in a row (the second call reuses the
shared scratch array left behind by the first)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("case", [
    (24, 12, 12, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM),
    (33, 10, 12, I.BC_MBB, I.LOAD_EDGE_X0_TOP),
])
def test_noalloc_matches_mesh_entry_points_twice(topo, case):
    import torch
    nx, ny, nz, bc, load = case
    rho = I.density_uniform(nx, ny, nz, 0.01, 1.0, 31)
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        m.set_density(rho)
        m.solve(topo.default_opts())
        u = m.displacement()
        dc_ref = m.sensitivity()
        c_ref = m.compliance_energy()
    u_d = torch.from_numpy(u).cuda()
    rho_d = torch.from_numpy(rho).cuda()
    for _ in range(2):
        dc_d = torch.full((nx * ny * nz,), float("nan"), dtype=torch.float64, device="cuda")
        c_d = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        topo.sensitivity_noalloc(nx, ny, nz, u_d, rho_d, dc_d, c_d)
        torch.cuda.synchronize()
        dc = dc_d.cpu().numpy()
        c = float(c_d.item())
        # the tolerances of the parity tests: dc to 1e-6 of its max-norm, c to 1e-9
        assert np.abs(dc - dc_ref).max() <= 1e-6 * np.abs(dc_ref).max()
        assert abs(c - c_ref) <= 1e-9 * abs(c_ref)


def test_noalloc_rejects_grids_beyond_its_scratch(topo):
    import ctypes
    import torch
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    tiny32 = torch.zeros(8, dtype=torch.float32, device="cuda")
    # through the C ABI itself: 256 * 256 * 129 elements > 8,388,608 is
    # refused before anything is enqueued (the pointers are never touched)
    p = [ctypes.c_void_p(t.data_ptr()) for t in (tiny, tiny32, tiny, tiny)]
    st = topo.lib().topo_sensitivity_noalloc(256, 256, 129, None, *p, None)
    assert st == topo.ERR_INVALID
    # the binding refuses arrays that do not fit the grid, before the call
    with pytest.raises(ValueError):
        topo.sensitivity_noalloc(4, 2, 2, tiny, tiny32, tiny, tiny)
