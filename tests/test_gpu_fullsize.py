"""Full-size workloads the oracle cannot factor (1.8 M and 8.3 M nodes): the
oracle checks the GPU displacement with its own FP64 matrix-free operator
(oracle/fullsize.c, pinned to the assembled K) on every DOF: the true
relative residual over all free DOFs, the compliance identity, and every
element's sensitivity recomputed from u.  On the 192x96x96 cantilever the
autograd gradient is also checked against central finite differences of GPU
solves on 50 seeded elements."""
import numpy as np
import pytest

from oracle import fem
from oracle import fullsize as FS
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


def _check_solution(topo, w, m, u, info):
    g = fem.Grid(w.nx, w.ny, w.nz)
    rho = w.density()
    E = fem.simp_modulus(rho)
    k0 = fem.element_stiffness(1.0, 0.3)
    f = fem.load_vector(g, w.load)
    fixed = fem.fixed_dofs(g, w.bc)
    f[fixed] = 0.0
    # the oracle's own FP64 residual over every free DOF meets the target
    rel = FS.rel_residual(g, E, k0, f, fixed, u)
    assert rel <= 1.01e-8, rel
    c = m.compliance()
    assert abs(c - float(f @ u)) <= 1e-12 * c
    assert abs(m.compliance_energy() - c) <= 1e-7 * c
    # every element's sensitivity (Eq. (3)) from u by the oracle
    dc = m.sensitivity()
    ref = -3.0 * rho.astype(np.float64) ** 2 * (1 - 1e-9) * FS.element_energies(g, k0, u)
    # both FP64, different formulas: soft elements carry a cancellation floor ~1e-11 of max|dc|
    assert np.all(np.abs(dc - ref) <= 1e-8 * np.abs(ref) + 1e-9 * np.abs(ref).max())
    assert np.all(dc <= 0.0)
    return {"rel_residual_oracle": rel, "c": c}


def test_cantilever_voids_192x96x96_solution_and_fd_gradient(topo):
    import torch
    from paper_2605_04735_gb300.autograd import compliance
    w = I.WORKLOADS["cantilever_voids_192x96x96"]
    rho = w.density()
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load) as m:
        m.set_density(rho)
        info = m.solve()
        assert info.rel_residual <= 1e-8 and info.iters <= 200
        u = m.displacement()
        _check_solution(topo, w, m, u, info)
        # autograd backward at a tight solve, then central differences
        tight = topo.default_opts(rtol=1e-11, max_outer=20)
        rho_t = torch.from_numpy(rho).cuda().requires_grad_(True)
        c0 = compliance(rho_t, m, tight)
        c0.backward()
        grad = rho_t.grad.double().cpu().numpy()
        base = m.displacement()
        h = 1e-3
        for e in I.fd_elements(rho, 50, 3):
            vals = []
            steps = (h, -h) if rho[e] + h <= 1.0 else (-h, -2 * h)
            for s in steps:
                r2 = rho.copy()
                r2[e] = np.float32(rho[e] + s)
                m.set_density(r2)
                m.set_displacement(base)
                m.solve(topo.default_opts(rtol=1e-11, max_outer=20, warm_start=1))
                vals.append(m.compliance())
            if steps[0] > 0:
                ds = float(np.float32(rho[e] + h)) - float(np.float32(rho[e] - h))
                fd = (vals[0] - vals[1]) / ds
            else:  # one-sided second order at rho = 1
                fd = (3 * c0.item() - 4 * vals[0] + vals[1]) / (2 * h)
            g = grad[e]
            assert abs(fd - g) <= 2e-3 * abs(g) + 1e-6 * np.abs(grad).max(), (e, rho[e], fd, g)


def test_cantilever_voids_320x160x160_solution(topo):
    w = I.WORKLOADS["cantilever_voids_320x160x160"]
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load) as m:
        m.set_density(w.density())
        info = m.solve()
        assert info.rel_residual <= 1e-8 and info.iters <= 200
        _check_solution(topo, w, m, m.displacement(), info)
