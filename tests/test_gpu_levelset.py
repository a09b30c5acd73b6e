"""The ersatz-material state (level-set stage, Eqs. (7)-(10)) on the device
against the FP64 oracle, through the C ABI.

Tolerances as in test_gpu_parity: solves to a true FP64 relative residual of
1e-10 match the direct solution to 1e-8 (2-norm) and the compliance to 1e-8;
element moduli and volume are FP64 on both sides (1e-12); element energies of
the same u agree to FP64 rounding of the modal quadratic form (1e-10 of the
largest)."""
import numpy as np
import pytest

from oracle import levelset as L
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
    (24, 12, 12, I.BC_CANTILEVER, I.LOAD_EDGE_XL_BOTTOM, 6, 1.0),
    (33, 10, 12, I.BC_MBB, I.LOAD_EDGE_X0_TOP, 5, 1.5),
    (40, 20, 20, I.BC_CORNERS, I.LOAD_DISC_XL, 10, 1.0),
]


@pytest.mark.parametrize("nx,ny,nz,bc,load,nvoid,eta", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_ersatz_state_matches_oracle(topo, nx, ny, nz, bc, load, nvoid, eta, prec):
    eps0 = 1e-3
    phi = I.levelset_voids(nx, ny, nz, nvoid, seed=31 + nx)
    P = L.Problem(nx, ny, nz, bc, load, phi, eta, eps0)
    u_ref = P.solve()
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        vol = m.set_levelset(phi, eta=eta, eps0=eps0)
        info = m.solve(topo.default_opts(precision=prec, rtol=1e-10,
                                         precond=topo.PRECOND_JACOBI if prec == 0
                                         else topo.PRECOND_GMG))
        u = m.displacement()
        c = m.compliance()
        ce = m.compliance_energy()
        w = m.element_energy()
    assert vol == pytest.approx(L.volume(phi, nx, ny, nz, eta), rel=1e-12)
    assert info.rel_residual <= 1e-10
    assert _rel(u, u_ref) <= 1e-8
    assert c == pytest.approx(P.compliance(u_ref), rel=1e-8)
    assert ce == pytest.approx(c, rel=1e-8)
    w_ref = P.element_energies_unit(u)  # the same u on both sides
    assert np.abs(w - w_ref).max() <= 1e-10 * np.abs(w_ref).max()


def test_levelset_then_density_restores_simp_state(topo):
    """set_density after set_levelset gives exactly the SIMP state again."""
    nx, ny, nz = 20, 8, 8
    rho = I.density_uniform(nx, ny, nz, 0.1, 1.0, 3)
    phi = I.levelset_voids(nx, ny, nz, 3, seed=5)
    with topo.Mesh(nx, ny, nz) as m:
        m.set_density(rho)
        m.solve(topo.default_opts(rtol=1e-10))
        c0 = m.compliance()
        m.set_levelset(phi)
        m.solve(topo.default_opts(rtol=1e-10))
        c1 = m.compliance()
        m.set_density(rho)
        m.solve(topo.default_opts(rtol=1e-10))
        c2 = m.compliance()
    assert c1 != pytest.approx(c0, rel=1e-3)
    assert c2 == pytest.approx(c0, rel=1e-9)


def test_levelset_rejects_bad_input(topo):
    nx, ny, nz = 6, 3, 3
    with topo.Mesh(nx, ny, nz) as m:
        phi = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
        with pytest.raises(RuntimeError):
            m.set_levelset(phi[:-1])
        with pytest.raises(RuntimeError):
            m.set_levelset(phi, eta=0.0)
        phi[5] = np.nan
        with pytest.raises(RuntimeError):
            m.set_levelset(phi)
        with pytest.raises(RuntimeError):
            m.element_energy()  # no solve yet


# ---- shape derivatives, extension, evolution, reinitialisation -----------

def _ls_case(topo, nx=24, ny=10, nz=10, bc=I.BC_CANTILEVER, load=I.LOAD_EDGE_XL_BOTTOM,
             eta=1.5):
    phi = I.levelset_voids(nx, ny, nz, 5, seed=77)
    m = topo.Mesh(nx, ny, nz, bc, load)
    m.set_levelset(phi, eta=eta, eps0=1e-3)
    m.solve(topo.default_opts(precision=0, precond=topo.PRECOND_JACOBI, rtol=1e-11))
    return m, phi


def test_shape_rhs_matches_oracle(topo):
    from oracle import fem
    nx, ny, nz, eta = 24, 10, 10, 1.5
    m, phi = _ls_case(topo, nx, ny, nz, eta=eta)
    with m:
        u = m.displacement()
        bJ, bV = m.shape_rhs()
    rJ, rV = L.shape_rhs(fem.Grid(nx, ny, nz), u, phi, eta)  # the same u on both sides
    assert np.abs(bJ - rJ).max() <= 1e-12 * np.abs(rJ).max()
    assert np.abs(bV - rV).max() <= 1e-12 * np.abs(rV).max()
    assert np.count_nonzero(rV) > 0


@pytest.mark.parametrize("ell", [0.0, 1.0, 3.0])
def test_hilbertian_solve_matches_oracle(topo, ell):
    from oracle import fem
    nx, ny, nz = 24, 10, 10
    m, phi = _ls_case(topo, nx, ny, nz)
    g = fem.Grid(nx, ny, nz)
    with m:
        u = m.displacement()
        rJ, rV = L.shape_rhs(g, u, phi, 1.5)
        b = rJ - 0.3 * rV                      # an augmented-Lagrangian style right-hand side
        v, iters = m.hilbertian_solve(b, ell, rtol=1e-12)
    dirichlet = L.loaded_nodes(g, I.LOAD_EDGE_XL_BOTTOM)
    ref = L.hilbertian_solve(g, ell, b, dirichlet)
    assert iters > 0
    assert np.all(v[dirichlet] == 0.0)
    assert np.linalg.norm(v - ref) <= 1e-9 * np.linalg.norm(ref)


def test_hj_evolution_and_reinit_match_oracle(topo):
    from oracle import fem
    nx, ny, nz = 20, 9, 8
    g = fem.Grid(nx, ny, nz)
    phi = I.levelset_voids(nx, ny, nz, 4, seed=3)
    v = np.sin(0.3 * np.arange(g.n_nodes)) * 0.7      # any smooth-ish speed of both signs
    with topo.Mesh(nx, ny, nz) as m:
        m.set_levelset(phi)
        dt = m.hj_evolve(v, gamma=0.5, steps=5)
        evolved = m.levelset()
        steps = m.reinit(gamma=0.5, tol=0.0, max_steps=24)
        reinit = m.levelset()
        vol = m.set_levelset(None, eta=1.0)           # moduli from the evolved level set
    assert dt == pytest.approx(L.cfl_dt(g, v, 0.5), rel=1e-15)
    ref = L.hj_evolve(g, phi, v, 0.5, 5)
    assert np.abs(evolved - ref).max() <= 1e-12 * np.abs(ref).max()
    ref2, s2 = L.reinit(g, ref, gamma=0.5, tol=0.0, max_steps=24)
    assert steps == s2 == 24
    assert np.abs(reinit - ref2).max() <= 1e-11 * np.abs(ref2).max()
    assert vol == pytest.approx(L.volume(reinit, nx, ny, nz, 1.0), rel=1e-12)


def test_reinit_stops_on_tolerance(topo):
    nx, ny, nz = 16, 6, 6
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    sdf = (i - 7.4).astype(np.float64).ravel()
    with topo.Mesh(nx, ny, nz) as m:
        m.set_levelset(sdf)
        steps = m.reinit(gamma=0.5, tol=1e-9, max_steps=200)
        out = m.levelset()
    assert steps <= 16                                # an exact distance is already steady
    inner = (i.ravel() > 0) & (i.ravel() < nx)
    assert np.abs(out[inner] - sdf[inner]).max() < 1e-9
