"""The SIMP -> level-set geometry transfer on the device (Eqs. (25)-(30))
against the FP64 oracle, through the C ABI.

Tolerances: nodal densities and every triangle vertex are FP64 on both sides
with the same formulas (the least-squares solve differs in rounding only):
1e-12 absolute for densities in [0, 1], 1e-10 for coordinates and distances
in element units.  The triangle soups are compared as sets: the same count,
and a one-to-one matching of triangles whose vertex sets agree within the
tolerance (the emission order is the kernel's business)."""
import numpy as np
import pytest

from oracle import transfer as T
from tests.geometry_compare import assert_same_triangle_set
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


CASES = [
    (24, 12, 12, lambda: I.density_voids(24, 12, 12, 6, seed=11, rmin=2.0, rmax=4.0)),
    (17, 9, 7, lambda: I.density_uniform(17, 9, 7, 0.0, 1.0, 5)),
    (20, 10, 10, lambda: I.density_cone_smoothed(20, 10, 10, 9)),
]


@pytest.mark.parametrize("nx,ny,nz,make", CASES)
def test_nodal_density_matches_oracle(topo, nx, ny, nz, make):
    rho = make()
    with topo.Mesh(nx, ny, nz) as m:
        m.set_density(rho)
        rn = m.nodal_density()
    ref = T.nodal_density(rho, nx, ny, nz)
    assert np.abs(rn - ref).max() <= 1e-12


@pytest.mark.parametrize("nx,ny,nz,make", CASES)
def test_levelset_from_density_matches_oracle(topo, nx, ny, nz, make):
    rho = make()
    with topo.Mesh(nx, ny, nz) as m:
        m.set_density(rho)
        ntri = m.levelset_from_density(0.5)
        tris = m.surface()
        phi = m.levelset()
        vol = m.set_levelset(None, eta=1.0)
    ref_phi, ref_rn, ref_tris = T.levelset_from_density(rho, nx, ny, nz, 0.5)
    assert ntri == len(ref_tris) > 0
    assert_same_triangle_set(tris, ref_tris)
    assert np.abs(phi - ref_phi).max() <= 1e-10
    assert np.all((phi < 0) == (ref_rn >= 0.5))
    assert 0.0 < vol < nx * ny * nz


def test_paper_problem_simp_to_levelset_round_trip(topo):
    """A few SIMP iterations on the paper's 40x20x20 MBB, then the transfer and
    the surface of the resulting level set; both against the oracle."""
    nx, ny, nz, bc, load = I.PAPER_PROBLEMS["paper_mbb_40x20x20"]
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        rho0 = np.full(nx * ny * nz, 0.4, np.float32)
        topo.simp_optimize(m, rho0, topo.default_simp_opts(volfrac=0.4), max_iter=6, tol=0.0)
        rho = m.density()
        m.levelset_from_density(0.5)
        phi = m.levelset()
        n2 = m.extract_levelset_surface()
        tris2 = m.surface()
    # the surface in full, the distances at 600 seeded nodes (the oracle's
    # brute-force distance over all nodes would take minutes here)
    rn = T.nodal_density(rho, nx, ny, nz)
    ref_tris = T.iso_surface(rn, nx, ny, nz, 0.5)
    sample = np.random.default_rng(8).choice(len(phi), 600, replace=False)
    d = T.surface_distance(T._node_xyz(nx, ny, nz)[sample], ref_tris)
    ref_phi = T.signed_distance(rn[sample], d, 0.5)
    assert np.abs(phi[sample] - ref_phi).max() <= 1e-10
    ref2 = T.iso_surface(phi, nx, ny, nz, 0.0, inside_above=False)
    assert n2 == len(ref2)
    assert_same_triangle_set(tris2, ref2)


def test_transfer_without_a_boundary_is_rejected(topo):
    with topo.Mesh(8, 4, 4) as m:
        m.set_density(np.ones(8 * 4 * 4, np.float32))
        with pytest.raises(RuntimeError):
            m.levelset_from_density(0.5)
