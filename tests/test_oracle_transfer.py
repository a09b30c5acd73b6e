"""Pins of the geometry-transfer oracle (Eqs. (25)-(30)) against what the
definitions and the geometry fix, independent of the oracle's formulas."""
import numpy as np
import pytest

from oracle import transfer as T


def _centroids(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) + 0.5


def test_nodal_density_reproduces_linear_fields_inside_and_copies_corners():
    nx, ny, nz = 6, 5, 4
    a, b = np.array([0.05, -0.03, 0.08]), 0.4
    rho = _centroids(nx, ny, nz) @ a + b
    rn = T.nodal_density(rho, nx, ny, nz)
    X = T._node_xyz(nx, ny, nz)
    inner = np.all((X > 0) & (X < [nx, ny, nz]), axis=1)
    assert np.allclose(rn[inner], X[inner] @ a + b, atol=1e-13)
    # m = 1 at the 8 domain corners: the corner element's own density
    r3 = rho.reshape(nz, ny, nx)
    assert rn[0] == r3[0, 0, 0]
    assert rn[-1] == r3[-1, -1, -1]


def test_nodal_density_interior_is_the_mean_of_the_eight_on_a_uniform_grid():
    """The fitted plane passes through the mean of the data at the mean of the
    design points, and an interior node is the mean of its 8 centroids."""
    nx, ny, nz = 5, 4, 3
    rho = np.random.default_rng(2).uniform(0, 1, nx * ny * nz)
    rn = T.nodal_density(rho, nx, ny, nz).reshape(nz + 1, ny + 1, nx + 1)
    r3 = rho.reshape(nz, ny, nx)
    assert rn[1, 1, 1] == pytest.approx(r3[0:2, 0:2, 0:2].mean(), abs=1e-14)
    # a face node has 4 coplanar centroids (singular normal equations) at equal
    # distances: the distance-weighted average is their mean
    assert rn[0, 2, 2] == pytest.approx(r3[0, 1:3, 1:3].mean(), abs=1e-14)
    # an edge node: 2 elements
    assert rn[0, 0, 2] == pytest.approx(r3[0, 0, 1:3].mean(), abs=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_closest_point_distance_against_sampling(seed):
    g = np.random.default_rng(seed)
    tri = g.normal(size=(3, 3))
    if seed == 2:
        tri[2] = tri[0] + 0.5 * (tri[1] - tri[0])  # degenerate (collinear) triangle
    p = g.normal(size=(40, 3)) * 2
    d = T.closest_point_distance(p, tri)
    s = np.linspace(0, 1, 301)
    L1, L2 = np.meshgrid(s, s)
    keep = (L1 + L2) <= 1.0
    lam = np.stack([L1[keep], L2[keep], 1 - L1[keep] - L2[keep]], 1)
    pts = lam @ tri
    brute = np.min(np.linalg.norm(p[:, None, :] - pts[None], axis=2), axis=1)
    edge = max(np.linalg.norm(tri[0] - tri[1]), np.linalg.norm(tri[1] - tri[2]),
               np.linalg.norm(tri[2] - tri[0]))
    assert np.all(d <= brute + 1e-12)
    assert np.all(d >= brute - 2 * edge / 300)


def test_iso_surface_of_a_plane_lies_on_it_with_the_cross_section_area():
    nx, ny, nz = 7, 4, 3
    X = T._node_xyz(nx, ny, nz)
    tris = T.iso_surface(X[:, 0] - 3.3, nx, ny, nz, 0.0, inside_above=False)
    assert np.allclose(tris[:, :, 0], 3.3, atol=1e-14)
    area = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    assert area.sum() == pytest.approx(ny * nz, rel=1e-13)
    d = T.surface_distance(X, tris)
    assert np.allclose(d, np.abs(X[:, 0] - 3.3), atol=1e-13)


def test_iso_surface_of_a_ball_is_closed_and_close_to_the_sphere():
    n, r = 12, 3.7
    X = T._node_xyz(n, n, n)
    c = np.array([6.1, 5.8, 6.3])
    f = np.linalg.norm(X - c, axis=1) - r
    tris = T.iso_surface(f, n, n, n, 0.0, inside_above=False)
    # watertight: every edge is shared by exactly two triangles
    edges = {}
    for t in np.round(tris, 12):
        for a, b in ((0, 1), (1, 2), (2, 0)):
            key = tuple(sorted((tuple(t[a]), tuple(t[b]))))
            edges[key] = edges.get(key, 0) + 1
    counts = np.array(list(edges.values()))
    degenerate = sum(1 for k in edges if k[0] == k[1])
    assert degenerate == 0 and np.all(counts == 2)
    area = 0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1)
    assert area.sum() == pytest.approx(4 * np.pi * r * r, rel=0.05)
    # vertices on the sphere to interpolation accuracy; node distances close to |f|
    assert np.abs(np.linalg.norm(tris.reshape(-1, 3) - c, axis=1) - r).max() < 0.15
    d = T.surface_distance(X, tris)
    assert np.abs(d - np.abs(f)).max() < 0.15


def test_levelset_from_density_of_a_half_space():
    nx, ny, nz = 10, 3, 3
    rho = np.where(_centroids(nx, ny, nz)[:, 0] < 4.0, 1.0, 1e-3)
    phi, rn, tris = T.levelset_from_density(rho, nx, ny, nz)
    X = T._node_xyz(nx, ny, nz)
    # nodal densities: 1 for x < 4, 0.5005 (mean of 1 and 1e-3) at x = 4, 1e-3
    # beyond: the 0.5 crossing on the edge from x = 4 to x = 5 is at
    # t = 0.0005 / (0.5005 - 0.001), the iso-surface is that plane and phi = x - c
    c = 4.0 + 0.0005 / 0.4995
    assert np.allclose(tris[:, :, 0], c, atol=1e-12)
    assert np.allclose(phi, X[:, 0] - c, atol=1e-12)
    assert np.all((phi < 0) == (rn >= 0.5))
