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


def _brute_distance(p, tri, n=401):
    """min over a fine barycentric lattice of the triangle (brute force)."""
    s = np.linspace(0, 1, n)
    L1, L2 = np.meshgrid(s, s)
    keep = (L1 + L2) <= 1.0
    lam = np.stack([L1[keep], L2[keep], 1 - L1[keep] - L2[keep]], 1)
    pts = lam @ tri
    return np.min(np.linalg.norm(p[:, None, :] - pts[None], axis=2), axis=1)


def test_closest_many_closed_forms_face_edge_vertex():
    """The broadcast form of Eq. (28)/(29) on the unit right triangle in z = 0,
    at points whose nearest feature is the face, each edge or each vertex:
    the distances are the closed forms (and independent of triangle order)."""
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    p = np.array([
        [0.2, 0.3, 0.7],     # above the face: |z|
        [0.25, 0.25, -1.5],  # below the face
        [0.5, -0.4, 0.3],    # nearest the edge y = 0: sqrt(0.4^2 + 0.3^2)
        [-0.6, 0.5, 0.0],    # nearest the edge x = 0, in plane: 0.6
        [0.8, 0.8, 0.2],     # nearest the hypotenuse x + y = 1 at (0.5, 0.5, 0)
        [-0.3, -0.4, 1.2],   # nearest vertex (0, 0, 0)
        [1.5, -0.2, 0.0],    # nearest vertex (1, 0, 0)
        [-0.1, 1.9, -0.3],   # nearest vertex (0, 1, 0)
    ])
    want = np.array([0.7, 1.5, 0.5, 0.6, np.sqrt(2 * 0.3 ** 2 + 0.2 ** 2),
                     np.sqrt(0.09 + 0.16 + 1.44), np.sqrt(0.25 + 0.04),
                     np.sqrt(0.01 + 0.81 + 0.09)])
    for order in ([0, 1, 2], [2, 0, 1], [1, 0, 2]):
        d = T._closest_many(p, tri[order][None])[:, 0]
        assert np.allclose(d, want, atol=1e-14, rtol=0)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_closest_many_against_sampling_many_triangles(seed):
    """Every (point, triangle) pair of the broadcast form against brute-force
    sampling of each triangle, with triangles of every shape: general, thin,
    collinear (degenerate) and all three vertices equal (a point)."""
    g = np.random.default_rng(100 + seed)
    tris = g.normal(size=(6, 3, 3))
    tris[1, 2] = tris[1, 0] + 0.02 * g.normal(size=3) + 0.5 * (tris[1, 1] - tris[1, 0])  # thin
    tris[2, 2] = tris[2, 0] + 0.3 * (tris[2, 1] - tris[2, 0])                            # collinear
    tris[3, 1] = tris[3, 0]
    tris[3, 2] = tris[3, 0]                                                                # a point
    p = g.normal(size=(50, 3)) * 2
    # points just above the face, just off an edge and just off a vertex of tris[0]
    a, b, c = tris[0]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    p[:3] = [(a + b + c) / 3 + 0.3 * n, (a + b) / 2 + 0.4 * ((a + b) / 2 - c), a + 0.5 * (a - (b + c) / 2)]
    d = T._closest_many(p, tris)
    assert d.shape == (len(p), len(tris))
    for m in range(len(tris)):
        brute = _brute_distance(p, tris[m])
        edge = max(np.linalg.norm(tris[m, 0] - tris[m, 1]), np.linalg.norm(tris[m, 1] - tris[m, 2]),
                   np.linalg.norm(tris[m, 2] - tris[m, 0]))
        assert np.all(d[:, m] <= brute + 1e-12)
        assert np.all(d[:, m] >= brute - 2 * edge / 400 - 1e-12)
        # the scalar form of the same rule agrees exactly in case
        assert np.allclose(d[:, m], T.closest_point_distance(p, tris[m]), atol=1e-13, rtol=0)
    # the point triangle is the distance to its vertex
    assert np.allclose(d[:, 3], np.linalg.norm(p - tris[3, 0], axis=1), atol=1e-13)


def test_triangle_set_comparison_ignores_order_but_not_geometry():
    """The order-free comparison the device parity tests use: a permuted soup
    with rotated vertex orders matches; a moved vertex does not."""
    from tests.geometry_compare import assert_same_triangle_set
    n = 10
    X = T._node_xyz(n, n, n)
    f = np.linalg.norm(X - np.array([4.9, 5.2, 5.1]), axis=1) - 3.3
    tris = T.iso_surface(f, n, n, n, 0.0, inside_above=False)
    g = np.random.default_rng(5)
    perm = tris[g.permutation(len(tris))]
    perm = np.stack([np.roll(t, g.integers(3), axis=0) for t in perm])
    assert_same_triangle_set(perm, tris)
    bad = perm.copy()
    bad[7, 1] += 1e-6
    with pytest.raises(AssertionError):
        assert_same_triangle_set(bad, tris)
    # a duplicated triangle in place of another is not the same set
    dup = perm.copy()
    dup[3] = dup[4]
    with pytest.raises(AssertionError):
        assert_same_triangle_set(dup, tris)
