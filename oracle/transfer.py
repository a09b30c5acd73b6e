"""FP64 CPU oracle of the SIMP -> level-set geometry transfer (Sec. 3.2-3.4).

TEST INFRASTRUCTURE ONLY: imported by tests/ and never by the library.

  nodal_density(...)     local linear least squares of the element densities
                         at every node (Eqs. (25)-(27)), distance-weighted
                         averaging where the normal equations are singular
  iso_surface(...)       triangulated iso-surface of a nodal field, by linear
                         interpolation on the edges of the 6 tetrahedra of the
                         Kuhn split of every hexahedron (marching tetrahedra,
                         Sec. 3.3); returns (n_tri, 3, 3) vertex coordinates
  closest_point_distance(p, tri)  distance from points to one triangle by the
                         constrained projection of Eq. (28)
  surface_distance(...)  unsigned distance to a triangle soup, Eq. (29) (brute force)
  signed_distance(...)   Eq. (30): -d where rho_n >= rho_t, +d elsewhere

Grid conventions as in oracle.fem: unit edge h, node n = i + (nx+1)(j + (ny+1)k),
element e = i + nx(j + ny k), element centroid (i + 1/2, j + 1/2, k + 1/2) h.
"""
from __future__ import annotations

import itertools

import numpy as np


def _node_xyz(nx, ny, nz, h=1.0):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64) * h


def nodal_density(rho_e, nx: int, ny: int, nz: int, h: float = 1.0) -> np.ndarray:
    """rho_n for every node from the densities of the m elements sharing it:
    the linear polynomial [1 x^T] a fitted by the normal equations
    X^T X a = X^T rho (X rows [1 x_e^T], x_e the element centroids) and
    evaluated at the node, when m >= 4 and X^T X is non-singular (centroids
    not coplanar); otherwise (1 < m, singular) the average with weights
    1 / |x_n - x_e|; for m = 1 the element's own density."""
    rho = np.asarray(rho_e, dtype=np.float64).reshape(nz, ny, nx)
    out = np.empty((nz + 1) * (ny + 1) * (nx + 1))
    n = 0
    for k in range(nz + 1):
        for j in range(ny + 1):
            for i in range(nx + 1):
                xs, vals = [], []
                for dk, dj, di in itertools.product((-1, 0), repeat=3):
                    ei, ej, ek = i + di, j + dj, k + dk
                    if 0 <= ei < nx and 0 <= ej < ny and 0 <= ek < nz:
                        xs.append(((ei + 0.5) * h, (ej + 0.5) * h, (ek + 0.5) * h))
                        vals.append(rho[ek, ej, ei])
                xs = np.asarray(xs)
                vals = np.asarray(vals)
                xn = np.array([i * h, j * h, k * h])
                m = len(vals)
                value = None
                if m >= 4:
                    X = np.hstack([np.ones((m, 1)), xs])
                    A = X.T @ X
                    if np.linalg.matrix_rank(A) == 4:
                        a = np.linalg.solve(A, X.T @ vals)
                        value = float(np.concatenate([[1.0], xn]) @ a)
                if value is None:
                    if m == 1:
                        value = float(vals[0])
                    else:
                        w = 1.0 / np.linalg.norm(xs - xn, axis=1)
                        value = float(w @ vals / w.sum())
                out[n] = value
                n += 1
    return out


# Kuhn split of the unit cube: 6 tetrahedra along the diagonal from corner 0
# to corner 7 (corner c = dx + 2 dy + 4 dz), one per order of the axis steps;
# neighbouring cubes split their shared faces along the same diagonal.
KUHN_TETS = []
for perm in itertools.permutations((1, 2, 4)):
    a = perm[0]
    b = perm[0] + perm[1]
    KUHN_TETS.append((0, a, b, 7))

# the six edges of a tetrahedron (vertex index pairs)
TET_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def _tet_triangles(P, g):
    """Triangles of the zero set of the linear interpolant of g on the
    tetrahedron with vertices P (4, 3); inside means g >= 0.  One inside (or
    one outside) vertex gives one triangle over its three edges; two give the
    quadrilateral over the four mixed edges as two triangles."""
    ins = [g[v] >= 0.0 for v in range(4)]
    cnt = sum(ins)
    if cnt in (0, 4):
        return []

    def cut(a, b):
        t = g[a] / (g[a] - g[b])
        return P[a] + t * (P[b] - P[a])

    if cnt in (1, 3):
        lone = [v for v in range(4) if ins[v] == (cnt == 1)][0]
        others = [v for v in range(4) if v != lone]
        return [np.array([cut(lone, others[0]), cut(lone, others[1]), cut(lone, others[2])])]
    a, b = [v for v in range(4) if ins[v]]
    c, d = [v for v in range(4) if not ins[v]]
    q0, q1, q2, q3 = cut(a, c), cut(a, d), cut(b, d), cut(b, c)  # a cycle around the quad
    return [np.array([q0, q1, q2]), np.array([q0, q2, q3])]


def iso_surface(field, nx: int, ny: int, nz: int, level: float, inside_above: bool = True,
                h: float = 1.0) -> np.ndarray:
    """Triangle soup of {field = level} for a nodal field; `inside_above`: the
    material side is field >= level (densities), else field <= level (level
    sets).  Cells in element order, the tetrahedra in KUHN_TETS order, the
    triangles of a tetrahedron as in _tet_triangles."""
    f = np.asarray(field, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1)
    g = (f - level) if inside_above else (level - f)
    tris = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                corner_g = np.array([g[k + (c >> 2), j + ((c >> 1) & 1), i + (c & 1)]
                                     for c in range(8)])
                corner_x = np.array([[(i + (c & 1)) * h, (j + ((c >> 1) & 1)) * h,
                                      (k + (c >> 2)) * h] for c in range(8)])
                for tet in KUHN_TETS:
                    tris.extend(_tet_triangles(corner_x[list(tet)], corner_g[list(tet)]))
    return np.array(tris).reshape(-1, 3, 3)


def _segment_distance(p, a, b):
    ab = b - a
    L2 = float(ab @ ab)
    if L2 == 0.0:
        return np.linalg.norm(p - a, axis=-1)
    t = np.clip(((p - a) @ ab) / L2, 0.0, 1.0)
    return np.linalg.norm(p - (a + t[..., None] * ab), axis=-1)


def closest_point_distance(p, tri):
    """min over the triangle of |p - x(lambda)| subject to sum lambda = 1,
    lambda >= 0 (Eq. (28)): the orthogonal projection when its barycentric
    coordinates are all non-negative, else the nearest point of the three
    edges (the clamped segment projections).  p: (..., 3)."""
    p = np.asarray(p, dtype=np.float64)
    a, b, c = (np.asarray(v, dtype=np.float64) for v in tri)
    n = np.cross(b - a, c - a)
    nn = float(n @ n)
    d_edges = np.minimum(np.minimum(_segment_distance(p, a, b), _segment_distance(p, b, c)),
                         _segment_distance(p, c, a))
    if nn == 0.0:  # degenerate triangle: only its edges
        return d_edges
    s = ((p - a) @ n) / nn
    q = p - s[..., None] * n                           # projection onto the plane
    # barycentric coordinates of q from the sub-triangle areas
    l1 = (np.cross(c - b, q - b) @ n) / nn
    l2 = (np.cross(a - c, q - c) @ n) / nn
    l3 = 1.0 - l1 - l2
    inside = (l1 >= 0.0) & (l2 >= 0.0) & (l3 >= 0.0)
    return np.where(inside, np.abs(s) * np.sqrt(nn), d_edges)


def _closest_many(p, T):
    """closest_point_distance for points p (P, 3) and triangles T (M, 3, 3) at
    once, (P, M): the same projection / clamped-edge rule, broadcast."""
    a, b, c = T[:, 0], T[:, 1], T[:, 2]

    def seg(a, b):
        ab = b - a                                          # (M, 3)
        L2 = np.einsum("mk,mk->m", ab, ab)
        ap = p[:, None, :] - a[None]                        # (P, M, 3)
        with np.errstate(invalid="ignore", divide="ignore"):
            t = np.clip(np.einsum("pmk,mk->pm", ap, ab) / L2, 0.0, 1.0)
        t = np.where(L2 > 0.0, t, 0.0)
        q = ap - t[..., None] * ab[None]
        return np.sqrt(np.einsum("pmk,pmk->pm", q, q))

    de = np.minimum(np.minimum(seg(a, b), seg(b, c)), seg(c, a))
    n = np.cross(b - a, c - a)
    nn = np.einsum("mk,mk->m", n, n)
    ok = nn > 0.0
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.einsum("pmk,mk->pm", p[:, None, :] - a[None], n) / nn
        q = p[:, None, :] - s[..., None] * n[None]
        l1 = np.einsum("pmk,mk->pm", np.cross(c - b, q - b[None]), n) / nn
        l2 = np.einsum("pmk,mk->pm", np.cross(a - c, q - c[None]), n) / nn
    l3 = 1.0 - l1 - l2
    inside = ok & (l1 >= 0.0) & (l2 >= 0.0) & (l3 >= 0.0)
    return np.where(inside, np.abs(s) * np.sqrt(nn), de)


def surface_distance(points, tris, chunk: int = 256) -> np.ndarray:
    """Eq. (29): d(x) = min over the triangles of the closest-point distance
    (every point against every triangle, in chunks of triangles)."""
    points = np.asarray(points, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.float64).reshape(-1, 3, 3)
    d = np.full(points.shape[0], np.inf)
    for s in range(0, len(tris), chunk):
        np.minimum(d, _closest_many(points, tris[s:s + chunk]).min(axis=1), out=d)
    return d


def signed_distance(rho_n, d, rho_t: float = 0.5) -> np.ndarray:
    """Eq. (30): phi = -d where rho_n >= rho_t (material), +d elsewhere."""
    return np.where(np.asarray(rho_n) >= rho_t, -np.asarray(d), np.asarray(d))


def levelset_from_density(rho_e, nx, ny, nz, rho_t: float = 0.5, h: float = 1.0):
    """The whole transfer: nodal densities, iso-surface at rho_t, signed
    distance at the nodes.  Returns (phi, rho_n, triangles)."""
    rho_n = nodal_density(rho_e, nx, ny, nz, h)
    tris = iso_surface(rho_n, nx, ny, nz, rho_t, True, h)
    d = surface_distance(_node_xyz(nx, ny, nz, h), tris)
    return signed_distance(rho_n, d, rho_t), rho_n, tris
