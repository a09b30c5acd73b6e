"""Order-free comparison of triangle soups for the geometry-transfer parity
tests (the order in which a kernel emits triangles is not part of the result)."""
import numpy as np
from scipy.spatial import cKDTree


def assert_same_triangle_set(a, b, tol=1e-10):
    """a, b: (n, 3, 3) triangle soups.  Equal as sets of triangles, each a set
    of three vertices, within tol (independent of triangle and vertex order):
    every triangle of a is matched to a distinct triangle of b whose three
    vertices are a's three vertices within tol."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, 3, 3)
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3, 3)
    assert len(a) == len(b), (len(a), len(b))
    if len(a) == 0:
        return
    k = min(8, len(b))
    d, J = cKDTree(b.mean(axis=1)).query(a.mean(axis=1), k=k)
    d, J = d.reshape(len(a), k), J.reshape(len(a), k)
    used = np.zeros(len(b), dtype=bool)
    for t in range(len(a)):
        for dist, j in zip(d[t], J[t]):
            if dist > tol:
                break
            if used[j]:
                continue  # an identical triangle already took this one
            dv = np.linalg.norm(a[t][:, None, :] - b[j][None, :, :], axis=2)
            if dv.min(axis=1).max() <= tol and dv.min(axis=0).max() <= tol:
                used[j] = True
                break
        else:
            raise AssertionError(f"triangle {t} of the first soup has no match")
    assert used.all()
