"""The seeded input recipes: determinism, ranges and the stated weights."""
import numpy as np

from paper_2605_04735_gb300 import inputs as I


def test_seeded_fields_are_deterministic():
    a = I.density_cone_smoothed(8, 4, 4, 11)
    b = I.density_cone_smoothed(8, 4, 4, 11)
    c = I.density_cone_smoothed(8, 4, 4, 12)
    assert a.dtype == np.float32 and a.shape == (128,)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_cone_filter_weights_and_clip():
    # a constant field is a fixed point of any normalised filter
    raw = np.full((3, 4, 5), 0.37)
    assert np.allclose(raw.mean(), 0.37)
    rho = I.density_cone_smoothed(10, 6, 6, 3)
    assert rho.min() >= 1e-3 and rho.max() <= 1.0
    # interior value equals the hand-written stencil average of the raw draw
    raw = I.rng(3).uniform(0.0, 1.0, size=(6, 6, 10))
    k, j, i = 3, 2, 4
    w_face, w_edge = 0.5, 1.5 - np.sqrt(2.0)
    num, den = 1.5 * raw[k, j, i], 1.5
    for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        num += w_face * raw[k + d[2], j + d[1], i + d[0]]
        den += w_face
    for a in (-1, 1):
        for b in (-1, 1):
            for (di, dj, dk) in ((a, b, 0), (a, 0, b), (0, a, b)):
                num += w_edge * raw[k + dk, j + dj, i + di]
                den += w_edge
    assert abs(rho[i + 10 * (j + 6 * k)] - np.float32(num / den)) < 1e-7


def test_void_field_floor_and_binary_far_field():
    rho = I.density_voids(40, 20, 20, 6, 5)
    assert rho.min() >= np.float32(1e-3) and rho.max() == 1.0
    assert (rho == 1.0).mean() > 0.2 and (rho < 0.01).sum() > 0
    # the bounding-box shortcut matches the brute-force definition
    c, r = I.void_spheres(40, 20, 20, 6, 5)
    k, j, i = np.meshgrid(np.arange(20), np.arange(20), np.arange(40), indexing="ij")
    x = np.stack([i + 0.5, j + 0.5, k + 0.5], axis=-1)
    d = np.min(np.linalg.norm(x[..., None, :] - c, axis=-1) - r, axis=-1)
    brute = np.maximum(1e-3, 1.0 / (1.0 + np.exp(-8.0 * d))).reshape(-1).astype(np.float32)
    assert np.array_equal(rho, brute)


def test_workload_sizes():
    w = I.WORKLOADS["mbb_96x32x32"]
    assert (w.n_elem, w.n_nodes) == (98304, 105633)
    w = I.WORKLOADS["cantilever_voids_320x160x160"]
    assert (w.n_elem, w.n_nodes) == (8192000, 8320641)


def test_serving_stream_shapes():
    reqs = I.serving_stream(n_requests=6, n_steps=3, rate=2.0, max_ny=16)
    assert len(reqs) == 6
    assert all(r.nx == 2 * r.ny and r.nz == r.ny and r.ny % 4 == 0 for r in reqs)
    assert all(b.arrival > a.arrival for a, b in zip(reqs, reqs[1:]))
    f = reqs[0].factor(1)
    assert f.min() >= 0.95 and f.max() <= 1.05 and f.size == reqs[0].rho0.size
    p = I.perturb(reqs[0].rho0, f)
    assert p.dtype == np.float32 and p.min() >= np.float32(1e-3)
