"""Pins of the SIMP-update oracle (sensitivity filter Eq. (4), OC update)."""
import numpy as np
import pytest

from oracle import simp


def test_filter_weights_closed_form_R2():
    w = dict(simp.filter_weights(2.0))
    assert len(w) == 27  # |d| < 2 keeps the 3x3x3 block; |d| = 2 has weight 0
    assert w[(0, 0, 0)] == 2.0
    assert all(abs(w[d] - 1.0) < 1e-15 for d in [(1, 0, 0), (0, -1, 0), (0, 0, 1)])
    assert abs(w[(1, 1, 0)] - (2 - np.sqrt(2))) < 1e-15
    assert abs(w[(-1, 1, 1)] - (2 - np.sqrt(3))) < 1e-15


def _brute(nx, ny, nz, rho, dc, R, guard=1e-3):
    """Eq. (4) by brute force over all element pairs and centroid distances."""
    n = nx * ny * nz
    cen = np.array([[i + 0.5, j + 0.5, k + 0.5] for k in range(nz) for j in range(ny)
                    for i in range(nx)])
    out = np.zeros(n)
    for e in range(n):
        num = den = 0.0
        for i in range(n):
            H = max(0.0, R - np.linalg.norm(cen[e] - cen[i]))
            num += rho[i] * H * dc[i]
            den += H
        out[e] = num / (max(rho[e], guard) * den)
    return out


@pytest.mark.parametrize("R", [2.0, 1.5, 2.6])
def test_filter_matches_brute_force(R):
    nx, ny, nz = 5, 4, 3
    g = np.random.default_rng(0)
    rho = g.uniform(0.01, 1, nx * ny * nz)
    dc = -g.uniform(0, 3, nx * ny * nz)
    got = simp.sensitivity_filter(nx, ny, nz, rho, dc, R)
    assert np.allclose(got, _brute(nx, ny, nz, rho, dc, R), rtol=1e-13, atol=0)


def test_filter_normalisation_and_density_weighting():
    nx, ny, nz = 6, 5, 4
    n = nx * ny * nz
    # constant rho and dc: unchanged
    out = simp.sensitivity_filter(nx, ny, nz, np.full(n, 0.4), np.full(n, -2.0))
    assert np.allclose(out, -2.0, rtol=1e-14)
    # rho_i dc_i = c everywhere: the filtered value is exactly c / rho_e
    rho = np.random.default_rng(1).uniform(0.1, 1, n)
    out = simp.sensitivity_filter(nx, ny, nz, rho, -3.0 / rho)
    assert np.allclose(out, -3.0 / rho, rtol=1e-13)


def test_oc_volume_bounds_and_moves():
    g = np.random.default_rng(2)
    rho = g.uniform(0.001, 1, 500)
    dcf = -g.uniform(0.0, 5.0, 500)
    new, lam = simp.oc_update(rho, dcf, 0.4)
    assert abs(new.mean() - 0.4) < 1e-10
    assert new.min() >= 1e-3 - 1e-15 and new.max() <= 1.0
    assert np.all(np.abs(new - rho) <= 0.2 + 1e-15)
    # a larger |dc| never gives a smaller update (monotone in the stimulus)
    new2, _ = simp.oc_update(rho, dcf * np.where(np.arange(500) == 7, 2.0, 1.0), 0.4)
    assert new2[7] >= new[7] - 1e-12


def test_oc_closed_form_lambda_without_clipping():
    """With no bound or move limit active, sum rho (b/lam)^eta = V gives
    lam = (sum rho b^eta / V)^(1/eta) exactly."""
    g = np.random.default_rng(3)
    rho = g.uniform(0.4, 0.6, 200)
    b = g.uniform(0.9, 1.1, 200)
    V = rho.sum()
    lam_exact = (np.sum(rho * np.sqrt(b)) / V) ** 2
    new, lam = simp.oc_update(rho, -b, V / rho.size)
    assert abs(lam / lam_exact - 1) < 1e-11
    assert np.allclose(new, rho * np.sqrt(b / lam_exact), rtol=1e-11)


def test_oc_fixed_point_uniform():
    rho = np.full(64, 0.3)
    new, _ = simp.oc_update(rho, np.full(64, -1.7), 0.3)
    assert np.allclose(new, 0.3, rtol=1e-12)
