"""Plain CPU oracle of the rest of a SIMP iteration: sensitivity filter and
Optimality Criteria update (TEST INFRASTRUCTURE ONLY; same rules as fem.py).

Sensitivity filter, Sec. 2.1.3, Eq. (4) (general-mesh form):
    dJ~/drho_e = sum_{i in N_e} (rho_i / V_i) H_ei dJ/drho_i
                 / ( (rho_e / V_e) sum_{i in N_e} H_ei ),
    H_ei = max(0, R - |x_e - x_i|),  N_e = elements with centroids within R.
Readings: uniform element volumes (structured grid), R = 2h as in Sec. 4.1,
and rho_e in the denominator taken as max(rho_e, 1e-3) (the paper gives no
guard against rho_e = 0; the OC update below never goes under 1e-3 anyway).

Optimality Criteria update (Sec. 2.1.2 names OC; Sec. 4.1 uses it with a
volume fraction V_f; the paper prints no move limit or damping): the
standard heuristic rho_new = clip(rho * (-dJ~/dV / lambda)^eta, lower, upper)
with lower = max(rho_min, rho - move), upper = min(1, rho + move), and
lambda found by bisection so that the volume constraint holds with
equality, sum_e rho_new_e V_e = V_f sum_e V_e (dV_e/drho_e = V_e, uniform).
Readings: move = 0.2, eta = 0.5, rho_min = 1e-3.
"""
from __future__ import annotations

import numpy as np


def filter_weights(radius: float):
    """(offset, weight) pairs of max(0, R - |d|) over integer offsets d."""
    reach = int(np.ceil(radius))
    out = []
    for dk in range(-reach, reach + 1):
        for dj in range(-reach, reach + 1):
            for di in range(-reach, reach + 1):
                w = radius - np.sqrt(di * di + dj * dj + dk * dk)
                if w > 0.0:
                    out.append(((di, dj, dk), w))
    return out


def sensitivity_filter(nx: int, ny: int, nz: int, rho: np.ndarray, dc: np.ndarray,
                       radius: float = 2.0, rho_guard: float = 1e-3) -> np.ndarray:
    """Eq. (4) on a structured grid (element units), element order x fastest."""
    r = np.asarray(rho, np.float64).reshape(nz, ny, nx)
    g = np.asarray(dc, np.float64).reshape(nz, ny, nx)
    num = np.zeros_like(g)
    den = np.zeros_like(g)
    for (di, dj, dk), w in filter_weights(radius):
        tk = slice(max(0, -dk), nz - max(0, dk))
        tj = slice(max(0, -dj), ny - max(0, dj))
        ti = slice(max(0, -di), nx - max(0, di))
        sk = slice(max(0, dk), nz - max(0, -dk))
        sj = slice(max(0, dj), ny - max(0, -dj))
        si = slice(max(0, di), nx - max(0, -di))
        num[tk, tj, ti] += w * r[sk, sj, si] * g[sk, sj, si]
        den[tk, tj, ti] += w
    out = num / (np.maximum(r, rho_guard) * den)
    return out.reshape(-1)


def oc_update(rho: np.ndarray, dcf: np.ndarray, volfrac: float, move: float = 0.2,
              eta: float = 0.5, rho_min: float = 1e-3, tol: float = 1e-13):
    """One OC step; returns (rho_new, lambda)."""
    r = np.asarray(rho, np.float64)
    b = np.maximum(-np.asarray(dcf, np.float64), 0.0)  # -dJ/drho / dV (dV = 1)
    lower = np.maximum(rho_min, r - move)
    upper = np.minimum(1.0, r + move)
    target = volfrac * r.size

    def new(lam):
        return np.clip(r * (b / lam) ** eta, lower, upper)

    lo, hi = 1e-40, 1e40
    while hi / lo > 1.0 + tol:
        mid = np.sqrt(lo * hi)  # bisection in log lambda
        if new(mid).sum() > target:
            lo = mid
        else:
            hi = mid
    lam = np.sqrt(lo * hi)
    return new(lam), lam
