"""The paper's SIMP stage on its own test problems, on the device.

Sec. 4.1: a 2 x 1 x 1 domain of 40 x 20 x 20 hex8 elements, E0 = 1,
nu = 0.3, p = 3, filter radius R = 2h, volume fraction 0.4, OC updates from
a uniform 0.4, stopped when the largest density change is at most the
threshold (0.5 % ... 8 % in the paper).  Problems: the corner-supported
cantilever with a disc load (Sec. 4.2) and the MBB beam with a strip support
and a half-disc load (Sec. 4.3).  Each SIMP iteration here is one state solve
to a true FP64 relative residual of 1e-8 (FP32 GMG-PCG + FP64 refinement,
warm-started), compliance, sensitivities (Eq. (3)), filter (Eq. (4)) and the
OC update, all in libtopo.so.

    python -m paper_2605_04735_gb300.simp_run [--tol 0.01] [--scale 1]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import topo


def run(name: str, tol: float, scale: int = 1, max_iter: int = 400):
    nx, ny, nz, bc, load = I.PAPER_PROBLEMS[name]
    nx, ny, nz = nx * scale, ny * scale, nz * scale
    import torch
    with topo.Mesh(nx, ny, nz, bc, load) as m:
        rho0 = np.full(nx * ny * nz, 0.4, np.float32)
        so = topo.default_simp_opts(volfrac=0.4, filter_radius=2.0)
        # warm-up of the kernels and graphs (not timed)
        topo.simp_optimize(m, rho0, so, max_iter=2, tol=0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = topo.simp_optimize(m, rho0, so, max_iter=max_iter, tol=tol)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rho = m.density()
    its = len(hist)
    return {"problem": name, "grid": [nx, ny, nz], "tol": tol, "iterations": its,
            "seconds": wall, "ms_per_iteration": 1e3 * wall / its,
            "compliance_first": hist[0][0], "compliance_last": hist[-1][0],
            "volume_last": hist[-1][1], "change_last": hist[-1][2],
            "solid_fraction_gt_0.5": float((rho > 0.5).mean())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tol", type=float, default=0.01)
    ap.add_argument("--scale", type=int, default=1)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    out = [run(n, args.tol, args.scale) for n in I.PAPER_PROBLEMS]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
