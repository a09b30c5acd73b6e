"""Serving workload driver: a stream of seeded design requests through the
continuous-batching solve server (topo_server_* in libtopo.so).

Each request is a design (grid 2n x n x n, cantilever or MBB, cone-smoothed
random densities) that arrives at a Poisson time and then asks for
`n_steps` solves: after each solve the client submits the densities
perturbed by a factor in [0.95, 1.05] (a SIMP-style step; the whole
sequence is generated before the clock starts and replayed), which the
server warm-starts from the previous displacement.  The server admits
designs by device-memory footprint, keeps them resident, and overlaps all of
their solves on the GPU; this module only schedules arrivals and records
latencies.

    python -m paper_2605_04735_gb300.serving [--requests 64] [--steps 30]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import topo


def server_opts():
    """Solve options of the serving stream: the defaults with the convergence
    checked every 4 CG iterations (a warm-started SIMP-style re-solve
    converges in a few iterations, so a chunk of 8 mostly replays no-op
    kernels after it has; measured on the saturated stream: 4 -> 890,
    8 -> 854, 16 -> 754 solves/s)."""
    return topo.default_opts(check_every=4)


def trace(requests):
    """Every density each request will submit (step 0 and its n_steps - 1
    perturbations), generated up front: the stream is replayed from this
    trace, so the timed loop measures the server, not the client's random
    number generation (~1 ms of host time per solve of the mean grid)."""
    out = {}
    for r in requests:
        rho = r.rho0
        seq = [rho]
        for step in range(1, r.n_steps):
            rho = I.perturb(rho, r.factor(step))
            seq.append(rho)
        out[r.rid] = seq
    return out


def run_stream(requests, budget_bytes: int, max_active: int = 64, opts=None,
               realtime: bool = True, densities=None):
    """Drive the request stream; returns per-solve and per-request records.

    realtime: submit each request at its arrival time (wall clock since the
    start); False submits everything at once (saturation).  densities: the
    trace of every request's densities (default: made here, before the
    clock starts)."""
    if densities is None:
        densities = trace(requests)
    server = topo.Server(budget_bytes, max_active, opts=opts)
    pending = sorted(requests, key=lambda r: r.arrival)
    state = {}          # design -> [request, step, rho, arrival wall time]
    solves, reqs = [], []
    t0 = time.perf_counter()
    clock0 = None
    nxt = 0
    try:
        while nxt < len(pending) or state:
            now = time.perf_counter() - t0
            while nxt < len(pending) and (not realtime or pending[nxt].arrival <= now):
                r = pending[nxt]
                nxt += 1
                d = server.open(r.nx, r.ny, r.nz, r.bc, r.load)
                server.submit(d, r.rho0)
                state[d] = [r, 0, r.rho0, time.perf_counter() - t0]
            wait = not realtime or nxt >= len(pending)
            for res in server.poll(wait=wait):
                if clock0 is None:
                    clock0 = (time.perf_counter() - t0) - res.finish_s
                r, step, rho, t_arr = state[res.design]
                if res.status != 0:
                    raise topo.TopoError(res.status, f"request {r.rid} step {step} "
                                                     f"(failure detail {res.detail})")
                solves.append({"rid": r.rid, "step": step, "latency_s": res.finish_s - res.submit_s,
                               "queue_s": res.start_s - res.submit_s, "iters": res.iters,
                               "rel_residual": res.rel_residual, "compliance": res.compliance,
                               "n_dof": 3 * (r.nx + 1) * (r.ny + 1) * (r.nz + 1)})
                step += 1
                if step < r.n_steps:
                    rho = densities[r.rid][step]
                    server.submit(res.design, rho)
                    state[res.design] = [r, step, rho, t_arr]
                else:
                    reqs.append({"rid": r.rid, "latency_s": (clock0 + res.finish_s) - t_arr})
                    server.retire(res.design)
                    del state[res.design]
            if realtime and nxt < len(pending) and not state:
                time.sleep(max(0.0, min(0.01, pending[nxt].arrival - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        stats = server.stats()
    finally:
        server.close()
    return solves, reqs, wall, stats


def summarize(solves, reqs, wall, stats):
    lat = np.array([s["latency_s"] for s in solves]) * 1e3
    rl = np.array([r["latency_s"] for r in reqs]) * 1e3
    return {"solves": len(solves), "requests": len(reqs), "wall_s": wall,
            "solves_per_s": len(solves) / wall,
            "solve_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "request_latency_ms": {"p50": float(np.percentile(rl, 50)), "p99": float(np.percentile(rl, 99))},
            "iters_mean": float(np.mean([s["iters"] for s in solves])),
            "dof_mean": float(np.mean([s["n_dof"] for s in solves])),
            "max_rel_residual": float(max(s["rel_residual"] for s in solves)),
            "peak_device_bytes": stats["peak_bytes"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--max-ny", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--loads", default="0.5,0.8,1.0")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    budget = int(args.budget_gb * 2**30)
    # saturated throughput: every request at t = 0
    reqs = I.serving_stream(args.requests, args.steps, rate=0.0, max_ny=args.max_ny)
    sat = summarize(*run_stream(reqs, budget, args.max_active, opts=server_opts(),
                                realtime=False))
    lam_sat = sat["solves_per_s"] / args.steps   # requests per second
    out = {"workload": f"serving: {args.requests} requests x {args.steps} solves, grids 2n x n x n, "
                       f"n in 12..{args.max_ny} step 4, half cantilever / half MBB",
           "saturated": sat, "lambda_sat_req_per_s": lam_sat, "runs": {}}
    for f in [float(x) for x in args.loads.split(",")]:
        reqs = I.serving_stream(args.requests, args.steps, rate=f * lam_sat, max_ny=args.max_ny)
        out["runs"][f"{f:.2f}x"] = summarize(*run_stream(reqs, budget, args.max_active,
                                                         opts=server_opts()))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
