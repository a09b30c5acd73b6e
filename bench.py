"""Benchmark: PCG state solves/s (true FP64 relative residual 1e-8) of the
SIMP state solve + compliance + sensitivities, on the MBB half-beam
96x32x32 workload (cone-smoothed seeded densities), one JSON line.

A step is one pass of the whole hot path over a batch of B independent
designs (default 256, one mesh group solved in lockstep; `--streams` for
independent meshes): density upload and SIMP interpolation (Eq. (1)), the
state solve K(rho) u = f (Eq. (2)) to rel. residual 1e-8, the compliance
f^T u and the element sensitivities (Eq. (3)).  `value` times steps with
inputs already in HBM (device timeline, CUDA events on the library's
stream, L2 flushed between steps); `e2e` times the same through the public
API with host buffers.  `roofline` is the FP32 operator's CG applies timed
live over the timed steps, against the FP32 pipe (1152 flop per element).

Under torchrun every rank solves its own independent designs (weak
scaling); the only collectives are the timing barrier and max-reduction.
`--impl reference` times the CPU oracle (banded Cholesky) instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_04735_gb300 import inputs as I  # noqa: E402

METRIC = "PCG state solves/s at true FP64 rel. residual 1e-8 (solve + compliance + sensitivity)"
UNIT = "solves/s"
LARGE_WORKLOAD = "cantilever_voids_320x160x160"
PAIR_AUTO_MIN_NX = 150  # the library's automatic modal form pairs columns from this nx on


def operator_kernel(op: int, nx: int) -> str:
    """The FP32 operator kernel that runs for operator choice `op` on a grid
    of nx elements in x (topo.OPERATOR_*)."""
    if op == 1:
        return "k_stencil_tma (FP32 node-centric 27-node gather)"
    if op == 3 or (op == 0 and nx >= PAIR_AUTO_MIN_NX):
        return "k_modal_pair (FP32 modal operator, two element columns per thread, packed f32x2)"
    return "k_modal_tma (FP32 modal operator, one element column per thread)"
# DRAM bytes (read + write) per launch of the default operator kernel from one
# ncu capture of the same kernel source, by workload; None until captured
# (k_modal_tma on 96x32x32: its 2.9 MB working set stays in L2, so the
# output is never written back during the launch; k_modal_pair on 320x160x160)
NCU_TRAFFIC: dict[str, float | None] = {"mbb_96x32x32": 1957888.0 + 0.0,
                                        LARGE_WORKLOAD: 183507712.0 + 69900032.0}


def operator_bytes(w: I.Workload) -> int:
    """Algorithmic HBM bytes of one operator application y = K(rho) x in
    FP32: x read and y written once per node (3 x 4 B each), E read once per
    element (4 B)."""
    return 24 * w.n_nodes + 4 * w.n_elem


FLOP_PER_ELEM = 2 * 24 * 24  # the dense K0 U_e product per element (multiply + add)


def fp32_peak_tflops(sm_mhz: float) -> float:
    """FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x the SM clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def roofline(w: I.Workload, avg_ms: float, peaks: dict, peaks_src: str, op: int = 0,
             designs: float = 1.0, traffic: float | None = None) -> dict:
    """The FP32 SIMT operator is bound by the FP32 pipe: achieved = the dense
    algorithmic 1152 flop per element x the elements one launch processes
    (`designs` grids) / the average launch time, against the FP32 peak from
    the unit counts and the maximum SM clock.  The HBM view (28 B per node
    of algorithmic traffic against the measured copy bandwidth) is given
    beside it."""
    t = avg_ms * 1e-3
    flops = FLOP_PER_ELEM * w.n_elem * designs
    achieved = flops / t / 1e12
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(mhz)
    hbm = operator_bytes(w) * designs / t / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": operator_kernel(op, w.nx), "workload": w.name,
            "designs_per_launch": designs,
            "flop_per_launch": flops, "avg_launch_us": avg_ms * 1e3,
            "gdofs": 3.0 * w.n_nodes * designs / t / 1e9,
            "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz; "
                           "1152 flop per element is the dense K0.U_e product (the modal "
                           "kernel computes the same result with ~165 FP32 lane-ops)",
            "hbm": {"bytes_per_launch": operator_bytes(w) * designs, "achieved": hbm,
                    "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                    "frac": hbm / float(peaks["hbm_gbs"]),
                    "peak_source": f"{peaks_src}: MEASURED_PEAKS.json hbm_gbs"}}


def large_operator(topo, stream, flush, op: int = 0, reps: int = 20):
    """The operator kernel alone on the 320x160x160 grid (inputs ~233 MB, above
    L2): `reps` launches between CUDA events on the caller stream, L2 flushed
    before; returns the average launch time in ms."""
    import torch
    w = I.WORKLOADS[LARGE_WORKLOAD]
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load, stream=stream) as m:
        m.set_operator(op)
        m.set_density(w.density())
        m.apply_internal(1, 3)  # warm-up
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.apply_internal(1, reps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def design_seeds(base_seed: int, rank: int, batch: int):
    """Seeds of the independent designs rank `rank` solves: disjoint across
    ranks (weak scaling: every rank gets its own batch, no data exchange)."""
    return [base_seed + 1000 * rank + b for b in range(batch)]


def job_throughput(local_ms: float, units_per_rank: int, dist_mod=None, device=None):
    """Whole-job throughput: units over all ranks / the slowest rank's time
    (max-reduction across ranks; the only collective of the benchmark)."""
    ws = 1
    t = local_ms
    if dist_mod is not None and dist_mod.is_initialized():
        import torch
        ws = dist_mod.get_world_size()
        x = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist_mod.all_reduce(x, op=dist_mod.ReduceOp.MAX)
        t = float(x.item())
    return ws * units_per_rank / (t / 1e3), t


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.first = threading.Event()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            # the sampler's start-up (driver queries) is over before the
            # caller's timed region begins: it measured up to ~130 ms of
            # stalled launches when it overlapped the first timed step
            self.first.wait(timeout=3.0)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()
        self.first.set()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(workload: I.Workload, budget_s: float = 20.0):
    """The oracle (assembled K, banded Cholesky, compliance, sensitivities)
    timed on a slab of the workload with the same y-z cross-section and fewer
    x layers, scaled to the full problem by the number of free DOFs (the
    banded factorisation costs n * b^2 with the same band b)."""
    from oracle import fem
    nx_s = max(2, min(workload.nx, 12))
    t_tot, n = 0.0, 0
    rho_full = workload.density().reshape(workload.nz, workload.ny, workload.nx)
    rho = np.ascontiguousarray(rho_full[:, :, :nx_s]).reshape(-1)
    free_s = None
    while t_tot < budget_s / 2 or n == 0:
        t0 = time.perf_counter()
        P = fem.Problem(nx_s, workload.ny, workload.nz, workload.bc, workload.load, rho)
        u = P.solve()
        P.compliance(u)
        P.sensitivity(u)
        t_tot += time.perf_counter() - t0
        n += 1
        free_s = int((~P.fixed).sum())
        if n >= 3:
            break
    g = fem.Grid(workload.nx, workload.ny, workload.nz)
    free_full = int((~fem.fixed_dofs(g, workload.bc)).sum())
    t_full = (t_tot / n) * free_full / free_s
    cores = os.cpu_count() or 1
    return {"value": 1.0 / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle solve(s) of the {nx_s}x{workload.ny}x{workload.nz} slab "
                      f"(same cross-section and band), {t_tot / n:.2f} s each, scaled by free DOFs "
                      f"{free_full}/{free_s}; LAPACK threads = all {cores} host cores"}


def run_reference(args, workload):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import fem
    nx_s = max(2, min(workload.nx, 12))
    rho_full = workload.density().reshape(workload.nz, workload.ny, workload.nx)
    rho = np.ascontiguousarray(rho_full[:, :, :nx_s]).reshape(-1)
    g = fem.Grid(workload.nx, workload.ny, workload.nz)
    free_full = int((~fem.fixed_dofs(g, workload.bc)).sum())
    times = []
    free_s = None
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        P = fem.Problem(nx_s, workload.ny, workload.nz, workload.bc, workload.load, rho)
        u = P.solve()
        P.compliance(u)
        P.sensitivity(u)
        dt = time.perf_counter() - t0
        free_s = int((~P.fixed).sum())
        if it >= args.warmup:
            times.append(dt * free_full / free_s)
    ms = 1e3 * float(np.mean(times))
    value = 1e3 / ms
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload.name, "nx": workload.nx, "ny": workload.ny,
                       "nz": workload.nz, "rtol": 1e-8, "solver": "banded Cholesky (LAPACK)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: oracle solve of the {nx_s}x{workload.ny}x"
                                       f"{workload.nz} slab, scaled by free DOFs {free_full}/"
                                       f"{free_s}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mbb_96x32x32", choices=sorted(I.WORKLOADS))
    ap.add_argument("--batch", type=int, default=256,
                    help="independent designs solved concurrently per step")
    ap.add_argument("--check-every", type=int, default=0,
                    help="CG iterations between host convergence checks (0: the library's "
                         "default); a batch compacts its launches to the live designs at "
                         "each check")
    ap.add_argument("--groups", type=int, default=1,
                    help="mesh groups the batch is split into, each solved in lockstep by its "
                         "own host thread (their launches overlap on the GPU)")
    ap.add_argument("--inner-rtol", type=float, default=0.0,
                    help="relative residual reduction of each inner FP32 solve (0: the "
                         "library's default)")
    ap.add_argument("--smooth-degree", type=int, default=0,
                    help="Chebyshev smoothing degree of the V-cycle (0: the library's default)")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--precond", type=int, default=1)
    ap.add_argument("--operator", type=int, default=0, choices=[0, 1, 2, 3],
                    help="operator kernel family (topo.OPERATOR_*)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the plain FP64 Jacobi-PCG path timed for comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--streams", action="store_true",
                    help="independent meshes on their own streams instead of one mesh group "
                         "solved in lockstep (one launch per step for all designs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    workload = I.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, workload)
        return

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2605_04735_gb300 import build as _b
    if not os.path.exists(os.path.join(ROOT, "paper_2605_04735_gb300", "libtopo.so")):
        _b.build()
    from paper_2605_04735_gb300 import topo

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = workload
    B = max(1, args.batch)
    # independent designs: rank r, slot b gets seed + 1000 r + b (weak scaling)
    rhos_np = np.stack([I.dataclasses.replace(w, seed=sd).density()
                        for sd in design_seeds(w.seed, rank, B)])  # (B, n_elem)
    rho_dev = torch.from_numpy(rhos_np).cuda()
    dc_dev = torch.empty((B, w.n_elem), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    opts = topo.default_opts(precision=args.precision, precond=args.precond, rtol=1e-8)
    if args.check_every > 0:
        opts.check_every = args.check_every
    if args.smooth_degree > 0:
        opts.smooth_degree = args.smooth_degree
    if args.inner_rtol > 0:
        opts.inner_rtol = args.inner_rtol
    # one mesh group that solve_many runs as one batch (one launch per step
    # for all designs), or (--streams) independent meshes on their own streams
    batched = not args.streams and B > 1
    ng = max(1, min(args.groups, B // 2)) if batched else 1
    if not batched:
        meshes = [topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load, stream=stream) for _ in range(B)]
        groups = [meshes]
    else:
        sizes = [B // ng + (1 if g < B % ng else 0) for g in range(ng)]
        groups = [topo.create_batch(n, w.nx, w.ny, w.nz, w.bc, w.load, stream=stream, opts=opts)
                  for n in sizes]
        meshes = [m for g in groups for m in g]
    for m in meshes:
        m.set_operator(args.operator)

    pool = None
    if len(groups) > 1:
        from concurrent.futures import ThreadPoolExecutor
        pool = ThreadPoolExecutor(max_workers=len(groups))

    bounds = np.cumsum([0] + [len(g) for g in groups])

    def step_batch(rhos, dcs, opt):
        """rhos, dcs: (B, n_elem) arrays (numpy on the host or CUDA tensors);
        densities, compliances and sensitivities go through the batched
        entry points (one launch per group)."""
        for g, a, b in zip(groups, bounds[:-1], bounds[1:]):
            topo.set_density_many(g, rhos[a:b])
        if pool is None:
            infos = topo.solve_many(meshes, opt)
        else:  # the groups' solves overlap on the GPU (the library calls release the GIL)
            infos = [i for f in [pool.submit(topo.solve_many, g, opt) for g in groups]
                     for i in f.result()]
        cs = np.concatenate([topo.compliance_many(g) for g in groups])
        for g, a, b in zip(groups, bounds[:-1], bounds[1:]):
            topo.sensitivity_many(g, dcs[a:b])
        return infos, cs

    def step_one(m, opt, rho, dc):
        m.set_density(rho)
        info = m.solve(opt)
        c = m.compliance()
        m.sensitivity(dc)
        return info, c

    m0 = meshes[0]
    heads = [g[0] for g in groups]
    # the batch's CG applies are timed live with events (design 0 of each
    # group holds the group's timing); a warm-up step captures the profiled graphs
    if batched:
        for h in heads:
            h.profile(True)
    # warm-up: all but the last step here, the last one once the clock
    # sampler runs (its start-up must not land in a timed step)
    for _ in range(max(0, args.warmup - 1)):
        step_batch(rho_dev, dc_dev, opts)
    torch.cuda.synchronize()

    # ---- timed region: K batched steps, inputs resident in HBM ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    recs = []
    with ClockSampler(local) as clk:  # sampling from before the barrier to after the sync
        if args.warmup > 0:
            step_batch(rho_dev, dc_dev, opts)
        torch.cuda.synchronize()
        for m in meshes:
            m.profile_read(reset=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))  # evict the previous step's data from L2
            ev[k][0].record(stream)
            infos, cs = step_batch(rho_dev, dc_dev, opts)
            ev[k][1].record(stream)
            recs.extend((i.iters, i.outer, i.rel_residual, c) for i, c in zip(infos, cs))
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    reads = [m.profile_read(reset=True) for m in meshes]
    launches = sum(r[2] for r in reads)
    # summed over the groups: their launches overlap, so with several groups
    # the per-launch time includes the sharing of the GPU
    batch_op_ms = sum(r[0] for m, r in zip(meshes, reads) if m in heads)
    batch_op_units = sum(r[1] for m, r in zip(meshes, reads) if m in heads)
    for h in heads:
        h.profile(False)
    value, total_ms = job_throughput(float(step_ms.sum()), B * args.steps, dist, "cuda")

    # ---- single-design latency and the operator kernel's own timing ----
    m0.profile(True)
    lat = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step_one(m0, opts, rho_dev[0], dc_dev[0])
        b.record(stream)
        torch.cuda.synchronize()
        lat.append(a.elapsed_time(b))
    prof_ms, prof_n, _ = m0.profile_read(reset=True)
    m0.profile(False)
    lat = np.array(lat)

    # ---- e2e through the public API with pinned host buffers ----
    rho_host = torch.from_numpy(rhos_np).pin_memory()
    dc_host = torch.empty((B, w.n_elem), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e_t = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_batch(rho_host.numpy(), dc_host.numpy(), opts)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = ws * B / float(np.mean(e2e_t))

    # ---- the plain FP64 Jacobi-PCG GPU path on design 0 (comparison) ----
    fp64 = None
    if args.fp64_steps > 0 and rank == 0:
        o64 = topo.default_opts(precision=topo.PREC_FP64, precond=topo.PRECOND_JACOBI, rtol=1e-8)
        step_one(m0, o64, rho_dev[0], dc_dev[0])
        ts, its = [], []
        for k in range(args.fp64_steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            info, _ = step_one(m0, o64, rho_dev[0], dc_dev[0])
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
            its.append(info.iters)
        fp64 = {"solves_per_s": 1e3 / float(np.mean(ts)), "ms_per_solve": float(np.mean(ts)),
                "iters": int(np.mean(its)), "batch": 1}

    if rank != 0:
        if pool is not None:
            pool.shutdown()
        for m in meshes:
            m.close()
        if dist:
            dist.destroy_process_group()
        return

    peaks, peaks_src = _peaks()
    avg_ms = prof_ms / max(prof_n, 1)
    lw = I.WORKLOADS[LARGE_WORKLOAD]
    large = roofline(lw, large_operator(topo, stream, flush, args.operator), peaks, peaks_src,
                     args.operator,
                     traffic=NCU_TRAFFIC.get(lw.name) if args.operator == 0 else None)
    single = roofline(w, avg_ms, peaks, peaks_src, args.operator,
                      traffic=NCU_TRAFFIC.get(w.name) if args.operator == 0 else None)
    single["timed"] = "CG applies of the single-design loop (one design alone)"
    single["launches"] = prof_n
    if batched and batch_op_units > 0:
        # design-launch units: the flops of the timed launches over their
        # summed duration (each launch covered the designs still iterating)
        main = roofline(w, batch_op_ms / batch_op_units, peaks, peaks_src, args.operator)
        main["designs_per_launch"] = "varies (designs still iterating)"
        main["avg_launch_us"] = None
        main["timed"] = ("every CG apply of the timed batched steps, CUDA events on the "
                         "library's stream; flops counted per design the launch advanced")
        main["design_launches"] = batch_op_units
        main["total_ms"] = batch_op_ms
    else:
        main = single
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(w)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == 1 else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz,
                   "n_dof": 3 * w.n_nodes, "bc": "mbb" if w.bc == 1 else "cantilever",
                   "density": w.recipe, "rtol": 1e-8, "batch": B,
                   "layout": (f"{len(groups)} mesh group(s) solved in lockstep (one launch "
                              "per step for all designs of a group; groups on their own host "
                              "threads)" if batched else "independent meshes on streams"),
                   "solver": ("FP32 PCG + FP64 refinement" if args.precision == 1 else "FP64 PCG")
                   + (" / Jacobi" if args.precond == 0 else " / GMG V-cycle"),
                   "l2": "flushed between steps (256 MB write)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "batch_step_p50": float(np.percentile(step_ms, 50)),
                       "batch_steps_ms": [round(float(t), 3) for t in step_ms],
                       "what": "one design alone: density, solve, compliance, sensitivities"},
        "solve": {"iters_mean": float(np.mean([r[0] for r in recs])),
                  "outer_mean": float(np.mean([r[1] for r in recs])),
                  "rel_residual_max": float(max(r[2] for r in recs)),
                  "compliance_design0": recs[0][3]},
        "fp64_jacobi_pcg": fp64,
        # the CG apply (operator fused with p.Ap): over the timed batched
        # steps, alone for one design, and alone on the 320x160x160 grid
        "roofline": main,
        "roofline_single": single,
        "roofline_large": dict(large, timed="20 back-to-back applies, CUDA events, inputs "
                                            "above L2"),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * w.n_elem * B,
                "d2h_bytes_per_step": (8 * w.n_elem + 8) * B},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if pool is not None:
        pool.shutdown()
    for m in meshes:
        m.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
