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
API with host buffers.  `roofline` is the step's largest kernel, the FP32
operator with the multigrid's Chebyshev-step epilogue on the finest level,
timed live over the timed steps against the HBM copy bandwidth (algorithmic
bytes); `roofline_cg_apply` the CG applies the same way (28 B per node).
`same_batch` times one step of the same batch with plain FP64 Jacobi-PCG and
with FP32 Jacobi-PCG inside FP64 refinement; `serving` runs the serving
stream; `cpu_baseline` is one full oracle solve on the host's cores.

Under torchrun every rank solves its own independent designs (weak
scaling); the only collectives are the timing barrier and max-reduction.
`--impl reference` times the CPU oracle (banded Cholesky of the full
problem, one design per step) instead.
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
SAME_BATCH = 256  # designs of the precision / preconditioner comparison group
PAIR_AUTO_MIN_NX = 150  # the library's automatic modal form pairs columns from this nx on


def exec_ops(op: int, nx: int, role: str) -> float | None:
    """FP32 lane-operations per element executed by the default operator
    kernels in `role` ("cheb_step" or "cg_apply"); None for the other forms
    (not counted)."""
    if op != 0:
        return None
    if role == "cheb_step":
        return None if nx >= PAIR_AUTO_MIN_NX else EXEC_FP32_OPS_PER_ELEM["cheb_step"]
    return EXEC_FP32_OPS_PER_ELEM["cg_apply_pair" if nx >= PAIR_AUTO_MIN_NX else "cg_apply_tma"]


def operator_kernel(op: int, nx: int) -> str:
    """The FP32 operator kernel that runs for operator choice `op` on a grid
    of nx elements in x (topo.OPERATOR_*)."""
    if op == 1:
        return "k_stencil_tma (FP32 node-centric 27-node gather)"
    if op == 4:
        return "k_tc_tma (tensor cores: K0.U_e as TF32 tcgen05 GEMMs, accumulator in TMEM)"
    if op == 5 and nx <= 128:
        return ("k_modal_tma, cluster form (FP32 modal operator, one element column per thread, "
                "the x tiles of a grid row as one thread-block cluster)")
    if op == 3 or (op == 0 and nx >= PAIR_AUTO_MIN_NX):
        return "k_modal_pair (FP32 modal operator, two element columns per thread, packed f32x2)"
    return "k_modal_tma (FP32 modal operator, one element column per thread)"


# DRAM bytes (read + write) per launch of the CG apply (operator + p.Ap) from
# one ncu capture of the same kernel source, by workload; None until captured
# on the current source (k_modal_tma on one 96x32x32 design, not recaptured
# since its march was packed; k_modal_pair on 320x160x160)
NCU_TRAFFIC: dict[str, float | None] = {"mbb_96x32x32": None,
                                        LARGE_WORKLOAD: 183507712.0 + 69900032.0}
# DRAM bytes per design of the batched finest-level launches, from one ncu
# capture of a 64-design launch of the current kernel source
# (profiles/k_modal_tma_batch64_mbb_96x32x32.md): the Chebyshev step in its
# x-added form (8.00 MB algorithmic per design); the CG apply not recaptured
# since its march was packed
NCU_TRAFFIC_BATCH: dict[str, float | None] = {"cheb_step": (303747840.0 + 198051328.0) / 64,
                                              "cg_apply": None}
# FP32 lane-operations the modal kernels execute per element of the grid
# (ncu smsp__sass_thread_inst_executed_op_fp32_pred_on, a packed f32x2
# instruction counted as two; halo columns and idle thread slots included),
# the basis of the executed-operation floor: the Chebyshev step and the CG
# apply of k_modal_tma in a 64-design 96x32x32 launch (1.744 G and 1.615 G
# for 6.29 M elements; counted on the scalar march, which executes the same
# FP32 lane-operations as the packed one), k_modal_pair's CG apply at
# 320x160x160 (2.125 G for 8.19 M elements)
EXEC_FP32_OPS_PER_ELEM = {"cheb_step": 277.1, "cg_apply_tma": 256.7, "cg_apply_pair": 259.4}
FLOP_PER_ELEM = 2 * 24 * 24  # the dense K0 U_e product per element (multiply + add)


def operator_bytes(w: I.Workload) -> int:
    """Algorithmic HBM bytes of one CG apply y = K(rho) x (+ x.y) in FP32: x
    read and y written once per node (3 x 4 B each), the modulus read once
    per element (4 B)."""
    return 24 * w.n_nodes + 4 * w.n_elem


def fp32_lane_ops_per_s(sm_mhz: float) -> float:
    """FP32 SIMT issue rate: 152 SMs x 128 FP32 lanes x the SM clock."""
    return 152 * 128 * sm_mhz * 1e6


def hbm_roofline(kernel: str, w: I.Workload, bytes_per_launch: float, avg_ms: float,
                 designs: float, peaks: dict, peaks_src: str, traffic: float | None = None,
                 ops: float | None = None) -> dict:
    """An operator kernel against the HBM roofline: achieved = its
    algorithmic bytes per launch / its average launch time (CUDA events),
    peak = the measured copy bandwidth.  Beside it the arithmetic view: the
    dense-equivalent rate (1152 flop per element) and, given `ops` (FP32
    lane-operations executed per element), the floor the FP32 pipe sets."""
    t = avg_ms * 1e-3
    peak = float(peaks["hbm_gbs"])
    achieved = bytes_per_launch / t / 1e9
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    elems = w.n_elem * designs
    alu = {"dense_equivalent_tflops": FLOP_PER_ELEM * elems / t / 1e12,
           "note": "1152 flop per element is the dense K0.U_e product; the modal kernels reach "
                   "the same result with fewer executed operations"}
    if ops is not None:
        floor_s = elems * ops / fp32_lane_ops_per_s(mhz)
        alu.update({"executed_fp32_ops_per_element": ops,
                    "executed_floor_us": floor_s * 1e6,
                    "executed_frac_of_fp32_pipe": floor_s / t,
                    "peak_source": f"derived: 152 SMs x 128 FP32 lanes x {mhz:.0f} MHz"})
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kernel, "workload": w.name,
            "bytes_per_launch": bytes_per_launch, "designs_per_launch": designs,
            "avg_launch_us": avg_ms * 1e3, "gdofs": 3.0 * w.n_nodes * designs / t / 1e9,
            "hbm_floor_us": bytes_per_launch / (peak * 1e9) * 1e6,
            "peak_source": f"{peaks_src}: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
            "alu_view": alu}


def large_operator(topo, stream, flush, op: int = 0, batches: int = 10, per_batch: int = 5):
    """The operator kernel alone on the 320x160x160 grid (inputs ~233 MB, above
    L2): batches x per_batch back-to-back launches, each batch between its own
    pair of CUDA events on the caller stream (the library fences its own
    stream to the caller's once per batch), L2 flushed before the first;
    returns the median over the batches of the mean launch time, in ms."""
    import torch
    w = I.WORKLOADS[LARGE_WORKLOAD]
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load, stream=stream) as m:
        m.set_operator(op)
        m.set_density(w.density())
        m.apply_internal(1, 3)  # warm-up
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(batches + 1)]
        ev[0].record(stream)
        for k in range(batches):
            m.apply_internal(1, per_batch)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        return float(np.median([ev[k].elapsed_time(ev[k + 1]) / per_batch
                                for k in range(batches)]))


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


SEED_STRIDE = 1_000_000  # seeds per rank: ranks' batches never overlap (batch < stride)


def design_seeds(base_seed: int, rank: int, batch: int):
    """Seeds of the independent designs rank `rank` solves: disjoint across
    ranks (weak scaling: every rank gets its own batch, no data exchange)."""
    if batch > SEED_STRIDE:
        raise ValueError(f"at most {SEED_STRIDE} designs per rank")
    return [base_seed + SEED_STRIDE * rank + b for b in range(batch)]


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
        pw = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            try:
                pw.append(float(f[3]))
            except (ValueError, IndexError):
                pass
        out = {"sm_mhz": float(np.median(sm)), "sm_min_mhz": min(sm), "sm_max_mhz": max(mx),
               "reasons": sorted(reasons), "samples": len(sm)}
        if pw:
            out["power_w_median"] = float(np.median(pw))
            out["power_w_max"] = max(pw)
        return out


def oracle_step(workload: I.Workload, rho: np.ndarray) -> float:
    """One full oracle pass of the workload on the host (assembled FP64 K,
    LAPACK banded Cholesky of the whole problem, compliance, sensitivities);
    returns its wall time in seconds."""
    from oracle import fem
    t0 = time.perf_counter()
    P = fem.Problem(workload.nx, workload.ny, workload.nz, workload.bc, workload.load, rho)
    u = P.solve()
    P.compliance(u)
    P.sensitivity(u)
    return time.perf_counter() - t0


def slab(workload: I.Workload, rho: np.ndarray, nx_s: int = 12):
    """The first nx_s element layers of the workload (same cross-section and
    band): a short oracle run that warms the host's BLAS threads up."""
    w = I.dataclasses.replace(workload, nx=min(nx_s, workload.nx))
    r = np.ascontiguousarray(rho.reshape(workload.nz, workload.ny, workload.nx)[:, :, :w.nx])
    return w, r.reshape(-1)


def cpu_baseline(workload: I.Workload):
    """The oracle timed on the full workload: one complete direct solve of
    design 0 with its compliance and sensitivities, on all host cores."""
    rho = workload.density()
    t = oracle_step(workload, rho)
    cores = os.cpu_count() or 1
    return {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 full oracle solve of {workload.name} (assembled FP64 K, LAPACK banded "
                      f"Cholesky of all {3 * workload.n_nodes} DOFs, compliance, sensitivities) in "
                      f"{t:.2f} s; LAPACK threads = all {cores} host cores"}


def run_reference(args, workload):
    """The CPU oracle as the reference arm: every timed step is one complete
    oracle solve of the full workload (a design of the benchmark's batch);
    warm-up steps solve the 12-layer slab of it (same band), which warms the
    BLAS threads without spending minutes on untimed work."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    rhos = [I.dataclasses.replace(workload, seed=sd).density()
            for sd in design_seeds(workload.seed, 0, max(1, args.steps))]
    for it in range(args.warmup):
        w_s, r_s = slab(workload, rhos[it % len(rhos)])
        oracle_step(w_s, r_s)
    times = [oracle_step(workload, rhos[k % len(rhos)]) for k in range(args.steps)]
    ms = 1e3 * float(np.mean(times))
    value = 1e3 / ms
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload.name, "nx": workload.nx, "ny": workload.ny,
                       "nz": workload.nz, "rtol": 1e-8, "solver": "banded Cholesky (LAPACK)",
                       "warmup": "12-layer slab solves (same band)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each timed step: one full oracle solve of {workload.name} "
                                       f"(all {3 * workload.n_nodes} DOFs), compliance and "
                                       f"sensitivities; {args.steps} designs of the benchmark's "
                                       f"seeds; step times {min(times):.2f}-{max(times):.2f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def serving_cpu_baseline(reqs) -> dict:
    """The oracle on a bounded sample of the serving stream's designs: one
    cold FP64 solve (density, solve, compliance, sensitivities) of the
    smallest grid (direct Cholesky) and of the median grid (the oracle's
    matrix-free Jacobi-PCG to 1e-8: a direct band would need ~9 GB), on all
    host cores; a power law in the DOF count through the two times gives
    the mean time per solve over the stream's grid mix."""
    from oracle import fem
    from oracle import fullsize as FS
    by_ny = sorted(reqs, key=lambda r: r.ny)
    picks = [by_ny[0], by_ny[len(by_ny) // 2]]
    pts = []
    for r in picks:
        t0 = time.perf_counter()
        g = fem.Grid(r.nx, r.ny, r.nz)
        if r.ny <= 16:
            P = fem.Problem(r.nx, r.ny, r.nz, r.bc, r.load, r.rho0)
            u = P.solve()
            P.compliance(u)
            P.sensitivity(u)
            how = "banded Cholesky"
        else:
            E = fem.simp_modulus(r.rho0)
            k0 = fem.element_stiffness(1.0, 0.3)
            f = fem.load_vector(g, r.load)
            fixed = fem.fixed_dofs(g, r.bc)
            u, it, rel = FS.cg(g, E, k0, f, fixed, rtol=1e-8)
            fem.sensitivity(g, u, r.rho0, k0)
            how = f"Jacobi-PCG, {it} iterations"
        pts.append((g.n_dof, time.perf_counter() - t0, f"{r.nx}x{r.ny}x{r.nz} ({how})"))
    (n0, t0_, _), (n1, t1_, _) = pts
    b = np.log(t1_ / t0_) / np.log(n1 / n0) if n1 != n0 else 1.0
    mean_t = float(np.mean([t0_ * (3 * (r.nx + 1) * (r.ny + 1) * (r.nz + 1) / n0) ** b
                            for r in reqs]))
    cores = os.cpu_count() or 1
    return {"value": 1.0 / mean_t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "; ".join(f"{name}: {t:.2f} s" for _, t, name in pts)
                      + f"; mean over the stream's grids by t ~ DOF^{b:.2f}: {mean_t:.2f} s per "
                        "cold solve (the GPU's solves are warm-started)"}


def large_configs(topo, stream, flush, steps: int = 3, cpu_iters: int = 10,
                  peaks: dict | None = None, peaks_src: str = "") -> dict:
    """The full-size cantilevers with voids (192x96x96: 5.4 M DOF, 40 voids;
    320x160x160: 25.0 M DOF, 120 voids), one design each, through the public
    API: the mixed-precision GMG-PCG step (density, solve to a true FP64
    relative residual of 1e-8, compliance, sensitivities) timed with CUDA
    events over `steps` steps after one warm-up step; one solve of the plain
    FP64 Jacobi-PCG GPU path to the same residual; and the oracle's FP64
    matrix-free Jacobi-PCG on the host, `cpu_iters` iterations timed on all
    cores, its solve estimated at the iteration count the GPU's FP64
    Jacobi-PCG needed (the same algorithm in the same arithmetic)."""
    import torch
    from oracle import fem
    from oracle import fullsize as FS
    out = {}
    for name in ("cantilever_voids_192x96x96", LARGE_WORKLOAD):
        w = I.WORKLOADS[name]
        rho = w.density()
        rec = {"dof": 3 * w.n_nodes}
        with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load, stream=stream) as m:
            rd = torch.from_numpy(rho).cuda()
            dc = torch.empty(w.n_elem, dtype=torch.float64, device="cuda")

            def step(o):
                m.set_density(rd)
                info = m.solve(o)
                m.compliance()
                m.sensitivity(dc)
                return info

            opts = topo.default_opts(rtol=1e-8)
            step(opts)  # hierarchy and graphs
            ts, its = [], []
            for k in range(steps):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                info = step(opts)
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
                its.append((info.iters, info.outer, info.rel_residual))
            rec["mixed_gmg"] = {"solves_per_s": 1e3 / float(np.mean(ts)),
                                "ms_per_step": float(np.mean(ts)),
                                "iters": its[-1][0], "outer": its[-1][1],
                                "rel_residual": its[-1][2]}
            if name == LARGE_WORKLOAD and peaks:
                # the step's largest kernel, the finest-level Chebyshev step,
                # timed live by the library's event pair around each launch
                # (in separate steps: the events ride in the captured graphs,
                # whose first profiled use captures them again)
                m.profile(True)
                step(opts)
                m.profile_read_smoother(reset=True)
                for k in range(steps):
                    flush.fill_(float(k))
                    step(opts)
                torch.cuda.synchronize()
                cms, cn, cb = m.profile_read_smoother(reset=True)
                m.profile(False)
                if cn > 0:
                    r = hbm_roofline(operator_kernel(0, w.nx) + " with the Chebyshev-step "
                                     "epilogue, finest level", w, cb / cn, cms / cn, 1.0, peaks,
                                     peaks_src)
                    r.update({"bytes_rule": "per node 60 B (x stored) or 72 B (x added), per "
                                            "element 4 B",
                              "launches": cn,
                              "timed": f"every finest-level Chebyshev step of {steps} full "
                                       "steps of one design, CUDA events on the library's "
                                       "stream; inputs above L2"})
                    rec["roofline_cheb_step"] = r
            o64 = topo.default_opts(precision=topo.PREC_FP64, precond=topo.PRECOND_JACOBI,
                                    rtol=1e-8)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            info = step(o64)
            b.record(stream)
            torch.cuda.synchronize()
            ms64 = a.elapsed_time(b)
            rec["fp64_jacobi_pcg"] = {"solves_per_s": 1e3 / ms64, "ms_per_step": ms64,
                                      "iters": info.iters, "rel_residual": info.rel_residual}
            rec["gain_over_fp64_jacobi"] = ms64 / rec["mixed_gmg"]["ms_per_step"]
        g = fem.Grid(w.nx, w.ny, w.nz)
        E = fem.simp_modulus(rho)
        k0 = fem.element_stiffness(1.0, 0.3)
        f = fem.load_vector(g, w.load)
        fixed = fem.fixed_dofs(g, w.bc)
        t0 = time.perf_counter()
        _, it, _ = FS.cg(g, E, k0, f, fixed, rtol=0.0, maxiter=cpu_iters)
        per_it = (time.perf_counter() - t0) / max(it, 1)
        n64 = rec["fp64_jacobi_pcg"]["iters"]
        rec["cpu_baseline"] = {"value": 1.0 / (per_it * n64), "unit": UNIT,
                               "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": f"{it} iterations of the oracle's FP64 matrix-free "
                                         f"Jacobi-PCG: {per_it * 1e3:.1f} ms each; a solve "
                                         f"to 1e-8 = {n64} iterations (the GPU FP64 "
                                         f"Jacobi-PCG's count): {per_it * n64:.1f} s"}
        out[name] = rec
    return out


def serving_summary(budget_gb: float = 40.0, loads=(0.5, 0.8, 1.0)):
    """The serving workload (64 requests x 30 solves, grids 24x12x12 ..
    128x64x64, half cantilever / half MBB) through the continuous-batching
    server: saturated throughput, then Poisson arrivals at fractions of it."""
    from paper_2605_04735_gb300 import serving as SV
    budget = int(budget_gb * 2**30)
    opts = SV.server_opts()
    reqs = I.serving_stream(64, 30, rate=0.0)
    sat = SV.summarize(*SV.run_stream(reqs, budget, 64, opts=opts, realtime=False))
    lam = sat["solves_per_s"] / 30
    out = {"workload": "64 requests x 30 solves, grids 2n x n x n, n in 12..64 step 4, half "
                       "cantilever / half MBB, densities perturbed +-5 % per solve",
           "budget_gb": budget_gb, "check_every": opts.check_every, "saturated": sat, "lambda_sat_req_per_s": lam, "runs": {}}
    for f in loads:
        reqs_f = I.serving_stream(64, 30, rate=f * lam)
        out["runs"][f"{f:.2f}x"] = SV.summarize(*SV.run_stream(reqs_f, budget, 64, opts=opts))
    out["cpu_baseline"] = serving_cpu_baseline(reqs)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mbb_96x32x32", choices=sorted(I.WORKLOADS))
    ap.add_argument("--batch", type=int, default=1024,
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
    ap.add_argument("--operator", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="operator kernel family (topo.OPERATOR_*)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the plain FP64 Jacobi-PCG path timed for comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--large", type=int, default=1,
                    help="1: also time one design of 192x96x96 and of 320x160x160 (mixed GMG, "
                         "plain FP64 Jacobi-PCG, the oracle's per-iteration time on the host)")
    ap.add_argument("--same-batch", type=int, default=1,
                    help="1: also time one step of the same batch with FP32 Jacobi-PCG + FP64 "
                         "refinement and with plain FP64 Jacobi-PCG")
    ap.add_argument("--serving", type=int, default=1,
                    help="1: also run the serving stream (64 requests x 30 solves) and report "
                         "its latency and throughput")
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
            m.profile_read_smoother(reset=True)
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
    # the finest-level Chebyshev steps of the V-cycles (the step's largest kernel)
    sreads = [h.profile_read_smoother(reset=True) for h in heads]
    cheb_ms, cheb_units, cheb_bytes = (sum(r[q] for r in sreads) for q in range(3))
    for h in heads:
        h.profile(False)
    value, total_ms = job_throughput(float(step_ms.sum()), B * args.steps, dist, "cuda")

    # ---- single-design latency (no per-launch events: on launches of a few
    # microseconds they would add to what is measured), then the operator
    # kernel's own timing in separate, instrumented steps of the same design ----
    m0.profile(False)
    step_one(m0, opts, rho_dev[0], dc_dev[0])  # its single-design graphs
    torch.cuda.synchronize()
    lat = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step_one(m0, opts, rho_dev[0], dc_dev[0])
        b.record(stream)
        torch.cuda.synchronize()
        lat.append(a.elapsed_time(b))
    lat = np.array(lat)
    m0.profile(True)
    for k in range(max(3, args.steps // 2)):
        flush.fill_(float(k))
        step_one(m0, opts, rho_dev[0], dc_dev[0])
    torch.cuda.synchronize()
    prof_ms, prof_n, _ = m0.profile_read(reset=True)
    m0.profile(False)

    # ---- e2e through the public API with pinned host buffers (one untimed
    # step first: the batch's graphs were captured with the per-launch events
    # of the timed steps and are captured again without them) ----
    rho_host = torch.from_numpy(rhos_np).pin_memory()
    dc_host = torch.empty((B, w.n_elem), dtype=torch.float64).pin_memory()
    step_batch(rho_host.numpy(), dc_host.numpy(), opts)
    torch.cuda.synchronize()

    def copy_gbs(dst, src):
        """GB/s of one copy of the pinned e2e buffers (CUDA events)."""
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dst.copy_(src, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        return src.numel() * src.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9

    copies = {"h2d_before": copy_gbs(rho_dev, rho_host), "d2h_before": copy_gbs(dc_host, dc_dev)}
    e2e_t = []
    with ClockSampler(local) as clk_e2e:
        for k in range(max(5, args.steps)):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_batch(rho_host.numpy(), dc_host.numpy(), opts)
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
    e2e_value = ws * B / float(np.mean(e2e_t))
    copies.update({"h2d_after": copy_gbs(rho_dev, rho_host),
                   "d2h_after": copy_gbs(dc_host, dc_dev)})

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

    # ---- the same designs (the first SAME_BATCH of the batch, one mesh group
    # of their own, same accuracy) with the mixed GMG path, with FP32
    # Jacobi-PCG inside FP64 refinement and with the plain FP64 Jacobi-PCG
    # path: the precision and preconditioner gains apart ----
    same_batch = None
    if args.same_batch and batched and rank == 0:
        nb = min(B, SAME_BATCH)
        sub = topo.create_batch(nb, w.nx, w.ny, w.nz, w.bc, w.load, stream=stream, opts=opts)
        r_sub, d_sub = rho_dev[:nb], dc_dev[:nb]

        def step_sub(o):
            topo.set_density_many(sub, r_sub)
            infos_s = topo.solve_many(sub, o)
            topo.compliance_many(sub)
            topo.sensitivity_many(sub, d_sub)
            return infos_s

        same_batch = {"what": f"one step of the first {nb} designs of the batch as one mesh "
                              "group (densities, solve to true rel. residual 1e-8, "
                              "compliances, sensitivities), lockstep, CUDA events, L2 flushed; "
                              "the Jacobi paths' graph capture included",
                      "designs": nb}
        for key, prec, pc in (("fp32_gmg_ir", topo.PREC_FP32, topo.PRECOND_GMG),
                              ("fp32_jacobi_ir", topo.PREC_FP32, topo.PRECOND_JACOBI),
                              ("fp64_jacobi_pcg", topo.PREC_FP64, topo.PRECOND_JACOBI)):
            oj = opts if pc == topo.PRECOND_GMG else topo.default_opts(
                precision=prec, precond=pc, rtol=1e-8)
            if pc == topo.PRECOND_GMG:
                step_sub(oj)  # hierarchy and graphs
            flush.fill_(3.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            infos_j = step_sub(oj)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            same_batch[key] = {"solves_per_s": nb * 1e3 / ms, "ms_per_step": ms,
                               "iters_mean": float(np.mean([i.iters for i in infos_j])),
                               "outer_mean": float(np.mean([i.outer for i in infos_j])),
                               "rel_residual_max": float(max(i.rel_residual for i in infos_j))}
        for m in sub:
            m.close()
        g32, g64 = same_batch["fp32_jacobi_ir"], same_batch["fp64_jacobi_pcg"]
        same_batch["gain_fp32_over_fp64_jacobi"] = g32["solves_per_s"] / g64["solves_per_s"]
        same_batch["gain_gmg_over_jacobi_fp32"] = (same_batch["fp32_gmg_ir"]["solves_per_s"] /
                                                   g32["solves_per_s"])
        same_batch["gain_total_over_fp64_jacobi"] = (same_batch["fp32_gmg_ir"]["solves_per_s"] /
                                                     g64["solves_per_s"])

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
    kern = operator_kernel(args.operator, w.nx)
    large_kern = operator_kernel(args.operator, lw.nx)
    large = hbm_roofline(large_kern + ", CG apply", lw,
                         operator_bytes(lw), large_operator(topo, stream, flush, args.operator),
                         1.0, peaks, peaks_src,
                         traffic=NCU_TRAFFIC.get(lw.name) if args.operator == 0 else None,
                         ops=exec_ops(args.operator, lw.nx, "cg_apply"))
    large["timed"] = ("50 back-to-back CG applies in 10 batches of 5 between CUDA events: the "
                      "median of the batch means; inputs above L2")
    single = hbm_roofline(kern + ", CG apply", w, operator_bytes(w), avg_ms, 1.0, peaks,
                          peaks_src,
                          traffic=NCU_TRAFFIC.get(w.name) if args.operator == 0 else None,
                          ops=exec_ops(args.operator, w.nx, "cg_apply"))
    single["timed"] = ("CG applies of instrumented steps of one design alone (2.9 MB: "
                       "L2-resident), apart from the latency steps")
    single["launches"] = prof_n
    cg_apply = None
    if batched and batch_op_units > 0:
        # design-launch units: the bytes of the timed launches over their
        # summed duration (each launch covered the designs still iterating)
        cg_apply = hbm_roofline(kern + ", CG apply", w, operator_bytes(w),
                                batch_op_ms / batch_op_units, 1.0, peaks, peaks_src,
                                traffic=NCU_TRAFFIC_BATCH["cg_apply"] if args.operator == 0
                                else None, ops=exec_ops(args.operator, w.nx, "cg_apply"))
        cg_apply.update({"designs_per_launch": "varies (designs still iterating); figures per "
                                              "design-launch",
                         "avg_launch_us": None,
                         "timed": "every CG apply of the timed batched steps, CUDA events on the "
                                  "library's stream; bytes counted per design the launch advanced",
                         "design_launches": batch_op_units, "total_ms": batch_op_ms})
    main = cg_apply or single
    if batched and cheb_units > 0:
        # the dominant kernel of the batched step: the finest-level Chebyshev
        # smoothing step (operator + smoothing epilogue)
        main = hbm_roofline(kern + " with the Chebyshev-step epilogue", w,
                            cheb_bytes / cheb_units, cheb_ms / cheb_units, 1.0, peaks, peaks_src,
                            traffic=NCU_TRAFFIC_BATCH["cheb_step"] if args.operator == 0
                            else None, ops=exec_ops(args.operator, w.nx, "cheb_step"))
        main["traffic_note"] = ("ncu, one 64-design launch of the x-added form (8.00 MB "
                                "algorithmic per design; bytes_per_launch averages the stored "
                                "and added forms): DRAM / algorithmic = 0.98")
        main.update({"designs_per_launch": "varies (designs still iterating); figures per "
                                          "design-launch",
                     "avg_launch_us": None,
                     "bytes_rule": "per node 60 B (x stored) or 72 B (x added), per element 4 B",
                     "timed": "every finest-level Chebyshev step of the timed batched steps, CUDA "
                              "events on the library's stream; bytes counted per design the "
                              "launch advanced",
                     "design_launches": cheb_units, "total_ms": cheb_ms})
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
        "same_batch": same_batch,
        # the dominant kernel of the timed steps (finest-level Chebyshev step),
        # the CG apply (operator fused with p.Ap) over the timed batched steps,
        # alone for one design, and alone on the 320x160x160 grid
        "roofline": main,
        "roofline_cg_apply": cg_apply,
        "roofline_single": single,
        "roofline_large": large,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * w.n_elem * B,
                "d2h_bytes_per_step": (8 * w.n_elem + 8) * B,
                "steps_ms": [round(1e3 * t, 2) for t in e2e_t], "clocks": clk_e2e.summary(),
                "copy_gbs": {k: round(v, 1) for k, v in copies.items()},
                "host_cpus": sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                else None},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    if pool is not None:
        pool.shutdown()
    for m in meshes:
        m.close()
    # the side measurements after the headline: a failure there is reported
    # in its own key and does not lose the headline line
    if args.large and ws == 1 and args.operator == 0:
        try:
            line["large_configs"] = large_configs(topo, stream, flush, peaks=peaks,
                                                  peaks_src=peaks_src)
            cheb_large = line["large_configs"].get(LARGE_WORKLOAD, {}).get("roofline_cheb_step")
            if cheb_large:
                line["roofline_large_cheb_step"] = cheb_large
        except Exception as e:  # noqa: BLE001
            line["large_configs"] = {"error": f"{type(e).__name__}: {e}"}
    if args.serving and ws == 1:
        try:
            line["serving"] = serving_summary()
        except Exception as e:  # noqa: BLE001
            line["serving"] = {"error": f"{type(e).__name__}: {e}"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
