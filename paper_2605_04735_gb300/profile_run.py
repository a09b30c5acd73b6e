"""Small, self-contained drivers for profiler captures of the hot path.

    python -m paper_2605_04735_gb300.profile_run apply <workload> [reps] [operator]
        one mesh, density set, `reps` internal applications of the FP32
        operator (the CG apply with its fused p.Ap reduction) on a
        non-default stream: the capture target of the operator kernel
        (operator: topo.OPERATOR_*, default the automatic modal form).
    python -m paper_2605_04735_gb300.profile_run apply64 <workload> [reps]
        the same with the FP64 operator.
    python -m paper_2605_04735_gb300.profile_run applydw <workload> [reps]
        the same with the double-word operator (the refinement residual's).
    python -m paper_2605_04735_gb300.profile_run solve <workload> [reps]
        `reps` full steps (density, FP32 GMG-PCG + FP64 refinement to 1e-8,
        compliance, sensitivities) on one mesh: the launch list of a step.
    python -m paper_2605_04735_gb300.profile_run simp <workload> [iters]
        `iters` SIMP iterations (solve, sensitivity, filter, OC update).
    python -m paper_2605_04735_gb300.profile_run batch <workload> [designs]
        (an optional last argument selects the operator for these modes too)
        one mesh group of `designs` seeded designs (default 16) solved in
        lockstep twice (a warm-up and the captured step) through the batched
        entry points (densities, solve, compliances, sensitivities): the
        launch list of a batched step.

    python -m paper_2605_04735_gb300.profile_run serving <requests> [steps]
        a saturated serving stream (every request at once) of `requests`
        seeded requests x `steps` solves through the solve server.

Workloads are the seeded recipes of `inputs.WORKLOADS`; nothing is read
from disk.  Each command prints one line starting with "ok".
"""
from __future__ import annotations

import sys


def main(argv):
    import numpy as np
    import torch

    from . import inputs as I
    from . import topo

    mode = argv[0] if argv else "apply"
    if mode == "serving":
        from . import serving as SV
        torch.cuda.set_device(0)
        n = int(argv[1]) if len(argv) > 1 else 8
        steps = int(argv[2]) if len(argv) > 2 else 5
        reqs = I.serving_stream(n, steps, rate=0.0)
        res = SV.summarize(*SV.run_stream(reqs, 1 << 35, 64, realtime=False))
        print("ok", mode, n, steps, res["solves"], round(res["solves_per_s"], 1))
        return
    name = argv[1] if len(argv) > 1 else "cantilever_voids_320x160x160"
    reps = int(argv[2]) if len(argv) > 2 else (1 if mode.startswith("apply") else 3)
    op = int(argv[3]) if len(argv) > 3 else 0
    w = I.WORKLOADS[name]
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    if mode == "batch":
        n = int(argv[2]) if len(argv) > 2 else 16
        rhos = [I.dataclasses.replace(w, seed=w.seed + b).density() for b in range(n)]
        opts = topo.default_opts(rtol=1e-8)
        meshes = topo.create_batch(n, w.nx, w.ny, w.nz, w.bc, w.load, stream=s, opts=opts)
        for m in meshes:
            m.set_operator(op)
        rho_dev = torch.from_numpy(np.stack(rhos)).cuda()
        dc_dev = torch.empty((n, w.nx * w.ny * w.nz), dtype=torch.float64, device="cuda")
        try:
            for _ in range(2):  # the batched entry points, as the benchmark's step
                topo.set_density_many(meshes, rho_dev)
                infos = topo.solve_many(meshes, opts)
                topo.compliance_many(meshes)
                topo.sensitivity_many(meshes, dc_dev)
            torch.cuda.synchronize()
        finally:
            for m in meshes:
                m.close()
        print("ok", mode, name, n, max(i.iters for i in infos), max(i.outer for i in infos))
        return
    with topo.Mesh(w.nx, w.ny, w.nz, w.bc, w.load, stream=s) as m:
        m.set_operator(op)
        rho = w.density()
        if mode in ("apply", "apply64", "applydw"):
            m.set_density(rho)
            m.apply_internal({"apply": 1, "apply64": 0, "applydw": 2}[mode], 3 * reps)
            torch.cuda.synchronize()
            print("ok", mode, name, reps)
        elif mode == "solve":
            info = None
            for _ in range(reps):
                m.set_density(rho)
                info = m.solve()
                m.compliance()
                m.sensitivity()
            torch.cuda.synchronize()
            print("ok", mode, name, info.iters, info.outer, info.rel_residual)
        elif mode == "simp":
            r0 = np.full(w.n_elem, 0.4, np.float32)
            hist = topo.simp_optimize(m, r0, topo.default_simp_opts(volfrac=0.4),
                                      max_iter=reps, tol=0.0)
            torch.cuda.synchronize()
            print("ok", mode, name, len(hist), hist[-1][0])
        else:
            raise SystemExit(f"unknown mode {mode!r}")


if __name__ == "__main__":
    main(sys.argv[1:])
