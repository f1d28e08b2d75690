#!/usr/bin/env python
"""Benchmark: KFBI solves/s on one GB300 (or N independent replicas).

Workload (default): the 2D interface problem with the flower interface
r = 0.5 + 0.1 sin(5 theta) in [-1, 1]^2, sigma_in/sigma_out = 1000,
u_in = sin x cos y, u_out = x^2 + y^2, on the 1024^2 grid, fourth order.
One step = one complete solve through the C ABI: BIE right-hand side,
matrix-free GMRES to the relative residual --rtol and the final evaluation on
the grid (kfbi_gmres_solve + kfbi_evaluate).  The geometry set-up
(kfbi_create_problem) is outside the timed region and reported separately.

Also reported: box-solve Mpts/s (kfbi_box_solve alone), the plain FP64 path at
the same tolerance, an end-to-end figure with host buffers, the roofline of
the dominant kernel class, and the CPU oracle on the host cores.

`--impl reference` times the CPU oracle (the plain FP64 NumPy/SciPy
implementation) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_ALU_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 2 FP64 FMA / clk / SM at 2070 MHz
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
METRIC = "KFBI solves/sec & box-solve Mpts/s vs plain FP64 GPU at 1e-8 rel err; %HBM"


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def workload(n):
    import workloads as W
    return W.flower_interface_2d(n)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
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
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def job_throughput(local_ms, units_per_rank, world, device="cuda"):
    """Whole-job throughput of independent replicas: every rank processes
    units_per_rank units, the slowest rank's time (max over ranks) bounds
    the job.  Returns (max time in ms, units per second of all ranks)."""
    total = float(local_ms)
    if world > 1:
        import torch
        t = torch.tensor([total], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total = float(t.item())
    return total, world * units_per_rank / (total / 1e3)


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import build, kfbi

    build.build()
    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    stream = torch.cuda.current_stream()
    w = workload(args.n)
    prec = kfbi.MIXED if args.precision == "mixed" else kfbi.FP64
    box = kfbi.BOX_MG if args.box == "mg" else kfbi.BOX_DST
    t0 = time.perf_counter()
    G = kfbi.Problem.from_workload(w, box_solver=box, precision=prec,
                                   box_rtol=args.box_rtol if prec == kfbi.MIXED else 0.0,
                                   box_max_iters=args.box_steps,
                                   relax=args.relax if prec == kfbi.MIXED else 0.0)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    d = w.dim
    xyz = torch.zeros((G.nb, d), dtype=torch.float64, device="cuda")
    nrm = torch.zeros((G.nb, d), dtype=torch.float64, device="cuda")
    kfbi.kfbi_dof_points(G.handle, xyz, nrm)
    g1, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
    grid = W.grid_data(w)
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
            (("g1", g1), ("g2", g2), ("f_in", grid["f_in"]), ("f_out", grid["f_out"]),
             ("lapf_in", grid["lapf_in"]), ("lapf_out", grid["lapf_out"]), ("g_b", grid["g_b"]))}
    devd = {k: v.cuda() for k, v in host.items()}
    data = kfbi.make_data(**devd)
    dens = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
    u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")
    opts = kfbi.GmresOpts(rtol=args.rtol, restart=100, max_iter=300, x0=None)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        info = kfbi.kfbi_gmres_solve(G.handle, data, opts, dens)
        kfbi.kfbi_evaluate(G.handle, data, dens, u)
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    kfbi.kfbi_launch_counts(G.handle, reset=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times = []
    iters = []
    refine = []
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        iters.append(info.iters)
        refine.append(info.refine_steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = kfbi.kfbi_launch_counts(G.handle, reset=True)
    total_ms, value = job_throughput(sum(times), args.steps, world)
    ms_per_step = total_ms / args.steps

    # accuracy of the last solve
    ex = W.exact_grid(w, _inside(G, kfbi))
    err = float(np.abs(u.cpu().numpy() - ex)[1:-1, 1:-1].max())

    # ---- end to end through the C ABI with host buffers
    e2e_times = []
    u_host = torch.empty(G.grid_shape, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in host.values())
    d2h = u.numel() * 8
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in host:
            devd[k].copy_(host[k], non_blocking=True)
        step()
        u_host.copy_(u, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    _, e2e_value = job_throughput(sum(e2e_times), len(e2e_times), world)

    # ---- box solve alone
    rhs = torch.randn(G.grid_shape, dtype=torch.float64, device="cuda")
    ub = torch.zeros_like(rhs)
    bt = []
    for _ in range(5):
        kfbi.kfbi_box_solve(G.handle, rhs, ub)
    for _ in range(30):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kfbi.kfbi_box_solve(G.handle, rhs, ub)
        e1.record(stream)
        e1.synchronize()
        bt.append(e0.elapsed_time(e1))
    box_ms = statistics.median(bt)
    npts = (args.n - 1) ** d
    box_mpts = npts / (box_ms * 1e-3) / 1e6

    # ---- per-class profile (a separate pass with event timing enabled)
    kfbi.kfbi_profile_enable(G.handle, True)
    for _ in range(2):
        flush.zero_()
        step()
    prof = kfbi.kfbi_profile_read(G.handle)
    kfbi.kfbi_profile_enable(G.handle, False)
    steps_run = kfbi.kfbi_box_solve_info(G.handle)[0]
    roof = roofline(args, G, prof, prec, steps_run)

    # ---- the plain FP64 path at the same tolerance
    fp64 = None
    if args.compare_fp64 and prec != kfbi.FP64:
        G64 = kfbi.Problem.from_workload(w, box_solver=kfbi.BOX_DST, precision=kfbi.FP64)
        u64 = torch.zeros_like(u)
        d64 = torch.zeros_like(dens)
        for _ in range(2):
            kfbi.kfbi_gmres_solve(G64.handle, data, opts, d64)
            kfbi.kfbi_evaluate(G64.handle, data, d64, u64)
        t64 = []
        for _ in range(max(3, args.steps // 3)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kfbi.kfbi_gmres_solve(G64.handle, data, opts, d64)
            kfbi.kfbi_evaluate(G64.handle, data, d64, u64)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        err64 = float(np.abs(u64.cpu().numpy() - ex)[1:-1, 1:-1].max())
        diff = float(np.abs(u64.cpu().numpy() - u.cpu().numpy()).max())
        fp64 = {"solves_per_s": 1e3 / statistics.mean(t64), "ms_per_solve": statistics.mean(t64),
                "max_err_vs_exact": err64, "max_diff_vs_mixed": diff}
        G64.close()

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (FP32 box solve with FP64 residual refinement)" if prec else "f64",
        "data": "synthetic (manufactured solution, seeded, analytic level set)",
        "config": {"workload": f"flower interface 2D, N={args.n}, sigma_in/sigma_out=1000, "
                               f"4th order, GMRES rtol {args.rtol:g}",
                   "box_solver": args.box, "precision": args.precision, "n_b": G.nb,
                   "box_rtol": args.box_rtol if prec == kfbi.MIXED else None,
                   "box_steps": args.box_steps or None,
                   "relax": args.relax if prec == kfbi.MIXED else None,
                   "n_irr": G.nirr, "l2": "flushed (256 MB write) before every step",
                   "parallelism": "independent replicas" if world > 1 else "1 GPU"},
        "gmres_iterations": iters[-1], "max_err_vs_exact": err,
        "refine_steps_per_solve": refine[-1],
        "setup_ms": setup_ms, "wall_s_timed": wall,
        "box_solve_mpts_s": box_mpts, "box_solve_ms": box_ms,
        "fp64_path": fp64,
        "speedup_vs_fp64": (value / world) / fp64["solves_per_s"] if fp64 else None,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(launches.values())),
        "gpu_launches_by_class": launches,
        "kernel_ms_per_step": {k: v[0] / 2 for k, v in prof.items()},
        "roofline": roof,
    }
    G.close()
    legs = [("config1", args.config1, config1_leg), ("batched", args.batch > 0, batched),
            ("learned", args.learned_n > 0, learned_leg), ("threed", args.threed_n > 0, threed_leg),
            ("neumann", args.neumann_n > 0, neumann_leg), ("hetero", args.hetero_n > 0, hetero_leg),
            ("close", args.close_n2 > 0 or args.close_n3 > 0, close_leg), ("moving", args.moving_n > 0, moving_leg)]
    for name, on, leg in legs:
        if not on:
            continue
        # each leg starts from torch's allocator emptied of the previous legs'
        # blocks (the learned leg's training set alone is ~300 MB), so that a
        # leg's timing does not depend on what ran before it
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out[name] = leg(args, stream, flush)
    if rank == 0 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, budget_s=args.cpu_budget)
    return out


def _star_instances(count, seed, sizes, box_rtol, box_steps, relax=0.0):
    """Seeded star-interface problems (mixed precision); draws whose interface
    the drawn grid cannot resolve (KFBI_ERR_GEOMETRY) are dropped and counted,
    the seeded stream continues."""
    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    inst, redrawn = [], 0
    for w in W.star_batch_2d(count=4 * count, seed=seed, sizes=sizes):
        if len(inst) == count:
            break
        try:
            G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED, box_rtol=box_rtol,
                                           box_max_iters=box_steps, relax=relax)
        except kfbi.KfbiError as e:
            if e.status != 2:
                raise
            redrawn += 1
            continue
        inst.append((w, G))
    return inst, redrawn


def _instance_data(w, G):
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    xyz = torch.zeros((G.nb, w.dim), dtype=torch.float64, device="cuda")
    nrm = torch.zeros((G.nb, w.dim), dtype=torch.float64, device="cuda")
    kfbi.kfbi_dof_points(G.handle, xyz, nrm)
    g1, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
    grid = W.grid_data(w)
    keep = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
            (("g1", g1), ("g2", g2), ("f_in", grid["f_in"]), ("f_out", grid["f_out"]),
             ("lapf_in", grid["lapf_in"]), ("lapf_out", grid["lapf_out"]), ("g_b", grid["g_b"]))}
    return kfbi.make_data(**keep), keep


def batched(args, stream, flush):
    """The batched workload: 64 seeded star-interface problems on grids drawn
    from {128, 256, 512, 1024}^2, all solved by one batched GMRES
    (kfbi_gmres_solve_batch) plus one batched evaluation (kfbi_evaluate_batch).
    Compared with the same instances solved one after another by the plain
    FP64 path and by the mixed path.  Then the learned + mixed + batched form:
    a network trained on other seeded star problems (their own solves) gives
    every instance its start, inside the timed region.  Draws whose
    interface the drawn grid cannot resolve are skipped and counted (the
    seeded stream continues)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    sizes = (128, 256, 512, 1024)
    inst, redrawn = _star_instances(args.batch, 5965, sizes, args.box_rtol, args.box_steps, args.relax_batch)
    rows = []
    for w, G in inst:
        d, keep = _instance_data(w, G)
        rows.append(dict(w=w, G=G, keep=keep, d=d,
                         x=torch.zeros(G.nb, dtype=torch.float64, device="cuda"),
                         x0=torch.zeros(G.nb, dtype=torch.float64, device="cuda"),
                         u=torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")))
    opts = kfbi.GmresOpts(rtol=args.rtol, restart=100, max_iter=100, x0=None)
    B = kfbi.Batch([r["G"] for r in rows])
    datas = [r["d"] for r in rows]
    xs = [r["x"] for r in rows]

    us = [r["u"] for r in rows]

    def step():
        infos = B.gmres_solve(datas, opts, xs)
        B.evaluate(datas, xs, us)
        return infos

    def timed(fn, reps):
        t = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.median(t)

    for _ in range(2):
        infos = step()
    for r in rows:
        kfbi.kfbi_launch_counts(r["G"].handle, reset=True)
    ms_batch = timed(step, max(3, args.steps // 2))
    errs = []
    for r in rows:
        ins = _inside(r["G"], kfbi)
        ex = W.exact_grid(r["w"], ins)
        errs.append(float(np.abs(r["u"].cpu().numpy() - ex)[1:-1, 1:-1].max()))

    def sequential(prec_rows):
        def fn():
            for r, G in prec_rows:
                kfbi.kfbi_gmres_solve(G.handle, r["d"], opts, r["x2"])
                kfbi.kfbi_evaluate(G.handle, r["d"], r["x2"], r["u2"])
        fn()
        return timed(fn, 2)

    for r in rows:
        r["x2"] = torch.zeros_like(r["x"])
        r["u2"] = torch.zeros_like(r["u"])
    ms_mixed_seq = sequential([(r, r["G"]) for r in rows])
    errs_mixed = []
    for r in rows:
        ins = _inside(r["G"], kfbi)
        ex = W.exact_grid(r["w"], ins)
        errs_mixed.append(float(np.abs(r["u2"].cpu().numpy() - ex)[1:-1, 1:-1].max()))
    g64 = [kfbi.Problem.from_workload(r["w"], precision=kfbi.FP64) for r in rows]
    ms_fp64_seq = sequential(list(zip(rows, g64)))
    errs64 = []
    for r in rows:
        ins = _inside(r["G"], kfbi)
        ex = W.exact_grid(r["w"], ins)
        errs64.append(float(np.abs(r["u2"].cpu().numpy() - ex)[1:-1, 1:-1].max()))
    for G in g64:
        G.close()
    ratio = [e / max(e64, 1e-300) for e, e64 in zip(errs, errs64)]

    # ---- learned + mixed + batched: train on other seeded star problems
    learned = None
    if args.batch_learned:
        from paper_2309_05965_gb300 import learned as L
        t0 = time.perf_counter()
        train, _ = _star_instances(args.batch_train, 5966, (128, 256, 512), args.box_rtol, args.box_steps)
        ds = L.Dataset(sum(G.nb for _, G in train))
        topts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=100, x0=None)
        for w, G in train:
            d, keep = _instance_data(w, G)
            x = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
            kfbi.kfbi_gmres_solve(G.handle, d, topts, x)
            ds.add(G, d, x)
            G.close()
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        ws = L.WarmStart(seed=5965)
        hist = ws.fit(ds, epochs=args.learned_epochs, batch=4096, lr=2e-3, lr_final=1e-6,
                      min_steps=args.learned_steps)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        x0s = [r["x0"] for r in rows]

        def measure(rtol_l):
            lopts = kfbi.GmresOpts(rtol=rtol_l, restart=100, max_iter=100, x0=None)

            def step_learned():
                ws.predict_batch(B, datas, x0s)
                infos = B.gmres_solve(datas, lopts, xs, x0s=x0s)
                B.evaluate(datas, xs, us)
                return infos

            for _ in range(2):
                linfos = step_learned()
            ms_learned = timed(step_learned, max(3, args.steps // 2))
            lerrs = []
            for r in rows:
                ins = _inside(r["G"], kfbi)
                ex = W.exact_grid(r["w"], ins)
                lerrs.append(float(np.abs(r["u"].cpu().numpy() - ex)[1:-1, 1:-1].max()))
            worst = sorted(((e / max(e64, 1e-300), r["w"].sigma_in, r["w"].n, i.iters)
                            for e, e64, r, i in zip(lerrs, errs64, rows, linfos)), reverse=True)[:3]
            # start quality: relative max difference of the start from the solved density
            start_err = [float((r["x0"] - r["x"]).abs().max() / r["x"].abs().max()) for r in rows]
            return {"gmres_rtol": rtol_l, "solves_per_s": len(rows) / (ms_learned * 1e-3),
                    "ms_per_batch": ms_learned, "speedup_vs_fp64_sequential": ms_fp64_seq / ms_learned,
                    "speedup_vs_batched_zero_start": ms_batch / ms_learned,
                    "gmres_iterations": [i.iters for i in linfos],
                    "x0_rejected": sum(i.x0_rejected for i in linfos),
                    "max_err_ratio_vs_fp64": max(e / max(e64, 1e-300) for e, e64 in zip(lerrs, errs64)),
                    "worst_err_ratios": [{"ratio": a, "contrast": b, "n": c, "iters": d}
                                         for a, b, c, d in worst],
                    "start_rel_err_median": statistics.median(start_err),
                    "start_rel_err_max": max(start_err)}

        learned = {"same_rtol": measure(args.rtol), "rtol_tenth": measure(args.rtol / 10),
                   "train": {"solves": ds.solves, "samples": ds.n, "data_s": t_data, "train_s": t_train,
                             "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                             "workload": f"{ds.solves} star problems drawn with seed 5966 on "
                                         "{128,256,512}^2, GMRES rtol 1e-10"},
                   "note": "starts from one batched forward pass (kfbi_warm_start_batch) inside the "
                           "timed region; the learned path measured at the zero start's GMRES "
                           "tolerance and one decade tighter"}
        ws.close()
    nsz = {}
    for r in rows:
        nsz[r["w"].n] = nsz.get(r["w"].n, 0) + 1
    out = {"workload": f"{len(rows)} star-interface problems, grids {nsz}, contrast 10^U[0,3], "
                       f"GMRES rtol {args.rtol:g}",
           "instances": len(rows), "redrawn_unresolved": redrawn, "relax": args.relax_batch,
           "solves_per_s": len(rows) / (ms_batch * 1e-3), "ms_per_batch": ms_batch,
           "fp64_sequential_solves_per_s": len(rows) / (ms_fp64_seq * 1e-3),
           "mixed_sequential_solves_per_s": len(rows) / (ms_mixed_seq * 1e-3),
           "speedup_vs_fp64_sequential": ms_fp64_seq / ms_batch,
           "gmres_iterations": [i.iters for i in infos],
           "max_err_vs_exact": max(errs), "max_err_ratio_vs_fp64": max(ratio),
           "max_err_ratio_mixed_sequential_vs_fp64": max(e / max(e64, 1e-300)
                                                         for e, e64 in zip(errs_mixed, errs64)),
           "fp64_max_err_vs_exact": max(errs64),
           "tuned_tiles": dict(zip(("pass_ctas", "row_ctas"), B.tiles())),
           "learned": learned}
    B.close()
    for r in rows:
        r["G"].close()
    return out


def learned_leg(args, stream, flush):
    """Learned initial density on the wave-field ellipsoid family (random
    axes, fixed non-polynomial harmonic fields inside and outside, contrast
    10): train the network on the library's own solves of
    --learned-geometries ellipsoids (seed 5966) on a 64^3 grid (draws the grid
    cannot resolve are skipped and counted), then on held-out ellipsoids
    (seed 5967) at --learned-n^3 compare the plain FP64 path, the mixed path
    from zero and the mixed path from the learned start (the prediction is
    inside the timed region)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi, learned

    t0 = time.perf_counter()
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=100, x0=None)
    axes_train = W.ellipsoid_axes(5966, args.learned_geometries)
    # at 64^3 an ellipsoid with axes <= 0.7 has fewer than 12000 DOFs
    ds = learned.Dataset(len(axes_train) * 12000)
    skipped = 0
    # one problem moved from ellipsoid to ellipsoid (kfbi_update_levelset);
    # the fields, and so the grid data, are the same for every geometry
    w0 = W.wave_ellipsoid_3d(axes_train[0], 64)
    grid = W.grid_data(w0)
    gkeep = {k: torch.from_numpy(np.ascontiguousarray(grid[k])).cuda()
             for k in ("f_in", "f_out", "lapf_in", "lapf_out", "g_b")}
    G = None
    for axes in axes_train:
        w = W.wave_ellipsoid_3d(axes, 64)
        try:
            if G is None:
                G = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
            else:
                G.update_levelset(w.ls_kind, w.ls_params)
        except kfbi.KfbiError as e:
            if e.status != 2:
                raise
            skipped += 1
            continue
        xyz = torch.zeros((G.nb, 3), dtype=torch.float64, device="cuda")
        nrm = torch.zeros_like(xyz)
        kfbi.kfbi_dof_points(G.handle, xyz, nrm)
        g1, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
        g1t, g2t = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
        d = kfbi.make_data(g1=g1t, g2=g2t, **gkeep)
        x = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
        kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
        ds.add(G, d, x)
    if G is not None:
        G.close()
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    ws = learned.WarmStart(seed=5965)
    hist = ws.fit(ds, epochs=args.learned_epochs, batch=8192, lr=2e-3, lr_final=1e-6,
                  min_steps=args.learned_steps)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    n = args.learned_n
    eopts = kfbi.GmresOpts(rtol=args.rtol, restart=100, max_iter=100, x0=None)
    rows = {"fp64_zero": [], "mixed_zero": [], "mixed_learned": [], "mixed_learned_rtol_tenth": []}
    start_err = []
    for axes in W.ellipsoid_axes(5967, args.learned_eval):
        w = W.wave_ellipsoid_3d(axes, n)
        Gm = kfbi.Problem.from_workload(w, precision=kfbi.MIXED, box_rtol=args.box_rtol, relax=args.relax_3d)
        G64 = kfbi.Problem.from_workload(w, precision=kfbi.FP64)
        x = torch.zeros(Gm.nb, dtype=torch.float64, device="cuda")
        x0 = torch.zeros_like(x)
        u = torch.zeros(Gm.grid_shape, dtype=torch.float64, device="cuda")
        ins = _inside(Gm, kfbi)
        d, keep = _instance_data(w, Gm)
        ex = W.exact_grid(w, ins)
        for name, G, use, rt in (("fp64_zero", G64, False, args.rtol), ("mixed_zero", Gm, False, args.rtol),
                                 ("mixed_learned", Gm, True, args.rtol),
                                 ("mixed_learned_rtol_tenth", Gm, True, args.rtol / 10)):
            def run():
                o = eopts
                if use:
                    ws.predict(G, d, x0)
                    o = kfbi.GmresOpts(rtol=rt, restart=100, max_iter=100, x0=x0.data_ptr())
                info = kfbi.kfbi_gmres_solve(G.handle, d, o, x)
                kfbi.kfbi_evaluate(G.handle, d, x, u)
                return info
            run()
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = run()
            e1.record(stream)
            e1.synchronize()
            err = float(np.abs(u.cpu().numpy() - ex)[1:-1, 1:-1, 1:-1].max())
            rows[name].append((e0.elapsed_time(e1), info.iters, err, info.x0_rejected))
            if use and rt == args.rtol:
                start_err.append(float((x0 - x).abs().max() / x.abs().max()))
        Gm.close()
        G64.close()
    ws.close()

    def agg(r):
        ms = statistics.mean(v[0] for v in r)
        return {"solves_per_s": 1e3 / ms, "ms_per_solve": ms,
                "gmres_iterations": [v[1] for v in r], "max_err_vs_exact": max(v[2] for v in r),
                "x0_rejected": sum(v[3] for v in r)}
    out = {k: agg(v) for k, v in rows.items()}
    out["workload"] = (f"ellipsoid interface 3D, N={n}, contrast 10, fixed non-polynomial harmonic fields "
                       f"inside and outside; network 3 layers x 256 trained on {ds.solves} solves of other "
                       f"ellipsoids at 64^3 ({ds.n} DOF samples, {skipped} unresolved draws skipped), "
                       f"GMRES rtol {args.rtol:g}")
    out["start_rel_err"] = start_err
    out["relax_mixed"] = args.relax_3d
    out["train"] = {"data_s": t_data, "train_s": t_train, "loss_first_epoch": hist[0],
                    "loss_last_epoch": hist[-1], "epochs": len(hist)}
    out["speedup_learned_mixed_vs_fp64_zero"] = (out["mixed_learned"]["solves_per_s"]
                                                 / out["fp64_zero"]["solves_per_s"])
    out["speedup_learned_vs_mixed_zero"] = (out["mixed_learned"]["solves_per_s"]
                                            / out["mixed_zero"]["solves_per_s"])
    out["err_ratio_learned_vs_fp64"] = (out["mixed_learned"]["max_err_vs_exact"]
                                        / max(out["fp64_zero"]["max_err_vs_exact"], 1e-300))
    out["speedup_learned_rtol_tenth_vs_fp64_zero"] = (out["mixed_learned_rtol_tenth"]["solves_per_s"]
                                                      / out["fp64_zero"]["solves_per_s"])
    out["err_ratio_learned_rtol_tenth_vs_fp64"] = (out["mixed_learned_rtol_tenth"]["max_err_vs_exact"]
                                                   / max(out["fp64_zero"]["max_err_vs_exact"], 1e-300))
    return out


def threed_leg(args, stream, flush):
    """The 3D Dirichlet problem for modified Helmholtz (kappa = 1) with the
    torus interface, u = e^(x+y+z)/10, 4th order, at --threed-n^3: geometric
    multigrid (FP32 V(2,2) cycles, exact fixed-point residuals), the mixed DST
    path and the plain FP64 DST path, each to GMRES rtol --rtol; plus the
    multigrid's achieved bandwidth over one box solve."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    n = args.threed_n
    w = W.torus_helmholtz_3d(n)
    grid = W.grid_data(w)
    out = {"workload": f"torus Dirichlet 3D, N={n}, kappa=1, u=exp(x+y+z)/10, 4th order, "
                       f"GMRES rtol {args.rtol:g}", "relax_mixed_dst": args.relax_3d}
    opts = kfbi.GmresOpts(rtol=args.rtol, restart=100, max_iter=200, x0=None)
    npts = (n - 1) ** 3
    for name, box, prec in (("mg_mixed", kfbi.BOX_MG, kfbi.MIXED), ("dst_mixed", kfbi.BOX_DST, kfbi.MIXED),
                            ("dst_fp64", kfbi.BOX_DST, kfbi.FP64)):
        t0 = time.perf_counter()
        G = kfbi.Problem.from_workload(w, box_solver=box, precision=prec,
                                       box_max_iters=args.box_steps if prec == kfbi.MIXED else 0,
                                       relax=args.relax_3d if prec == kfbi.MIXED else 0.0)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        xyz = torch.zeros((G.nb, 3), dtype=torch.float64, device="cuda")
        nrm = torch.zeros_like(xyz)
        kfbi.kfbi_dof_points(G.handle, xyz, nrm)
        g1, _ = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
        keep = {"g1": torch.from_numpy(g1).cuda(),
                "f_in": torch.from_numpy(np.ascontiguousarray(grid["f_in"])).cuda(),
                "lapf_in": torch.from_numpy(np.ascontiguousarray(grid["lapf_in"])).cuda()}
        d = kfbi.make_data(**keep)
        x = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
        u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")

        def step():
            info = kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
            kfbi.kfbi_evaluate(G.handle, d, x, u)
            return info
        step()
        ts = []
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ins = _inside(G, kfbi)
        err = float(np.abs(u.cpu().numpy() - W.exact_grid(w, ins))[ins].max())
        rhs = torch.randn(G.grid_shape, dtype=torch.float64, device="cuda")
        ub = torch.zeros_like(rhs)
        kfbi.kfbi_box_solve(G.handle, rhs, ub)
        bt = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kfbi.kfbi_box_solve(G.handle, rhs, ub)
            e1.record(stream)
            e1.synchronize()
            bt.append(e0.elapsed_time(e1))
        box_ms = statistics.median(bt)
        r = {"solves_per_s": 1e3 / statistics.median(ts), "ms_per_solve": statistics.median(ts),
             "gmres_iterations": info.iters, "max_err_vs_exact": err, "setup_s": setup, "n_b": G.nb,
             "box_solve_ms": box_ms, "box_solve_mpts_s": npts / (box_ms * 1e-3) / 1e6}
        if box == kfbi.BOX_MG:
            # per-class device time of one box solve; V(2,2) algorithmic traffic per
            # fine point per cycle: 4 sweeps x 12 B + residual 12 B + restriction 4.5 B
            # + prolongation 8 B = 72.5 B, x 8/7 for the coarser levels (FP32)
            kfbi.kfbi_profile_enable(G.handle, True)
            kfbi.kfbi_box_solve(G.handle, rhs, ub)
            prof = kfbi.kfbi_profile_read(G.handle)
            kfbi.kfbi_profile_enable(G.handle, False)
            mg_ms, mg_launches = prof["mg"]
            steps, cycles, _, _ = kfbi.kfbi_box_solve_info(G.handle)
            achieved = npts * 72.5 * 8 / 7 * cycles / (mg_ms * 1e-3) / 1e9
            peak = measured_peaks().get("hbm_gbs", 6800.0)
            r["mg_roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                "frac": achieved / peak, "cycles": cycles, "outer_steps": steps,
                                "mg_ms": mg_ms, "launches": mg_launches,
                                "note": "cycles that ran (device counters); 82.9 B per fine point "
                                        "per V(2,2) cycle (FP32)"}
        else:
            steps, _, _, _ = kfbi.kfbi_box_solve_info(G.handle)
            peak = measured_peaks().get("hbm_gbs", 6800.0)
            achieved = 16.0 * npts / (box_ms * 1e-3) / 1e9
            r["box_roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                 "frac": achieved / peak, "steps": steps,
                                 "note": "16 B per interior point per box solve (FP64 R in, u out) "
                                         "over the whole box solve's time"}
        out[name] = r
        G.close()
    out["speedup_mixed_dst_vs_fp64"] = out["dst_mixed"]["solves_per_s"] / out["dst_fp64"]["solves_per_s"]
    out["err_ratio_mg_mixed_vs_fp64"] = out["mg_mixed"]["max_err_vs_exact"] / out["dst_fp64"]["max_err_vs_exact"]
    return out


# Sec. 7.2.1, Table 3: the paper's Neumann torus (N, N_b, GMRES iterations at
# tolerance 1e-10, RMS and maximum error, CPU seconds on the paper's machine)
PAPER_TABLE3 = {128: (24656, 21, 2.76e-05, 7.97e-05, 6.35), 256: (98668, 18, 2.38e-06, 5.98e-06, 25.0),
                512: (394548, 17, 1.68e-07, 4.01e-07, 135.0)}


def neumann_leg(args, stream, flush):
    """The paper's 3D Neumann Poisson problem on the torus (Sec. 7.2.1) at
    --neumann-n^3: mixed and FP64 DST box solves, GMRES to the paper's
    tolerance 1e-10 with the zero-mean projection, then the grid solution;
    errors with their mean over Omega removed (the solution is fixed up to a
    constant), beside the paper's Table 3 row."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    n = args.neumann_n
    w = W.neumann_torus_3d(n)
    grid = W.grid_data(w)
    out = {"workload": f"torus Neumann 3D (Sec. 7.2.1), N={n}, kappa=0, u=exp(z)(cos 2x + cos 3y), "
                       f"4th order, GMRES rtol 1e-10", "relax_mixed": args.relax_3d}
    if n in PAPER_TABLE3:
        nb, it, e2, einf, cpu_s = PAPER_TABLE3[n]
        out["paper"] = {"n_b": nb, "gmres_iterations": it, "e2": e2, "einf": einf, "cpu_s": cpu_s}
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=200, x0=None)
    for name, prec in (("dst_mixed", kfbi.MIXED), ("dst_fp64", kfbi.FP64)):
        G = kfbi.Problem.from_workload(w, precision=prec,
                                       box_max_iters=args.box_steps if prec == kfbi.MIXED else 0,
                                       relax=args.relax_3d if prec == kfbi.MIXED else 0.0)
        xyz = torch.zeros((G.nb, 3), dtype=torch.float64, device="cuda")
        nrm = torch.zeros_like(xyz)
        kfbi.kfbi_dof_points(G.handle, xyz, nrm)
        _, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
        keep = {"g2": torch.from_numpy(g2).cuda(),
                "f_in": torch.from_numpy(np.ascontiguousarray(grid["f_in"])).cuda(),
                "lapf_in": torch.from_numpy(np.ascontiguousarray(grid["lapf_in"])).cuda()}
        d = kfbi.make_data(**keep)
        x = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
        u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")

        def step():
            info = kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
            kfbi.kfbi_evaluate(G.handle, d, x, u)
            return info
        step()
        ts = []
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ins = _inside(G, kfbi)
        e = (u.cpu().numpy() - W.exact_grid(w, ins))[ins]
        e = e - e.mean()
        out[name] = {"solves_per_s": 1e3 / statistics.median(ts), "ms_per_solve": statistics.median(ts),
                     "gmres_iterations": info.iters, "einf": float(np.abs(e).max()),
                     "e2": float(np.sqrt(np.mean(e * e))), "n_b": G.nb,
                     "kernel_ms_by_class": _class_profile(G, kfbi, step)}
        G.close()
    out["speedup_mixed_vs_fp64"] = out["dst_mixed"]["solves_per_s"] / out["dst_fp64"]["solves_per_s"]
    out["err_ratio_mixed_vs_fp64"] = out["dst_mixed"]["einf"] / out["dst_fp64"]["einf"]
    return out


def hetero_leg(args, stream, flush):
    """The general interface system (eq. (bie-ifp-1)) with Sec. 7.2.5's
    heterogeneous coefficients and spheres (radius 0.7, 0.0142 apart: stencils
    join two spheres) at --hetero-n^3: two box solves per operator
    application over 2 N_b unknowns, mixed and FP64 DST, GMRES to the paper's
    tolerance 1e-10, errors on each side of the interfaces."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    n = args.hetero_n
    w = W.hetero_spheres_3d(n, radius=0.7)
    grid = W.grid_data(w)
    out = {"workload": f"Sec. 7.2.5's three spheres r=0.7 (0.0142 apart) in [-1.5,1.5]^3, N={n}, "
                       f"sigma 1/4, kappa 0/10, general interface system, 4th order, GMRES rtol 1e-10",
           "relax_mixed": args.relax_3d}
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=200, x0=None)
    for name, prec in (("dst_mixed", kfbi.MIXED), ("dst_fp64", kfbi.FP64)):
        G = kfbi.Problem.from_workload(w, precision=prec,
                                       box_max_iters=args.box_steps if prec == kfbi.MIXED else 0,
                                       relax=args.relax_3d if prec == kfbi.MIXED else 0.0)
        xyz = torch.zeros((G.nb, 3), dtype=torch.float64, device="cuda")
        nrm = torch.zeros_like(xyz)
        kfbi.kfbi_dof_points(G.handle, xyz, nrm)
        g1, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
        keep = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
                (("g1", g1), ("g2", g2), ("f_in", grid["f_in"]), ("f_out", grid["f_out"]),
                 ("lapf_in", grid["lapf_in"]), ("lapf_out", grid["lapf_out"]), ("g_b", grid["g_b"]))}
        d = kfbi.make_data(**keep)
        x = torch.zeros(2 * G.nb, dtype=torch.float64, device="cuda")
        u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")

        def step():
            info = kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
            kfbi.kfbi_evaluate(G.handle, d, x, u)
            return info
        step()
        ts = []
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ins = _inside(G, kfbi)
        e = np.abs(u.cpu().numpy() - W.exact_grid(w, ins))
        inner = np.zeros_like(ins)
        inner[1:-1, 1:-1, 1:-1] = True
        out[name] = {"solves_per_s": 1e3 / statistics.median(ts), "ms_per_solve": statistics.median(ts),
                     "gmres_iterations": info.iters, "einf_inside": float(e[inner & ins].max()),
                     "einf_outside": float(e[inner & ~ins].max()), "n_b": G.nb,
                     "kernel_ms_by_class": _class_profile(G, kfbi, step)}
        G.close()
    out["speedup_mixed_vs_fp64"] = out["dst_mixed"]["solves_per_s"] / out["dst_fp64"]["solves_per_s"]
    out["err_ratio_mixed_vs_fp64"] = max(
        out["dst_mixed"][k] / out["dst_fp64"][k] for k in ("einf_inside", "einf_outside"))
    return out


def _solve_labels(w, prec, args, flush, stream, reps=3):
    """One workload solved end to end on device-resident data (GMRES to
    1e-10 and evaluation), timed over `reps` steps with L2 flushed before
    each: ms per solve, iterations, N_b and the max error per side label."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    mixed = prec == kfbi.MIXED
    relax = (args.relax_3d if w.dim == 3 else args.relax) if mixed else 0.0
    G = kfbi.Problem.from_workload(w, precision=prec, box_max_iters=args.box_steps if mixed else 0,
                                   relax=relax)
    xyz = torch.zeros((G.nb, w.dim), dtype=torch.float64, device="cuda")
    nrm = torch.zeros_like(xyz)
    ifc = torch.zeros(G.nb, dtype=torch.int32, device="cuda")
    kfbi.kfbi_dof_points(G.handle, xyz, nrm)
    kfbi.kfbi_dof_iface(G.handle, ifc)
    g1, g2 = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy(), ifc.cpu().numpy())
    grid = W.grid_data(w)
    keep = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
            (("g1", g1), ("g2", g2), ("f_in", grid["f_in"]), ("f_out", grid["f_out"]),
             ("lapf_in", grid["lapf_in"]), ("lapf_out", grid["lapf_out"]), ("g_b", grid["g_b"]))}
    d = kfbi.make_data(**keep, in_per_interface=grid["f_in"].ndim == w.dim + 1)
    nx = 2 * G.nb if w.kind == W.KIND_INTERFACE_GENERAL else G.nb
    x = torch.zeros(nx, dtype=torch.float64, device="cuda")
    u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=300, x0=None)

    def step():
        info = kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
        kfbi.kfbi_evaluate(G.handle, d, x, u)
        return info
    step()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    lab = torch.zeros(G.grid_shape, dtype=torch.uint8, device="cuda")
    kfbi.kfbi_inside_mask(G.handle, lab)
    lab = lab.cpu().numpy()
    e = np.abs(u.cpu().numpy() - W.exact_grid(w, lab))
    inner = np.zeros(e.shape, dtype=bool)
    inner[tuple(slice(1, w.n) for _ in range(w.dim))] = True
    errs = {int(l): float(e[inner & (lab == l)].max()) for l in np.unique(lab)}
    res = {"ms_per_solve": statistics.median(ts), "solves_per_s": 1e3 / statistics.median(ts),
           "gmres_iterations": info.iters, "n_b": G.nb, "n_entries": G.nent, "relax": relax,
           "einf_by_label": errs}
    G.close()
    return res


def close_leg(args, stream, flush):
    """Close and touching interfaces (the remark on arbitrarily close
    interfaces in Sec. 5.2): Sec. 7.1.2's eight circles and star (Table 2) at
    --close-n2^2 and Sec. 7.2.4's torus and ellipsoid touching along a circle
    (Table 6) at --close-n3^3, mixed and FP64 DST, GMRES to 1e-10, with the
    paper's numbers for the same grids (its CPU times on its own machine).
    A size of 0 leaves its case out."""
    import json as _json
    import pathlib

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    gold = pathlib.Path(__file__).parent / "tests" / "golden"
    t2 = _json.loads((gold / "paper_table2.json").read_text())["rows"]
    t6 = _json.loads((gold / "paper_table6.json").read_text())["rows"]
    out = {}
    cases = []
    if args.close_n2 > 0:
        cases.append(("table2", W.touching_interfaces_2d(args.close_n2), t2))
    if args.close_n3 > 0:
        cases.append(("table6", W.torus_ellipsoid_3d(args.close_n3), t6))
    for key, w, table in cases:
        rec = {"workload": f"{w.name}, N={w.n}, mu-form interface problem, sigma_i 1 / sigma_e 3, "
                           f"4th order, GMRES rtol 1e-10",
               "paper": table.get(str(w.n))}
        for name, prec in (("dst_mixed", kfbi.MIXED), ("dst_fp64", kfbi.FP64)):
            rec[name] = _solve_labels(w, prec, args, flush, stream)
        rec["speedup_mixed_vs_fp64"] = rec["dst_mixed"]["solves_per_s"] / rec["dst_fp64"]["solves_per_s"]
        out[key] = rec
    return out


def _class_profile(G, kfbi, step):
    """Device time and launches per kernel class over one more step, from the
    library's per-launch CUDA events (launches serialised by the events)."""
    kfbi.kfbi_profile_enable(G.handle, True)
    step()
    prof = kfbi.kfbi_profile_read(G.handle)
    kfbi.kfbi_profile_enable(G.handle, False)
    return {k: {"ms": round(v[0], 4), "launches": int(v[1])} for k, v in prof.items() if v[1] > 0}


def _inside(G, kfbi):
    import torch
    m = torch.zeros(G.grid_shape, dtype=torch.uint8, device="cuda")
    kfbi.kfbi_inside_mask(G.handle, m)
    return m.cpu().numpy().astype(bool)


# DRAM bytes (read + write) per launch of the three FP32 passes of a
# correction step at the 2D N = 1024 workload with 3 refinement steps, from
# one ncu capture of the current kernels (profiles/k_dst32_k_res_fix2_flower1024.md;
# cold cache: ncu flushes L2 before each replay, in the timed loop the grids
# stay in L2); None once the kernels change
NCU_DST_BYTES_PER_LAUNCH_1024 = (4.279e6 + 4.285e6 + 12.667e6) / 3


def roofline(args, G, prof, prec, box_steps=None):
    """Roofline of the box solve's transform passes (the dominant kernel class).

    Algorithmic bytes: one box solve reads the FP64 right-hand side and writes
    the FP64 solution once, 16 B per interior point (the minimum a box solve
    can move).  A box solve is `passes` launches of the class (3 per FP32
    solve in 2D, times the refinement steps that ran), so a launch's share is
    16 (N-1)^d / passes bytes; achieved = that / the class's average launch
    duration (per-launch CUDA events of the profiling pass on the library's
    stream).  The bytes the passes actually stream (the implementation's
    intermediate FP32/int64 grids, counted pass by pass) and the ncu DRAM
    bytes per launch go in `pass_bytes` and `traffic`."""
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    n = args.n
    npts = (n - 1) ** 2
    ms, launches = prof["dst"]
    per_launch_ms = ms / max(1, launches)
    if prec:
        # launches enqueued per box solve: 3 per FP32 solve for every step the
        # solver may take (steps stopped by the convergence flag still launch
        # and return at once, so the class time per box solve is the average
        # launch times this count)
        s = args.box_steps or 5
        # pass by pass: first FP32 solve FP64 R in -> FP32 (12), FP32 -> FP32
        # (8), -> FP32 u0 (8); each refinement step FP32 r in (8), FP32 (8),
        # FP32 + int64 u_fix read and written (20); the FP64 solution once (8)
        pass_bytes, passes = 28 + 36 * (s - 1) + 8, 3 * s
    else:
        s = 1
        pass_bytes, passes = 48, 3
    alg_launch = 16.0 * npts / passes
    achieved = alg_launch / (per_launch_ms * 1e-3) / 1e9
    r = {"kernel": "dst (k_dst32 FP32 transform passes)" if prec else "dst (k_dst_pass FP64)",
         "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
         "traffic": None,
         "algorithmic_bytes_per_launch": alg_launch, "launches_per_box_solve": passes,
         "box_solve_dst_us": per_launch_ms * passes * 1e3, "steps_run": box_steps,
         "avg_launch_us": per_launch_ms * 1e3,
         "pass_bytes_per_point": pass_bytes,
         "pass_bytes_per_launch": pass_bytes * npts / passes,
         "note": "peak of measured (MEASURED_PEAKS.json hbm_gbs); algorithmic bytes 16 B per interior "
                 "point per box solve (FP64 R in, u out)"}
    if prec and n == 1024 and s == 3 and NCU_DST_BYTES_PER_LAUNCH_1024:
        r["traffic"] = NCU_DST_BYTES_PER_LAUNCH_1024
        r["traffic_vs_algorithmic"] = NCU_DST_BYTES_PER_LAUNCH_1024 / alg_launch
        r["traffic_note"] = ("bytes per launch, ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                             "cold cache")
    return r


def cpu_baseline(args, budget_s=20.0):
    """The oracle as it stands on the host cores, run twice in fresh
    processes (BLAS and FFT thread counts are fixed at import): with one
    thread and with every core.  Each run times the stages of the GPU path on
    the same workload (box solve, one operator application, full solves,
    set-up excluded) and the 64^2 Dirichlet solve; `value` is the all-cores
    full-solve rate."""
    runs = {}
    for threads in (1, os.cpu_count() or 1):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-stages", str(threads), "--n", str(args.n),
               "--rtol", repr(args.rtol), "--cpu-budget", repr(budget_s / 2)]
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            raise RuntimeError("CPU oracle run failed:\n" + r.stdout[-2000:] + r.stderr[-2000:])
        runs[threads] = json.loads(r.stdout.strip().splitlines()[-1])
    allc = runs[max(runs)]
    one = runs[1]
    return {"value": allc["solves_per_s"], "unit": "solves/s", "cores": max(runs), "kind": "oracle",
            "sample": f"{allc['solves']} full oracle solves of the same workload (N={args.n}), set-up "
                      f"excluded, NumPy/SciPy with {max(runs)} BLAS/FFT threads; box solve and operator "
                      "application timed alone",
            "host": os.uname().machine, "cpu_count": os.cpu_count(),
            "all_cores": allc, "single_thread": one}


def cpu_stages(args):
    """Child process of cpu_baseline: the oracle's stages with the BLAS/FFT
    thread count given (environment set by the parent), one JSON line."""
    import numpy as np
    import scipy.fft

    import workloads as W
    from oracle import kfbi as OK
    threads = args.cpu_stages
    out = {"threads": threads}
    with scipy.fft.set_workers(threads):
        w = workload(args.n)
        t0 = time.perf_counter()
        P = OK.Problem(w)
        out["setup_s"] = time.perf_counter() - t0
        data = W.grid_data(w)
        g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
        rng = np.random.default_rng(0)
        R = W.sine_grid_rhs(2, args.n, 1)
        x = rng.standard_normal(P.nb)

        def med(fn, k):
            ts = []
            for _ in range(k):
                t = time.perf_counter()
                fn()
                ts.append(time.perf_counter() - t)
            return statistics.median(ts)
        box_s = med(lambda: P.box_solve(R), 3)
        out["box_solve_ms"] = box_s * 1e3
        out["box_solve_mpts_s"] = (args.n - 1) ** 2 / box_s / 1e6
        out["apply_ms"] = med(lambda: P.apply(x), 3) * 1e3
        t0 = time.perf_counter()
        count = 0
        while True:
            P.solve(g1, g2, data, rtol=args.rtol)
            count += 1
            if time.perf_counter() - t0 > args.cpu_budget or count >= 5:
                break
        el = time.perf_counter() - t0
        out["solves"] = count
        out["solves_per_s"] = count / el
        # the 64^2 Dirichlet BVP (ellipse, u = e^x sin y, FP64, rtol 1e-10)
        w1 = W.ellipse_dirichlet_2d(64)
        P1 = OK.Problem(w1)
        d1 = W.grid_data(w1)
        h1, h2 = W.boundary_data(w1, P1.surf.x, P1.surf.n)
        out["ellipse64_solve_ms"] = med(lambda: P1.solve(h1, h2, d1, rtol=1e-10), 5) * 1e3
    print(json.dumps(out))


def moving_leg(args, stream, flush):
    """A moving interface (the level-set method of the paper's closing
    remarks): the interface problem of sampled_interface_2d whose shape moves
    and turns over --moving-steps positions (moving_samples, t = 0.05 k), at
    --moving-n^2, mixed DST.  Each step takes the interface's node values
    (already on the device), sets the problem up for them
    (kfbi_update_levelset), computes the jump data at the new DOFs on the host
    from their coordinates, and solves to rtol 1e-8 with evaluation.  Timed by
    the host clock with the device synchronised, against the same steps with
    a new problem created (and destroyed) per position."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    n, T = args.moving_n, args.moving_steps
    ts = [0.05 * k for k in range(T)]
    samples = [torch.from_numpy(W.moving_samples(2, n, -1.0, 1.0, t)).cuda() for t in ts]
    w0 = W.moving_interface_2d(n, 0.0)
    grid = W.grid_data(w0)      # f and g_b do not depend on the interface's position
    gkeep = {k: torch.from_numpy(np.ascontiguousarray(grid[k])).cuda()
             for k in ("f_in", "f_out", "lapf_in", "lapf_out", "g_b")}
    opts = kfbi.GmresOpts(rtol=args.rtol, restart=100, max_iter=200, x0=None)
    kw = dict(precision=kfbi.MIXED, box_max_iters=args.box_steps, box_rtol=args.box_rtol, relax=args.relax)

    def step(G, k, errs, its):
        xyz = torch.zeros((G.nb, 2), dtype=torch.float64, device="cuda")
        nrm = torch.zeros_like(xyz)
        kfbi.kfbi_dof_points(G.handle, xyz, nrm)
        g1, g2 = W.boundary_data(w0, xyz.cpu().numpy(), nrm.cpu().numpy())
        g1t, g2t = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()   # alive through the solve
        d = kfbi.make_data(g1=g1t, g2=g2t, **gkeep)
        x = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
        u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")
        info = kfbi.kfbi_gmres_solve(G.handle, d, opts, x)
        kfbi.kfbi_evaluate(G.handle, d, x, u)
        del g1t, g2t
        its.append(info.iters)
        if errs is not None:
            wk = W.moving_interface_2d(n, ts[k])
            errs.append(float(np.abs(u.cpu().numpy() - W.exact_grid(wk, _inside(G, kfbi)))[1:-1, 1:-1].max()))

    out = {"workload": f"moving interface 2D (moving_samples, {T} positions), N={n}, contrast 10, "
                       f"4th order, mixed DST, GMRES rtol {args.rtol:g}"}
    # correctness pass (untimed): errors against the exact solution at every position
    G = kfbi.Problem.from_workload(w0, **kw)
    errs, its = [], []
    for k in range(T):
        G.update_levelset(W.LS_GRID, [], samples[k])
        step(G, k, errs, its)
    out["max_err_vs_exact"] = max(errs)
    out["gmres_iterations"] = its
    # timed: update per position
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_setup = 0.0
    its = []
    for k in range(T):
        s0 = time.perf_counter()
        G.update_levelset(W.LS_GRID, [], samples[k])
        t_setup += time.perf_counter() - s0
        step(G, k, None, its)
    torch.cuda.synchronize()
    t_upd = time.perf_counter() - t0
    nb = G.nb
    G.close()
    # timed: a new problem per position
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_create = 0.0
    for k in range(T):
        s0 = time.perf_counter()
        Gk = kfbi.Problem(2, n, -1.0, 1.0, W.LS_GRID, [], W.KIND_INTERFACE_MU, sigma_in=w0.sigma_in,
                          sigma_out=w0.sigma_out, ls_samples=samples[k], **kw)
        t_create += time.perf_counter() - s0
        step(Gk, k, None, [])
        Gk.close()
    torch.cuda.synchronize()
    t_new = time.perf_counter() - t0
    out.update({"steps": T, "n_b_last": nb,
                "update": {"steps_per_s": T / t_upd, "ms_per_step": 1e3 * t_upd / T,
                           "setup_ms_per_step": 1e3 * t_setup / T},
                "create_per_step": {"steps_per_s": T / t_new, "ms_per_step": 1e3 * t_new / T,
                                    "setup_ms_per_step": 1e3 * t_create / T},
                "note": "host clock around whole steps (set-up, jump data on the host from the new DOFs, "
                        "solve, evaluation); samples resident on the device"})
    out["speedup_update_vs_create"] = t_new / t_upd
    return out


def config1_leg(args, stream, flush):
    """The 2D interior Dirichlet BVP on the ellipse x^2/0.36 + y^2/0.16 < 1,
    u = e^x sin y, 64^2 grid, 4th order, FP64 DST, GMRES rtol 1e-10.  About
    100 DOFs and a 63^2 box: latency-bound, so reported as microseconds per
    solve, per GMRES iteration, per operator application and per box solve
    (CUDA events, median over repetitions, L2 flushed before each)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2309_05965_gb300 import kfbi
    w = W.ellipse_dirichlet_2d(64)
    G = kfbi.Problem.from_workload(w, box_solver=kfbi.BOX_DST, precision=kfbi.FP64)
    xyz = torch.zeros((G.nb, 2), dtype=torch.float64, device="cuda")
    nrm = torch.zeros_like(xyz)
    kfbi.kfbi_dof_points(G.handle, xyz, nrm)
    g1, _ = W.boundary_data(w, xyz.cpu().numpy(), nrm.cpu().numpy())
    grid = W.grid_data(w)
    keep = {"g1": torch.from_numpy(g1).cuda(),
            "f_in": torch.from_numpy(np.ascontiguousarray(grid["f_in"])).cuda(),
            "lapf_in": torch.from_numpy(np.ascontiguousarray(grid["lapf_in"])).cuda()}
    d = kfbi.make_data(**keep)
    x = torch.zeros(G.nb, dtype=torch.float64, device="cuda")
    u = torch.zeros(G.grid_shape, dtype=torch.float64, device="cuda")
    opts = kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=200, x0=None)
    rhs = torch.randn(G.grid_shape, dtype=torch.float64, device="cuda")
    ub = torch.zeros_like(rhs)
    y = torch.zeros_like(x)
    xr = torch.randn_like(x)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts) * 1e3

    infos = []

    def solve():
        infos.append(kfbi.kfbi_gmres_solve(G.handle, d, opts, x))
        kfbi.kfbi_evaluate(G.handle, d, x, u)

    for _ in range(5):
        solve()
    solve_us = timed(solve, 50)
    gmres_us = timed(lambda: infos.append(kfbi.kfbi_gmres_solve(G.handle, d, opts, x)), 50)
    apply_us = timed(lambda: kfbi.kfbi_apply_operator(G.handle, xr, y), 50)
    box_us = timed(lambda: kfbi.kfbi_box_solve(G.handle, rhs, ub), 50)
    it = infos[-1].iters
    ins = _inside(G, kfbi)
    err = float(np.abs(u.cpu().numpy() - W.exact_grid(w, ins))[ins].max())
    out = {"workload": "ellipse Dirichlet 2D, N=64, u=e^x sin y, 4th order, FP64 DST, GMRES rtol 1e-10",
           "n_b": G.nb, "gmres_iterations": it, "us_per_solve": solve_us,
           "solves_per_s": 1e6 / solve_us, "us_gmres": gmres_us,
           "us_per_gmres_iteration": gmres_us / max(1, it), "us_per_operator_application": apply_us,
           "us_per_box_solve": box_us, "max_err_vs_exact": err,
           "paper_table1_n64": {"n_b": 116, "gmres_iterations": 10, "einf": 1.31e-4, "cpu_s": 3.91e-3,
                                "note": "Sec. 7.1.1's rotated ellipse in [-1.2,1.2]^2 (a different "
                                        "geometry), on the paper's CPU"}}
    G.close()
    return out


def run_reference(args):
    """CPU oracle arm: the oracle as it stands, on the host, one FFT worker.
    A step is one application of the oracle's BIE operator (one GMRES
    iteration's work, which dominates a solve: about 2.5 s per full solve at
    1024^2 would make the default 200 steps run for minutes on end).  One
    full oracle solve runs first, untimed, for its GMRES iteration count;
    solves/s is then 1 / (t_step (iterations + 2)), the BIE right-hand side
    and the final evaluation (each a box solve with its corrections, as an
    application is) counted as one application each."""
    import scipy.fft

    import workloads as W
    from oracle import kfbi as OK
    w = workload(args.n)
    with scipy.fft.set_workers(1):
        P = OK.Problem(w)
        data = W.grid_data(w)
        g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
        _, x, iters, _ = P.solve(g1, g2, data, rtol=args.rtol)
        for _ in range(args.warmup):
            P.apply(x)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.apply(x)
        el = time.perf_counter() - t0
    per_solve = iters + 2
    v = args.steps / (el * per_solve)
    sample = (f"{args.steps} oracle operator applications at the solution density, a solve counted as "
              f"{iters} GMRES iterations (one untimed full oracle solve) + 2")
    return {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (manufactured solution, seeded, analytic level set)",
            "config": {"workload": f"flower interface 2D, N={args.n}, sigma_in/sigma_out=1000, "
                                   f"4th order, GMRES rtol {args.rtol:g}"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def profile_box(args):
    """Box solve alone on the 3D torus workload, for kernel profiles: two
    warm-up solves, five timed ones (CUDA events), one inside a profiler
    range."""
    import torch
    import workloads as W
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    n = args.threed_n
    w = W.torus_helmholtz_3d(n)
    box = kfbi.BOX_MG if args.profile_box == "mg" else kfbi.BOX_DST
    G = kfbi.Problem.from_workload(w, box_solver=box, precision=kfbi.MIXED, box_rtol=args.box_rtol,
                                   box_max_iters=args.box_steps)
    rhs = torch.randn(G.grid_shape, dtype=torch.float64, device="cuda",
                      generator=torch.Generator(device="cuda").manual_seed(5965))
    u = torch.zeros_like(rhs)
    st = torch.cuda.current_stream()
    for _ in range(2):
        kfbi.kfbi_box_solve(G.handle, rhs, u)
    ts = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        kfbi.kfbi_box_solve(G.handle, rhs, u)
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    print(f"{args.profile_box} mixed box solve {n}^3: {ms:.3f} ms ({(n - 1) ** 3 / ms / 1e3:.0f} Mpts/s)")
    torch.cuda.profiler.start()
    kfbi.kfbi_box_solve(G.handle, rhs, u)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    G.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--box-rtol", type=float, default=1e-11,
                    help="inner tolerance of the mixed box solve (correction size)")
    ap.add_argument("--box-steps", type=int, default=3,
                    help="steps of the mixed box solve at most (0: library default, 5)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--relax", type=float, default=0.05,
                    help="inexact GMRES on the 2D workload: omega of the relaxed box-solve tolerance (0: off)")
    ap.add_argument("--relax-3d", type=float, default=0.03,
                    help="the same for the 3D mixed DST legs (torus, Neumann, heterogeneous, learned)")
    ap.add_argument("--relax-batch", type=float, default=0.0,
                    help="the same for the batched star problems (off: with it some instances exceed "
                         "1.1x the FP64 path's error at rtol 1e-8)")
    ap.add_argument("--box", default="dst", choices=["dst", "mg"])
    ap.add_argument("--no-fp64-compare", dest="compare_fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-config1", dest="config1", action="store_false",
                    help="skip the 64^2 Dirichlet latency leg")
    ap.add_argument("--cpu-stages", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--batch", type=int, default=64,
                    help="instances of the batched star-interface workload (0: skip)")
    ap.add_argument("--no-batch-learned", dest="batch_learned", action="store_false",
                    help="skip the learned start of the batched workload")
    ap.add_argument("--batch-train", type=int, default=160,
                    help="training problems of the batched workload's learned start")
    ap.add_argument("--learned-n", type=int, default=256,
                    help="grid of the learned-start evaluation (0: skip)")
    ap.add_argument("--learned-geometries", type=int, default=400,
                    help="training ellipsoids (one solve each) of the 3D learned start")
    ap.add_argument("--learned-epochs", type=int, default=10)
    ap.add_argument("--learned-steps", type=int, default=8000,
                    help="minimum Adam steps of the networks' second training phase")
    ap.add_argument("--learned-eval", type=int, default=3)
    ap.add_argument("--threed-n", type=int, default=256,
                    help="grid of the 3D torus workload (0: skip)")
    ap.add_argument("--neumann-n", type=int, default=256,
                    help="grid of the Neumann torus leg (Sec. 7.2.1); 0 skips it")
    ap.add_argument("--moving-n", type=int, default=1024,
                    help="grid of the moving-interface leg (update per position vs create per position); 0 skips it")
    ap.add_argument("--moving-steps", type=int, default=16)
    ap.add_argument("--close-n2", type=int, default=1024,
                    help="grid of Table 2's circles and star in the close-interface leg; 0 skips that case")
    ap.add_argument("--close-n3", type=int, default=256,
                    help="grid of Table 6's torus and ellipsoid in the close-interface leg; 0 skips that case")
    ap.add_argument("--hetero-n", type=int, default=256,
                    help="grid of the heterogeneous interface leg (Sec. 7.2.5's coefficients); 0 skips it")
    ap.add_argument("--profile-box", default="", choices=["", "dst", "mg"],
                    help="profiling aid: on the 3D torus at --threed-n, time the mixed box solve alone and run "
                         "one more inside cudaProfilerStart/Stop (for ncu --profile-from-start off); no JSON line")
    args = ap.parse_args()
    if args.cpu_stages:
        cpu_stages(args)
        return
    if args.profile_box:
        profile_box(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
