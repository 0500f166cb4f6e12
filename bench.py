#!/usr/bin/env python3
"""Benchmark: time to a binary64 relative residual of 1e-10, mixed vs FP64
GMRES(m), on one GB300.

Workload (default): mixed binary32-inner / binary64-residual GMRES(100) with
CGSR on the 3-D 7-point upwind convection-diffusion stencil, 160^3 grid
(n = 4 096 000, nnz = 28 518 400), random seeded velocity in [-1, 1]^3,
b = A 1 + N(0, sigma^2) noise with sigma = 1e-3, x0 = 0, tol 1e-10; the FP64 GMRES(100) CGSR solve
of the same system is timed beside it.  One step = one full solve to 1e-10.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (its
OpenMP build, every host core) on whole restart cycles of the same workload
instead, scaled to the oracle's own schedule.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "convdiff3d_160"
SEED = 20110185
# Inner iterations and restart cycles of the oracle's own full solves of the
# workloads (python -m oracle.golden_fullsize schedule stores the 160^3 one in
# tests/golden/convdiff3d_160_schedule.json, which takes precedence; the solve
# took 1121 s on one x86 core); used to scale the oracle's measured restart
# cycle to a full solve.  The GPU solves take the same schedules.
SCHEDULE = {"convdiff3d_160": {"mixed": {"iters": 1300, "restarts": 13}}}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--compare-steps", "--fp64-steps", dest="compare_steps", type=int, default=1)
    p.add_argument("--spai-params", default=None)
    p.add_argument("--cgs-kernel", type=int, default=0, choices=[0, 2],
                   help="CGSR kernel family: 0 register-streaming rows (update split by "
                        "basis vectors), 2 the same with the update split by rows")
    p.add_argument("--l2-prefetch", type=int, default=None,
                   help="CGSR rows kernels: slices prefetched ahead into L2 (library default)")
    p.add_argument("--block-cluster", type=int, default=None,
                   help="block path: 1 block or an 8-block cluster per system (library default)")
    p.add_argument("--cluster-threads", type=int, default=None,
                   help="batched: threads per block of the large systems' clusters")
    p.add_argument("--cluster-rows", type=int, default=None,
                   help="batched: systems of at least this many rows use 8-block clusters")
    p.add_argument("--trsv-kernel", type=int, default=None,
                   help="ILU(0) triangular solves: 1 per-row flags, 2 level barrier, "
                        "3 barrier-free (library default: 3 or 2 per triangle)")
    p.add_argument("--batch-count", type=int, default=2048,
                   help="batched workload: number of systems (profiling a smaller batch)")
    p.add_argument("--batch-rows", type=int, nargs=2, default=[500, 50000],
                   metavar=("MIN", "MAX"), help="batched workload: range of system sizes")
    p.add_argument("--batch-ortho", default="mgs", choices=["mgs", "cgsr"],
                   help="batched workload: orthogonalisation of the timed solves")
    p.add_argument("--spmv-lanes", type=int, default=0,
                   help="lanes per CSR row (0: autotuned)")
    p.add_argument("--spmv-format", choices=["auto", "csr", "sliced"], default="auto",
                   help="storage of A for the Krylov step's product (auto: the autotuner's)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, world, device="cuda"):
    """The largest of every rank's value (the job's time is its slowest
    rank's); the value itself on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batched_seed(rank):
    """Seed of the batch rank `rank` solves: with several GPUs every rank
    solves its own independent batch of systems (the batched path shards by
    system, with no collective; weak scaling)."""
    return SEED + 104729 * rank


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_workload(name):
    from paper_2011_01850_gb300 import inputs as I
    spec = I.WORKLOADS[name]
    A, b, spec = I.workload(name, seed=SEED)
    return A, b, spec


# Comparisons timed beside the headline mode of each workload:
# (label, precision, ortho, preconditioner)
COMPARE = {
    "convdiff3d_160": [("fp64", "fp64", "cgsr", None), ("mixed_fp16", "mixed_fp16", "cgsr", None),
                       ("mixed_bf16", "mixed_bf16", "cgsr", None)],
    "convdiff3d_96_ilu": [("unpreconditioned", "mixed", "cgsr", "none"),
                          ("fp64_ilu0", "fp64", "cgsr", "ilu")],
    "convdiff3d_96": [("fp64", "fp64", "cgsr", None)],
    "convdiff2d_64": [("mixed_mgs", "mixed", "mgs", None), ("fp64_grid", "fp64", "mgs", "grid")],
    "powerlaw_2m": [("mixed_fp16", "mixed_fp16", "mgs", None), ("mixed_fp32", "mixed", "mgs", None),
                    ("fp64", "fp64", "mgs", None)],
    "aniso3d_128": [("unpreconditioned", "mixed", "cgsr", "none"),
                    ("jacobi", "mixed", "cgsr", "jacobi"), ("fp64", "fp64", "cgsr", "none")],
}
SPAI_PARAMS = os.path.join(ROOT, "paper_2011_01850_gb300", "data", "spai_aniso64.npy")
# DRAM bytes per algorithmic byte of the CGSR passes (binary32 basis), from
# one ncu capture of a mid-cycle step (51 vectors) at 96^3: 563.3 MB of DRAM
# traffic for 559.2 MB algorithmic; scaled to the timed launches.
CGSR_ROWS_TRAFFIC_RATIO = 1.007


def bench_ours(args):
    import torch

    from paper_2011_01850_gb300 import gmres as G

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if args.workload == "batched2048":
        return bench_batched(args, world, rank, local)
    A, b, spec = make_workload(args.workload)
    n = len(A[0]) - 1
    nnz = len(A[1])
    m, ortho, prec = spec["m"], spec["ortho"], spec["prec"]
    stream = torch.cuda.current_stream()
    solver = G.Solver(A, stream=stream)
    if args.spmv_lanes:
        lanes32 = lanes64 = args.spmv_lanes
        solver.set_opts(spmv_lanes=args.spmv_lanes)
    else:
        lanes32, lanes64 = G.gmres_autotune(solver.h)
    if args.spmv_format != "auto":
        solver.set_opts(spmv_format={"csr": G.SPMV_CSR, "sliced": G.SPMV_SLICED}[args.spmv_format])
    fmt32, fmt64 = G.gmres_spmv_format(solver.h)
    solver.set_opts(profile=1, cgs_kernel=args.cgs_kernel)
    if args.l2_prefetch is not None:
        solver.set_opts(l2_prefetch=args.l2_prefetch)
    if args.block_cluster is not None:
        solver.set_opts(block_cluster=args.block_cluster)
    if args.trsv_kernel is not None:
        solver.set_opts(trsv_kernel=args.trsv_kernel)
    learned = spec.get("precond") == "learned"
    spai_params = None
    if learned:
        from paper_2011_01850_gb300 import spai as S
        spai_params = np.load(args.spai_params).astype(np.float32)
        jac = S.jacobi_params()
    db = torch.tensor(b, device="cuda", dtype=torch.float64)
    dx = torch.zeros(n, device="cuda", dtype=torch.float64)

    ilu_state = {}

    def set_pre(kind):
        o = G.gmres_get_opts(solver.h)
        o.path = G.PATH_AUTO
        if kind in (None, "none"):
            o.precond = 0
        elif kind == "grid":
            o.precond = 0
            o.path = G.PATH_GRID
        elif kind == "ilu":
            if not ilu_state:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                G.gmres_ilu0(solver.h)
                ilu_state["setup_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
            o.precond = 2
        else:
            G.gmres_spai_set(solver.h, spai_params if kind == "learned" else jac)
            o.precond = 1
        G.gmres_set_opts(solver.h, o)

    def step(p, o_, collect):
        dx.zero_()
        st, info = G.gmres_solve(solver.h, db, dx, m, 1e-10, G.ORTHOS[o_], G.PRECISIONS[p],
                                 100000)
        if st != G.OK:
            raise RuntimeError("solve did not converge: %s %r" % (G.status_str(st),
                                                                   info.as_dict()))
        collect.append(info.as_dict())

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    main_pre = {"learned": "learned", "ilu": "ilu"}.get(spec.get("precond"))
    set_pre(main_pre)
    scratch = []
    for _ in range(args.warmup):
        step(prec, ortho, scratch)
    infos = []
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(prec, ortho, infos)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    # the paper's accuracy measure on the last timed solution (outside the
    # timed region)
    bwd_err = G.gmres_backward_error(solver.h, db, dx)
    # error against the oracle's binary64 solution where it is stored
    # (tests/golden/<workload>_x.npz, written by oracle/golden_fullsize.py)
    gold = None
    gpath = os.path.join(ROOT, "tests", "golden", args.workload + "_x.npz")
    if os.path.exists(gpath):
        z = np.load(gpath)
        gold = (torch.tensor(z["idx"].astype(np.int64), device="cuda"),
                torch.tensor(z["x"], device="cuda", dtype=torch.float64))

    def x_error():
        if gold is None:
            return None
        d = (dx[gold[0]] - gold[1]).abs() / gold[1].abs()
        return {"max": float(d.max()), "rms": float(torch.sqrt((d * d).mean())),
                "samples": int(d.numel())}

    headline_err = x_error()

    # end to end through the public API with host buffers (H2D of b and x0,
    # D2H of x inside every step)
    e2e = None
    if not args.no_e2e:
        bh = np.ascontiguousarray(b)
        xh = np.zeros(n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            xh[:] = 0.0
            st, info = G.gmres_solve(solver.h, bh, xh, m, 1e-10, G.ORTHOS[ortho],
                                     G.PRECISIONS[prec], 100000)
            assert st == G.OK
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        e2e = {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": 8 * n}

    # comparisons on the same system
    compare = {}
    if args.compare_steps > 0:
        for label, p_, o_, pre in COMPARE.get(args.workload, []):
            set_pre(pre)
            step(p_, o_, scratch)
            torch.cuda.synchronize()
            got = []
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.compare_steps):
                step(p_, o_, got)
            e1.record(stream)
            torch.cuda.synchronize()
            cms = e0.elapsed_time(e1) / args.compare_steps
            compare[label] = {"ms": round(cms, 3), "iters": got[0]["iters"],
                              "restarts": got[0]["restarts"], "relres": got[0]["relres"],
                              "speedup_of_headline": round(cms / ms_step, 3),
                              "err_vs_oracle": x_error()}
        set_pre(main_pre)
        if "setup_ms" in ilu_state:
            compare["ilu_factor_ms"] = ilu_state["setup_ms"]

    def agg(key, cls):
        return sum(i[key][cls] for i in infos)

    classes = ["residual", "spmv", "ortho", "normalize", "update", "precond", "block"]
    kms = {c: agg("kernel_ms", c) for c in classes}
    kbytes = {c: agg("kernel_bytes", c) for c in classes}
    klaunch = {c: agg("kernel_launches", c) for c in classes}
    dom = max(classes, key=lambda c: kms[c])
    peak, peak_kind = load_peaks()
    achieved = kbytes[dom] / (kms[dom] * 1e-3) / 1e9 if kms[dom] > 0 else 0.0
    launches = int(sum(i["launches"] for i in infos))
    tot_bytes = sum(kbytes.values())
    tot_kms = sum(kms.values())
    iters = infos[0]["iters"]
    restarts = infos[0]["restarts"]
    kernel_names = {"ortho": ("CGSR passes (k_cgs_rows x2 + k_cgs_passb_reg + "
                              "k_reduce_cols x2)" if prec == "mixed"
                              else "CGSR passes (k_cgs_rows x3 + k_reduce_cols x2)")
                    if ortho == "cgsr" else ("MGS step (cooperative: k_mgs_staged where its "
                                             "shared-memory ring fits, else k_mgs_persist)"),
                    "block": "single-block solver (k_block_solve)",
                    "spmv": ("SpMV (k_spmv_step_sell, sliced storage)"
                             if prec != "mixed_limited"
                             and (fmt64 if prec == "fp64" else fmt32) == G.SPMV_SLICED
                             else "SpMV (k_spmv_step)"),
                    "residual": "binary64 residual (k_residual)"}
    out = {
        "metric": "time-to-1e-10 residual and HBM GB/s: mixed vs FP64 GMRES(m), one GB300",
        "value": round(ms_step, 3),
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec != "fp64" else "f64",
        "data": "synthetic",
        "config": {
            "workload": args.workload, "description": spec.get("desc"),
            "n": n, "nnz": nnz, "m": m, "ortho": ortho, "precision": prec, "tol": 1e-10,
            "precond": {"learned": "learned SpAI", "ilu": "ILU(0), left"}.get(spec.get("precond")),
            "trsv_kernel": ({0: "auto", 1: "per-row flags", 2: "level barrier", 3: "barrier-free"}[
                int(G.gmres_get_opts(solver.h).trsv_kernel)]
                if spec.get("precond") == "ilu" else None),
            "rhs": "b = A 1 + N(0, sigma^2), sigma = 1e-3, x0 = 0", "seed": SEED,
            "l2": "inputs larger than L2" if nnz * 12 > 129e6
                  else "inputs L2-resident (no flush; small-system workload)",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "spmv_lanes": {"f32": lanes32, "f64": lanes64},
            "spmv_format": {"f32": "sliced" if fmt32 == G.SPMV_SLICED else "csr",
                            "f64": "sliced" if fmt64 == G.SPMV_SLICED else "csr"},
            "cgs_kernel": {0: "register-streaming rows, pass B slice in registers",
                           2: "register-streaming rows, per-row-group update"}[args.cgs_kernel],
            "l2_prefetch": int(G.gmres_get_opts(solver.h).l2_prefetch),
            "block_cluster": int(G.gmres_get_opts(solver.h).block_cluster),
        },
        "iters": iters, "restarts": restarts,
        "compare": compare,
        "solve_gbs": round(tot_bytes / (tot_kms * 1e-3) / 1e9, 1) if tot_kms else None,
        "kernel_gbs": {c: round(kbytes[c] / (kms[c] * 1e-3) / 1e9, 1) if kms[c] else None
                       for c in classes if kms[c] > 0},
        "kernel_share": {c: round(kms[c] / tot_kms, 4) for c in classes if kms[c] > 0},
        "roofline": {
            "bound": "hbm", "kernel": kernel_names.get(dom, dom),
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
            "traffic": (round(CGSR_ROWS_TRAFFIC_RATIO * kbytes[dom] / klaunch[dom])
                        if CGSR_ROWS_TRAFFIC_RATIO and dom == "ortho" and ortho == "cgsr"
                        and args.cgs_kernel == 0 and prec == "mixed" and klaunch[dom]
                        else None),
            "launches": int(klaunch[dom]),
            "bytes_per_launch": kbytes[dom] / klaunch[dom] if klaunch[dom] else None,
        },
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "relres": infos[0]["relres"],
        "err_vs_oracle": headline_err,
        "backward_error": bwd_err,
    }
    if "fp64" in compare:
        out["speedup_vs_fp64"] = compare["fp64"]["speedup_of_headline"]
    if learned:
        # inference of the learned preconditioner (features cached, the MLP on
        # every nonzero, M's values): once per matrix, outside the timed solves
        set_pre("learned")
        torch.cuda.synchronize()
        tinf = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.gmres_spai_set(solver.h, spai_params)
            e1.record(stream)
            torch.cuda.synchronize()
            tinf.append(e0.elapsed_time(e1))
        inf_ms = statistics.median(tinf)
        # 8 -> 64 -> 64 -> 1 network: 4672 multiply-adds per nonzero
        fwd_flop = 2.0 * 4672 * nnz
        # FP32 FMA peak from the unit counts: SMs x 128 FP32 lanes x 2 flop x
        # the maximum SM clock (MEASURED_PEAKS.json's, else 2070 MHz)
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f).get("sm_max_mhz", 2070.0))
        except (OSError, ValueError):
            mhz = 2070.0
        fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        out["spai"] = {"inference_ms": round(inf_ms, 3), "forward_gflop": round(fwd_flop / 1e9, 1),
                       "achieved_tflops": round(fwd_flop / (inf_ms * 1e-3) / 1e12, 2),
                       "fp32_peak_tflops": round(fp32_peak, 1),
                       "frac": round(fwd_flop / (inf_ms * 1e-3) / 1e12 / fp32_peak, 3),
                       "solve_plus_inference_ms": round(ms_step + inf_ms, 3)}
    if dom == "precond" and spec.get("precond") == "ilu" and klaunch[dom]:
        # the triangular solves pass their dependency levels one after another:
        # bound by the latency of a level, not by bytes
        lo, up = G.gmres_ilu_levels(solver.h)
        per_launch_us = kms[dom] * 1e3 / klaunch[dom]
        out["roofline"].update({
            "bound": "latency", "kernel": "level-scheduled triangular solves (L, U)",
            "levels_per_launch": (lo + up) / 2,
            "us_per_level": round(per_launch_us / ((lo + up) / 2), 3),
            "note": "achieved/frac: algorithmic bytes over time against HBM, for context"})
    solver.close()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, A, b, spec, iters, restarts, m)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_batched(args, world, rank, local):
    """2048 independent 2-D systems (n log-uniform in [500, 50000]) solved by
    one persistent launch; a step is one batched solve of all systems."""
    import torch

    from paper_2011_01850_gb300 import gmres as G
    from paper_2011_01850_gb300 import inputs as I

    systems = I.batched_convdiff2d(count=args.batch_count, nmin=args.batch_rows[0],
                                   nmax=args.batch_rows[1], seed=batched_seed(rank))
    sys_ptr, rp, ci, va, b = G.pack_batch(systems)
    nsys = len(systems)
    stream = torch.cuda.current_stream()
    h = G.gmres_batch_create(nsys, sys_ptr, rp, ci, va, stream=stream)
    if args.cluster_rows is not None:
        G.gmres_batch_set_cluster_rows(h, args.cluster_rows)
    if args.cluster_threads is not None:
        G.gmres_batch_set_cluster_threads(h, args.cluster_threads)
    db = torch.tensor(b, device="cuda", dtype=torch.float64)
    dx = torch.zeros(len(b), device="cuda", dtype=torch.float64)
    m = 30
    # SpMV lanes per row from the library's autotuner (capped solves, untimed)
    bortho = {"mgs": G.ORTHO_MGS, "cgsr": G.ORTHO_CGSR}[args.batch_ortho]
    if args.spmv_lanes:
        lanes = {"fp64": args.spmv_lanes, "mixed": args.spmv_lanes}
    else:
        lanes = {p_: G.gmres_batch_autotune(h, db, m, bortho, G.PRECISIONS[p_], 2 * m)
                 for p_ in ("fp64", "mixed")}

    def step(prec, collect):
        # the tuned choice for this precision (lanes = 0 would reuse the last one tuned)
        dx.zero_()
        st, res, info = G.gmres_batch_solve(h, db, dx, m, 1e-10, bortho,
                                            G.PRECISIONS[prec], 100000, lanes=lanes[prec],
                                            nsys=nsys)
        if st != G.OK:
            raise RuntimeError("batched solve did not converge: %d" % st)
        collect.append((info.kernel_ms[G.K_BLOCK], info.kernel_bytes[G.K_BLOCK], info.iters,
                        info.restarts, res))

    scratch = []
    for _ in range(args.warmup):
        step("mixed", scratch)
    infos = []

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step("mixed", infos)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    compare = {}
    if args.compare_steps > 0:
        got = []
        step("fp64", scratch)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.compare_steps):
            step("fp64", got)
        e1.record(stream)
        torch.cuda.synchronize()
        cms = e0.elapsed_time(e1) / args.compare_steps
        compare["fp64"] = {"ms": round(cms, 3), "iters": got[0][2],
                           "speedup_of_headline": round(cms / ms_step, 3)}
    e2e = None
    if not args.no_e2e:
        xh = np.zeros(len(b))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            xh[:] = 0
            st, res, info = G.gmres_batch_solve(h, b, xh, m, 1e-10, bortho, G.MIXED,
                                                100000, lanes=lanes["mixed"], nsys=nsys)
            assert st == G.OK
        e2e = {"value": round((time.perf_counter() - t0) * 1e3 / args.steps, 3), "unit": "ms",
               "h2d_bytes_per_step": 16 * len(b), "d2h_bytes_per_step": 8 * len(b)}
    G.gmres_batch_destroy(h)
    kms = sum(i[0] for i in infos)
    kb = sum(i[1] for i in infos)
    peak, peak_kind = load_peaks()
    ach = kb / (kms * 1e-3) / 1e9
    out = {
        "metric": "time-to-1e-10 residual and HBM GB/s: mixed vs FP64 GMRES(m), one GB300",
        "value": round(ms_step, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched2048", "systems": nsys,
                   "system_rows": list(args.batch_rows), "rows": int(len(b)),
                   "nnz": int(len(ci)), "m": m, "ortho": args.batch_ortho, "precision": "mixed",
                   "tol": 1e-10,
                   "launch": "one-block and 8-block-cluster persistent launches, concurrent",
                   "spmv_lanes": lanes, "l2": "inputs larger than L2"},
        "systems_per_s": round(world * nsys / (ms_step * 1e-3), 1),
        "iters_total": infos[0][2], "restarts_total": infos[0][3],
        "compare": compare,
        "roofline": {"bound": "hbm",
                     "kernel": "batched whole-solve kernels (k_block_solve + k_team_solve)",
                     "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4), "peak_kind": peak_kind, "traffic": None,
                     "launches": args.steps, "bytes_per_launch": kb / args.steps},
        "gpu_launches": args.steps, "clocks": clk, "e2e": e2e,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def host_cpu():
    """(cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return os.cpu_count() or 1, model or platform.machine()


def oracle_schedule(name, prec):
    """The oracle's own restart schedule of a workload: stored by
    oracle/golden_fullsize.py where it exists, else the table above."""
    path = os.path.join(ROOT, "tests", "golden", name + "_schedule.json")
    try:
        with open(path) as f:
            g = json.load(f)
        if g.get("prec") == prec:
            return {"iters": g["iters"], "restarts": g["restarts"]}
    except (OSError, ValueError, KeyError):
        pass
    return SCHEDULE.get(name, {}).get(prec)


def oracle_cycle_sample(A, b, spec, kmax):
    """Time, with the oracle's OpenMP build on every host core, one binary64
    residual and one restart cycle of kmax inner iterations on the full
    workload (the cycle starts from b, as the first one of a solve does).
    Returns (t_residual, t_cycle, threads)."""
    import oracle as O
    prec = {"fp64": O.FP64, "mixed": O.MIXED, "mixed_bf16": O.MIXED_BF16,
            "mixed_fp16": O.MIXED_FP16}[spec["prec"]]
    ortho = O.CGSR if spec["ortho"] == "cgsr" else O.MGS
    M = ilu = None
    with O.use(O.lib_omp()):
        threads = O.threads(os.cpu_count() or 1)
        if spec.get("precond") == "ilu":
            ilu = O.ilu0(A)  # the oracle's own factors (their time is not counted)
        elif spec.get("precond"):
            M = (A[0], A[1], O.spai_values(A, O.spai_jacobi_params()))
        t0 = time.perf_counter()
        O.residual_norm(A, b, np.zeros_like(b))
        t_res = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.arnoldi_cycle(A, b, spec["m"], ortho=ortho, prec=prec, kmax=kmax,
                        export_basis=False, M=M, ilu=ilu)
        t_cyc = time.perf_counter() - t0
    return t_res, t_cyc, threads


def scale_to_schedule(t_res, t_cyc, kmax, iters, restarts):
    """Solve time for a schedule of `restarts` cycles and `iters` inner
    iterations from a measured cycle of kmax iterations: every cycle of kmax
    iterations costs the measured time (exact when the schedule's cycles all
    have that length, as the 160^3 workload's 13 cycles of 100 do); a shorter
    last cycle costs its share of the orthogonalisation work, which grows
    like L (L + 1) / 2 inner products."""
    full, rem = divmod(iters, kmax)
    t = full * t_cyc + (restarts + 1) * t_res
    if rem:
        t += t_cyc * (rem * (rem + 1)) / (kmax * (kmax + 1))
    return t


def cpu_baseline(name, A, b, spec, iters, restarts, m):
    """The oracle timed on the host cores, scaled to the oracle's own schedule
    for the workload (or to the GPU's, where no oracle schedule is stored)."""
    sched = oracle_schedule(name, spec["prec"]) or {"iters": iters, "restarts": restarts}
    t_res, t_cyc, threads = oracle_cycle_sample(A, b, spec, m)
    est = scale_to_schedule(t_res, t_cyc, m, sched["iters"], sched["restarts"])
    cores, model = host_cpu()
    return {"value": round(est * 1e3, 1), "unit": "ms", "cores": threads, "kind": "oracle",
            "cpu": model, "host_cores": cores,
            "cycle_s": round(t_cyc, 3), "residual_s": round(t_res, 4),
            "sample": "the oracle's OpenMP build (-O3 -fopenmp, loops over rows and vector "
                      "entries on %d threads) timed on one whole restart cycle of %d inner "
                      "iterations (%.1f s) and one binary64 residual (%.3f s) of the full "
                      "workload, scaled to the oracle's schedule of %d iterations in %d "
                      "cycles" % (threads, m, t_cyc, t_res, sched["iters"], sched["restarts"])}


def bench_reference(args):
    """The reference arm: the oracle as it stands (OpenMP timing build, every
    host core), rank 0 only.  Warm-up steps time a 2-iteration cycle (thread
    start-up, page-in); every timed step times one whole restart cycle of m
    inner iterations and one residual of the full workload, scaled to the
    oracle's own schedule for it."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    A, b, spec = make_workload(args.workload)
    m = spec["m"]
    sched = oracle_schedule(args.workload, spec["prec"]) or {"iters": m, "restarts": 1}
    vals, cycles, residuals = [], [], []
    threads = 1
    for i in range(args.warmup + args.steps):
        if i < args.warmup:
            oracle_cycle_sample(A, b, spec, 2)
            continue
        t_res, t_cyc, threads = oracle_cycle_sample(A, b, spec, m)
        cycles.append(t_cyc)
        residuals.append(t_res)
        vals.append(scale_to_schedule(t_res, t_cyc, m, sched["iters"], sched["restarts"]) * 1e3)
    v = statistics.mean(vals)
    cores, model = host_cpu()
    sample = ("per step: one whole restart cycle of %d inner iterations (mean %.2f s) and one "
              "binary64 residual (mean %.3f s) of the full workload with the oracle's OpenMP "
              "build on %d threads, scaled to the oracle's schedule of %d iterations in %d "
              "cycles; warm-up steps: a 2-iteration cycle"
              % (m, statistics.mean(cycles), statistics.mean(residuals), threads,
                 sched["iters"], sched["restarts"]))
    out = {
        "impl": "reference",
        "metric": "time-to-1e-10 residual and HBM GB/s: mixed vs FP64 GMRES(m), one GB300",
        "value": round(v, 1), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if spec["prec"] != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "ortho": spec["ortho"],
                   "precision": spec["prec"], "tol": 1e-10, "seed": SEED},
        "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": threads, "kind": "oracle",
                         "cpu": model, "host_cores": cores, "sample": sample},
        "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.spai_params is None:
        args.spai_params = SPAI_PARAMS
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
