#!/usr/bin/env python
"""Throughput of the flip-free ADMM loop on one GB300.

Workload: 3D deformation of a jittered unit cube, 64^3 cells x 6 tetrahedra
(1,572,864 tets, 274,625 vertices), bottom face fixed, top face rotated 45
degrees and shifted, symmetric Dirichlet energy, mu_i = 10 w_i, FP32 local step
with the W step and reductions in double.  One step = one ADMM iteration
(W step, U/P/Lambda steps, error terms; the termination test every
check_every iterations).  The per-iteration working set (factor blocks and
element state, > 1 GB) is larger than L2, so no flush is needed between
iterations.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload family instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM iterations/sec and element-updates/sec at ~1.5M tets; % HBM roofline"
UNIT = "iter/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=64)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--check-every", type=int, default=50)
    ap.add_argument("--schedule", type=int, default=1, choices=[0, 1, 2],
                    help="supernodal solves: 0 one launch per tree level, 1 dynamic ready queue, "
                         "2 dynamic ready queue with a bulk-copy ring per block")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-cells", type=int, default=16)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--growth-cells", type=int, nargs="*", default=[24, 32],
                    help="cube sizes at which the oracle is also timed to measure its growth exponent")
    ap.add_argument("--oracle-probe", type=float, nargs=3, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--workload", default="cube_deform",
                    choices=["cube_deform", "cube_outcome", "batch256", "uv_disk", "uv_heightfield", "cube_handles",
                             "tutte", "decompose", "volume_correspondence"],
                    help="cube_deform: the throughput benchmark; the others report time to tolerance "
                         "(uv_disk, uv_heightfield), batched meshes, or forward + adjoint (cube_handles)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--local-variant", default="paper", choices=["paper", "joint"],
                    help="uv_disk / uv_heightfield: the paper's local step or the joint (U, P) prox variant")
    ap.add_argument("--factor", default="host", choices=["host", "device", "device64"],
                    help="where the numeric decomposition of L runs (setup and every rescaling event of "
                         "--penalties paper): host in double, device in float, device in double")
    ap.add_argument("--factors", nargs="*", default=["host", "device", "device64"],
                    choices=["host", "device", "device64"],
                    help="decompose: the placements of the decomposition to time")
    ap.add_argument("--top-inverse", type=int, default=0,
                    help="cube_deform: the top levels of the elimination tree solved as x_T = S^-1 t_T between "
                         "the passes (0 off, -1 automatic, k > 0 the top k levels)")
    ap.add_argument("--penalties", default="fixed", choices=["fixed", "paper"],
                    help="uv_disk / uv_heightfield / cube_outcome: mu = rho w fixed, or the paper's rescaling schedule")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


SOLVE_PROFILE = os.path.join(ROOT, "profiles", "k_solve_dynamic_cube48.md")


def solve_fingerprint() -> str:
    """sha256 of the device code of the supernodal solves (the task code and the
    per-level, dynamic and pipelined kernels the ncu traffic figure was taken on,
    up to the reset of their queues), of the task-shape constants and of the code
    that builds the task lists."""
    csrc = os.path.join(ROOT, "paper_2107_05200_gb300", "csrc")
    with open(os.path.join(csrc, "ffa_solve.cu")) as f:
        src = f.read()
    a = src.index("// supernodal solves.")
    b = src.index("// restores the ready queues", a)
    with open(os.path.join(csrc, "ffa_schedule.h")) as f:
        consts = "".join(line for line in f if line.startswith("constexpr"))
    with open(os.path.join(csrc, "ffa_schedule.cpp")) as f:
        sched = f.read()
    return hashlib.sha256((src[a:b] + consts + sched).encode()).hexdigest()[:16]


def profiled_solve_traffic():
    """DRAM bytes per full-size forward and backward launch from the committed ncu
    summary, or None when the solve kernels changed since it was taken."""
    if not os.path.exists(SOLVE_PROFILE):
        return None
    fp, fwd, bwd = None, None, None
    with open(SOLVE_PROFILE) as f:
        for line in f:
            if line.startswith("fingerprint:"):
                fp = line.split(":", 1)[1].strip().strip("`")
            elif line.startswith("full-size traffic per launch (bytes):"):
                parts = dict(x.strip().split(" ") for x in line.split(":", 1)[1].split(","))
                fwd, bwd = int(parts["forward"]), int(parts["backward"])
    if fp != solve_fingerprint() or fwd is None:
        return None
    return fwd, bwd


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="ffa_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_probe(cells: int, iters: int, seconds: float = 0.0):
    """Per-iteration wall time of the FP64 oracle on the cube of `cells`^3 cells:
    setup (the operator and its sparse LU, timed on its own) and one iteration
    untimed, then `iters` iterations (or as many as fit in `seconds`, at least
    `iters`).  Returns (tets, list of per-iteration seconds, setup seconds)."""
    from oracle import admm
    from paper_2107_05200_gb300 import workloads as wk
    wl = wk.cube_deform(cells=cells)
    t0 = time.perf_counter()
    o = admm.Oracle.from_workload(wl)
    setup_s = time.perf_counter() - t0
    s = o.init(wl.W0)
    s, _ = o.step(s)
    times = []
    t_end = time.perf_counter() + seconds
    while len(times) < iters or time.perf_counter() < t_end:
        t0 = time.perf_counter()
        s, _ = o.step(s)
        times.append(time.perf_counter() - t0)
    return wl.m, times, setup_s


def oracle_timings(sizes, iters, seconds, threads):
    """oracle_probe for each (cells) in `sizes`, each in a fresh process whose
    numerical libraries are limited to `threads` threads (None: their default).
    Returns {cells: (tets, per-iteration seconds list, setup seconds)}."""
    env = dict(os.environ)
    if threads is not None:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    out = {}
    for c, it, sec in zip(sizes, iters, seconds):
        proc = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-probe", str(c), str(it), str(sec)],
                              env=env, capture_output=True, text=True, check=True)
        d = json.loads(proc.stdout.strip().splitlines()[-1])
        out[c] = (d["tets"], d["times"], d["setup_s"])
    return out


def extrapolate(samples, m_full):
    """Per-iteration seconds at m_full tets from the medians measured at the sampled
    sizes: the largest sample scaled by (m_full / m)^alpha, with alpha the slope of
    log t against log m between the two largest samples (1 with a single sample).
    The local slope at the top of the sampled range is used rather than a fit over
    every size because the oracle's time per iteration is not a pure power of m:
    the share of its sparse triangular solves grows with the factor's fill.  On the
    benchmark recipe, against 22.3 s measured per iteration at 64^3 cells, the slope
    between 24^3 and 32^3 cells predicted 22.7 s and 19.0 s in two runs and a fit
    over 16^3, 24^3 and 32^3 predicted 20.2 s and 18.4 s: the slope is closer but
    noisier (an 8x extrapolation multiplies a 5% timing difference at 32^3 into
    13%), so the larger sizes take the median of five iterations.
    Returns (seconds, alpha)."""
    cs = sorted(samples, key=lambda c: samples[c][0])
    m1, t1 = samples[cs[-1]][0], statistics.median(samples[cs[-1]][1])
    if len(cs) < 2:
        return float(t1 * m_full / m1), 1.0
    m0, t0 = samples[cs[-2]][0], statistics.median(samples[cs[-2]][1])
    alpha = math.log(t1 / t0) / math.log(m1 / m0)
    return float(t1 * (m_full / m1) ** alpha), float(alpha)


def oracle_baseline(m_full: int, n_full: int, sample_cells: int, seconds: float, growth_cells, threads):
    """The oracle timed on a bounded sample (the same recipe on smaller cubes) and
    extrapolated to the full workload with the growth exponent measured between the
    two largest sampled sizes.  Returns the cpu_baseline / reference description."""
    sizes = [sample_cells] + list(growth_cells)
    samples = oracle_timings(sizes, [3] + [5] * len(growth_cells), [seconds] + [0.0] * len(growth_cells), threads)
    per_it, alpha = extrapolate(samples, m_full)
    m_s, t_s, _ = samples[sample_cells]
    per_s = statistics.median(t_s)
    return {
        "value": 1.0 / per_it, "unit": UNIT, "kind": "oracle",
        "cores": 1 if threads == 1 else (os.cpu_count() or 1),
        "threads": threads if threads is not None else "library default",
        "sample": (f"FP64 numpy/scipy oracle on the benchmark recipe at {sample_cells}^3 cells ({m_s} tets, "
                   f"{len(t_s)} timed iterations, median {per_s:.3f} s)"
                   + "".join(f", {c}^3 ({samples[c][0]} tets, {statistics.median(samples[c][1]):.3f} s)"
                             for c in growth_cells)
                   + f"; per-iteration time extrapolated from the largest size to {m_full} tets as m^{alpha:.3f}, "
                     "the exponent measured between the two largest sizes"),
        "sample_workload": f"cube_deform_{sample_cells}", "sample_tets": m_s, "sample_iter_per_s": 1.0 / per_s,
        "growth_exponent": alpha, "extrapolated_s_per_iter": per_it,
        "sizes": {f"cube_deform_{c}": {"tets": samples[c][0], "s_per_iter": statistics.median(samples[c][1]),
                                       "setup_s": samples[c][2]}
                  for c in sizes},
    }


def bench_config(args, m, n, rho, world):
    """The workload description both arms print (the GPU arm and the oracle arm)."""
    cfg = {"workload": f"cube_deform_{args.cells}", "tets": m, "vertices": n,
           "energy": "sym_dirichlet", "rho": rho, "local_precision": args.precision,
           "refine_sweeps": args.sweeps, "check_every": args.check_every,
           "solve_schedule": {0: "per_level", 1: "dynamic", 2: "pipelined"}[args.schedule],
           "l2": "working set > L2 (factor + element state), no flush",
           "parallelism": "replicas" if world > 1 else "single"}
    if getattr(args, "top_inverse", 0):
        cfg["top_inverse_levels"] = args.top_inverse
    return cfg


def run_reference(args, rank):
    """The oracle arm: the FP64 oracle timed on the host cores, on the benchmark recipe at
    a size it finishes (its own mesh named in config), single-threaded and with the
    numerical libraries' default threads; `value` is the single-threaded per-iteration
    rate extrapolated to the full cube with the measured growth exponent."""
    if rank != 0:
        return 0
    from paper_2107_05200_gb300 import workloads as wk
    V, T = wk.cube_tets(args.cells)
    m_full, n_full = T.shape[0], V.shape[0]
    rho_full = wk.cube_deform(cells=2).rho
    # the timed steps: `steps` iterations after `warmup` on the sample cube, one thread
    samples = oracle_timings([args.cpu_sample_cells], [args.warmup + args.steps], [0.0], 1)
    m_s, times, setup_s = samples[args.cpu_sample_cells]
    per_s = sum(times[args.warmup:]) / max(1, args.steps)
    single = oracle_baseline(m_full, n_full, args.cpu_sample_cells, 0.0, args.growth_cells, 1)
    multi = oracle_baseline(m_full, n_full, args.cpu_sample_cells, 0.0, args.growth_cells, None)
    value = single["value"]
    Vs, Ts = wk.cube_tets(args.cpu_sample_cells)
    cfg = bench_config(args, m_s, Vs.shape[0], rho_full, args.gpus)
    cfg["workload"] = f"cube_deform_{args.cpu_sample_cells}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "elem_updates_per_s": value * m_full,
            "config": cfg,
            "extrapolated_to": {"workload": f"cube_deform_{args.cells}", "tets": m_full, "vertices": n_full,
                                "rule": "per-iteration time of the largest sampled cube scaled to the full cube "
                                        "by the element-count ratio to the power measured between the two largest "
                                        "sampled cubes",
                                "growth_exponent": single["growth_exponent"],
                                "s_per_iter": single["extrapolated_s_per_iter"]},
            "sample_timed": {"workload": cfg["workload"], "tets": m_s, "iterations": args.steps,
                             "s_per_iter": per_s, "iter_per_s": 1.0 / per_s, "setup_s": setup_s},
            "cpu_baseline": single, "cpu_baseline_all_threads": multi,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, rank, world, local):
    """256 independent meshes solved to tolerance in one batch (one graph launch per
    check_every iterations for all of them) against the same meshes solved one after
    another with single-mesh contexts.  Metric: mesh-iterations per second."""
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import BatchSolver, Solver

    torch.cuda.set_device(local)
    wls = wk.batched_meshes(count=args.batch_count)
    max_iter = 2000
    t0 = time.perf_counter()
    bs = BatchSolver(wls, precision=args.precision, check_every=10, refine_sweeps=args.sweeps)
    t_setup = time.perf_counter() - t0
    bs.init([wl.W0 for wl in wls])
    tuning = bs.autotune(5)
    bs.init([wl.W0 for wl in wls])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats, nconv = bs.iterate(max_iter, stop_at_tol=True)
    t_batch = time.perf_counter() - t0
    iters_b = stats[0]["iters"]
    bs.close()
    # sequential: each mesh alone, to the same tolerance
    t_seq = 0.0
    iters_seq = 0
    conv_seq = 0
    for wl in wls:
        with Solver.from_workload(wl, precision=args.precision, check_every=10, refine_sweeps=args.sweeps) as sol:
            sol.init(wl.W0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            st = sol.iterate(max_iter, stop_at_tol=True)
            t_seq += time.perf_counter() - t1
            iters_seq += st["iters"]
            conv_seq += int(st["converged"] == 1)
    m_tot = sum(wl.m for wl in wls)
    line = {"metric": "batched meshes: mesh-iterations/sec to tolerance", "unit": "mesh-iter/s",
            "value": len(wls) * iters_b / t_batch, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": f"batch{len(wls)}", "meshes": len(wls), "elements": m_tot,
                       "tol": wls[0].eps_abs, "max_iter": max_iter},
            "batched": {"seconds": t_batch, "iterations": iters_b, "converged": nconv,
                        "setup_s": t_setup, "tuning": tuning},
            "sequential": {"seconds": t_seq, "mesh_iterations": iters_seq, "converged": conv_seq,
                           "value": iters_seq / t_seq},
            "speedup_time_to_tolerance": t_seq / t_batch}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_to_tolerance(args, local):
    """A 2D workload solved to its tolerance: wall time (setup excluded), iterations,
    flips, final energy; on the 48^2 disk also the CPU baseline (the FP64 oracle run
    for the same number of iterations, timed) and the GPU result's differences from
    it (W, energy, gradient)."""
    import numpy as np
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import Solver

    torch.cuda.set_device(local)
    wl = wk.uv_disk() if args.workload == "uv_disk" else wk.uv_heightfield()
    t0 = time.perf_counter()
    sol = Solver.from_workload(wl, precision=args.precision, check_every=10, refine_sweeps=args.sweeps,
                               penalties=args.penalties, local_variant=args.local_variant, factor=args.factor)
    t_setup = time.perf_counter() - t0
    sol.init(wl.W0)
    sol.iterate(10, stop_at_tol=False)          # warm-up (graph capture)
    sol.init(wl.W0)
    torch.cuda.synchronize()
    r0 = sol.info()["seconds_refactor"]
    t0 = time.perf_counter()
    st = sol.iterate(wl.max_iter, stop_at_tol=True)
    torch.cuda.synchronize()
    t_tol = time.perf_counter() - t0
    W = sol.W()
    E = sol.energy()
    dE = sol.gradient() if st["n_flipped"] == 0 else None
    t_refactor = sol.info()["seconds_refactor"] - r0   # the rescaling events inside the timed region
    sol.close()
    line = {"metric": "time to tolerance", "unit": "s", "value": t_tol, "n_gpus": 1, "higher_is_better": False,
            "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "elements": wl.m, "vertices": wl.n, "energy": wl.energy,
                       "rho": wl.rho, "eps_abs": wl.eps_abs, "eps_rel": wl.eps_rel, "max_iter": wl.max_iter,
                       "check_every": 10},
            "penalties": args.penalties, "local_variant": args.local_variant, "factor": args.factor,
            "rescales": st["rescales"], "refactor_s_total": t_refactor,
            "refactor_s_per_event": t_refactor / max(1, st["rescales"]),
            "iterations": st["iters"], "converged": st["converged"], "n_flipped": st["n_flipped"],
            "iter_per_s": st["iters"] / t_tol, "elem_updates_per_s": st["iters"] * wl.m / t_tol,
            "energy": E, "e_prim": st["e_prim"], "e_dual": st["e_dual"], "setup_s": t_setup}
    if args.workload == "uv_disk":
        # the CPU baseline of this workload: the FP64 oracle run for the same
        # iterations from the same start, timed on one host core; the GPU run's
        # differences from it are reported with it
        from oracle import admm, schedule
        t0 = time.perf_counter()
        o = admm.Oracle.from_workload(wl, local_variant=args.local_variant)
        t_o_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        if args.penalties == "paper":
            s_o, _, _ = schedule.run(o, wl.W0, st["iters"], stop_at_tol=False)
        else:
            s_o = o.init(wl.W0)
            for _ in range(st["iters"]):
                s_o, _ = o.step(s_o)
        t_o = time.perf_counter() - t0
        cb = {"value": t_o, "unit": "s", "cores": 1, "kind": "oracle", "setup_s": t_o_setup,
              "sample": f"the FP64 oracle on {wl.name}, the GPU run's {st['iters']} iterations from the same W0",
              "W_max_rel_diff": float(np.abs(W - s_o.W).max() / np.abs(s_o.W).max()),
              "energy_rel_diff": float(abs(E - o.energy(s_o.W)) / abs(o.energy(s_o.W)))}
        if dE is not None:
            g_o = o.energy_gradient(s_o.W)
            cb["gradient_rel_diff"] = float(np.linalg.norm(dE - g_o) / np.linalg.norm(g_o))
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    return 0


def run_handles(args, local):
    """The handle workload: 200 unrolled iterations with checkpoints every 20, then
    dL/db of the target loss; times both passes, and compares the FP32 gradient with
    the FP64 one."""
    import numpy as np
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import Solver

    torch.cuda.set_device(local)
    wl = wk.cube_handles()
    idx, tgt = wl.meta["target_idx"], wl.meta["targets"]
    out = {}
    for prec in ("fp32", "fp64"):
        with Solver.from_workload(wl, precision=prec) as sol:
            sol.set_handles(wl.pin_pos)
            sol.init(wl.W0)
            sol.forward_unrolled(20, 20)      # warm-up
            sol.init(wl.W0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol.forward_unrolled(200, 20)
            torch.cuda.synchronize()
            t_f = time.perf_counter() - t0
            W = sol.W()
            diff = W[idx] - tgt
            G = np.zeros_like(W)
            G[idx] = 2.0 * diff / len(idx)
            t0 = time.perf_counter()
            g = sol.backward_unrolled(G)
            torch.cuda.synchronize()
            t_b = time.perf_counter() - t0
            out[prec] = {"forward_s": t_f, "backward_s": t_b, "loss": float(np.mean(np.sum(diff * diff, 1))),
                         "grad": g}
    nb = wl.meta["n_bottom"]
    g32, g64 = out["fp32"]["grad"][nb:], out["fp64"]["grad"][nb:]
    line = {"metric": "forward + adjoint of 200 unrolled iterations", "unit": "s",
            "value": out[args.precision]["forward_s"] + out[args.precision]["backward_s"], "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32+f64" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "elements": wl.m, "vertices": wl.n, "handles": len(wl.pin_pos) - nb,
                       "iterations": 200, "checkpoint_every": 20},
            "fp32": {k: v for k, v in out["fp32"].items() if k != "grad"},
            "fp64": {k: v for k, v in out["fp64"].items() if k != "grad"},
            "grad_fp32_vs_fp64_rel": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64))}
    print(json.dumps(line), flush=True)
    return 0


def run_outcome(args, local):
    """The benchmark cube run to its configured 1000 iterations in both precisions
    (fixed mu = 10 w, or the paper's penalty schedule with --penalties paper): the statistics of eq. primaldualerror / primaldualthresholds every
    100 iterations, flipped elements and energy at the end, the FP32 iterate's
    difference from the FP64 one, and the wall time of each run (setup excluded)."""
    import numpy as np
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import Solver

    torch.cuda.set_device(local)
    wl = wk.cube_deform(cells=args.cells)
    iters = wl.max_iter
    out, Ws = {}, {}
    for prec in ("fp32", "fp64"):
        with Solver.from_workload(wl, precision=prec, check_every=100, refine_sweeps=args.sweeps,
                                  penalties=args.penalties, factor=args.factor) as sol:
            sol.init(wl.W0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hist = []
            for _ in range(iters // 100):
                st = sol.iterate(100, stop_at_tol=False)
                hist.append({"iter": st["checked_iter"], "e_prim": st["e_prim"], "thr_prim": st["thr_prim"],
                             "e_dual": st["e_dual"], "thr_dual": st["thr_dual"], "n_flipped": st["n_flipped"],
                             "energy_P": st["energy_P"], "rescales": st["rescales"]})
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            W = sol.W()
            E = sol.energy()
            Ws[prec] = W
            ref = sol.info()["seconds_refactor"]
            out[prec] = {"seconds": secs, "iter_per_s": iters / secs, "energy": E, "final": hist[-1],
                         "converged": st["converged"], "history": hist, "refactor_s_total": ref,
                         "refactor_s_per_event": ref / max(1, st["rescales"] + (args.penalties == "paper"))}
    d = float(np.abs(Ws["fp32"] - Ws["fp64"]).max() / np.abs(Ws["fp64"]).max())
    line = {"metric": "outcome after the configured iterations", "unit": "s", "value": out["fp32"]["seconds"],
            "n_gpus": 1, "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": wl.name, "elements": wl.m, "vertices": wl.n, "energy": wl.energy, "rho": wl.rho,
                       "eps_abs": wl.eps_abs, "eps_rel": wl.eps_rel, "iterations": iters,
                       "refine_sweeps": args.sweeps, "penalties": args.penalties, "factor": args.factor},
            "fp32": out["fp32"], "fp64": out["fp64"], "W_fp32_vs_fp64_max_rel": d}
    print(json.dumps(line), flush=True)
    return 0


def run_decompose(args, local):
    """The numeric decomposition of L_FF of the benchmark cube (Algorithm 2,
    decompose(L)) where each of --factors puts it: wall time at setup, and under the
    paper's penalty schedule the cost of one rescaling event (new L assembled and
    decomposed, right-hand-side terms refreshed) averaged over the events of the
    first 12 iterations, with the W-step residual after them."""
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import Solver

    torch.cuda.set_device(local)
    wl = wk.cube_deform(cells=args.cells)
    out = {}
    for factor in args.factors:
        with Solver.from_workload(wl, precision="fp32", factor=factor) as sol:
            info = sol.info()
        entry = {"setup_s": info["setup_seconds_factor"], "flops": info["factor_flops"]}
        with Solver.from_workload(wl, precision="fp32", penalties="paper", check_every=10, factor=factor) as sol:
            sol.init(wl.W0)
            r0 = sol.info()["seconds_refactor"]
            st = sol.iterate(12, stop_at_tol=False)
            entry["event_s"] = (sol.info()["seconds_refactor"] - r0) / max(1, st["rescales"])
            entry["events"] = st["rescales"]
            entry["wstep_residual"] = sol.wstep_residual()
        out[factor] = entry
    first = out[args.factors[0]]
    line = {"metric": "decomposition of L_FF", "unit": "s", "value": first["setup_s"], "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": wl.name, "elements": wl.m, "vertices": wl.n,
                       "factor": args.factors[0]},
            "placements": out}
    print(json.dumps(line), flush=True)
    return 0


def run_volume_correspondence(args, local):
    """Volume correspondence (Sec. Results): the Tutte start on the GPU (ffa_tutte),
    then the method to its termination test; wall times of both (setup excluded,
    the solver's graphs captured by a warm-up run), flips at the start and at the
    end."""
    import numpy as np
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import Solver, tutte

    torch.cuda.set_device(local)
    wl = wk.volume_correspondence(cells=args.cells, start=False)
    Vs, Ts = wk.cube_tets(2)                    # load the library, touch the device: one free vertex
    face = np.nonzero(np.any((Vs < 0.25) | (Vs > 0.75), axis=1))[0].astype(np.int32)
    tutte(Vs, Ts, face, Vs[face].copy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W0, rel = tutte(wl.V, wl.T, wl.pins, wl.pin_pos, factor=args.factor)
    t_tutte = time.perf_counter() - t0
    flipped0 = wk.flipped_fraction(W0, wl.T)
    t0 = time.perf_counter()
    sol = Solver.from_workload(wl, precision=args.precision, check_every=10, refine_sweeps=args.sweeps,
                               factor=args.factor)
    t_setup = time.perf_counter() - t0
    sol.init(W0)
    sol.iterate(10, stop_at_tol=False)          # warm-up (graph capture)
    sol.init(W0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = sol.iterate(wl.max_iter, stop_at_tol=True)
    torch.cuda.synchronize()
    t_admm = time.perf_counter() - t0
    E = sol.energy()
    sol.close()
    line = {"metric": "volume correspondence: Tutte start + the method to tolerance", "unit": "s",
            "value": t_tutte + t_admm, "n_gpus": 1, "higher_is_better": False,
            "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "elements": wl.m, "vertices": wl.n, "pinned": int(len(wl.pins)),
                       "energy": wl.energy, "rho": wl.rho, "eps_abs": wl.eps_abs, "eps_rel": wl.eps_rel,
                       "max_iter": wl.max_iter, "factor": args.factor},
            "tutte_s": t_tutte, "tutte_rel_residual": rel, "flipped_at_start": flipped0, "setup_s": t_setup,
            "admm_s": t_admm, "iterations": st["iters"], "converged": st["converged"],
            "n_flipped": st["n_flipped"], "energy": E, "e_prim": st["e_prim"], "e_dual": st["e_dual"]}
    print(json.dumps(line), flush=True)
    return 0


def run_tutte(args, local):
    """The Tutte initializer on a 1024^2-vertex disk (2.1M triangles): one ffa_tutte
    call (host ordering and factorization, GPU solve), against the oracle's sparse
    LU on the host."""
    import numpy as np
    import torch

    from oracle import tutte as ot
    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import tutte

    torch.cuda.set_device(local)
    grid = 1024
    V, T = wk.grid_triangles(grid, grid, no_ears=True)
    bnd = wk._grid_boundary_cycle(grid, grid)
    t = np.linspace(0.0, 2.0 * math.pi, len(bnd), endpoint=False)
    circ = np.stack([np.cos(t), np.sin(t)], 1)
    V4, T4 = wk.grid_triangles(4, 4, no_ears=True)
    b4 = wk._grid_boundary_cycle(4, 4)
    t4 = np.linspace(0.0, 2.0 * math.pi, len(b4), endpoint=False)
    tutte(V4, T4, b4, np.stack([np.cos(t4), np.sin(t4)], 1))   # load the library, touch the device
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W, rel = tutte(V, T, bnd, circ)
    t_gpu = time.perf_counter() - t0
    t0 = time.perf_counter()
    Wo = ot.tutte(V, T, bnd, circ)
    t_cpu = time.perf_counter() - t0
    line = {"metric": "Tutte initializer wall time", "unit": "s", "value": t_gpu, "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"tutte_disk_{grid}", "vertices": int(V.shape[0]), "triangles": int(T.shape[0])},
            "rel_residual": rel, "max_diff_vs_oracle": float(np.abs(W - Wo).max()),
            "flipped": float(wk.flipped_fraction(W, T)),
            "cpu_baseline": {"value": t_cpu, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": "scipy sparse LU of the same system"}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.oracle_probe is not None:
        cells, iters, secs = args.oracle_probe
        m, times, setup_s = oracle_probe(int(cells), int(iters), float(secs))
        print(json.dumps({"tets": m, "times": times, "setup_s": setup_s}), flush=True)
        return 0
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "batch256":
        return run_batch(args, rank, world, local)
    if args.workload in ("uv_disk", "uv_heightfield"):
        return run_to_tolerance(args, local) if rank == 0 else 0
    if args.workload == "cube_handles":
        return run_handles(args, local) if rank == 0 else 0
    if args.workload == "tutte":
        return run_tutte(args, local) if rank == 0 else 0
    if args.workload == "cube_outcome":
        return run_outcome(args, local) if rank == 0 else 0
    if args.workload == "decompose":
        return run_decompose(args, local) if rank == 0 else 0
    if args.workload == "volume_correspondence":
        return run_volume_correspondence(args, local) if rank == 0 else 0

    import numpy as np
    import torch

    from paper_2107_05200_gb300 import workloads as wk
    from paper_2107_05200_gb300.solver import Solver

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    stream = torch.cuda.current_stream()
    wl = wk.cube_deform(cells=args.cells)
    sol = Solver.from_workload(wl, precision=args.precision, refine_sweeps=args.sweeps, factor=args.factor,
                               check_every=args.check_every, schedule=args.schedule, stream=stream.cuda_stream,
                               top_inverse_levels=args.top_inverse)
    info = sol.info()
    W0 = torch.tensor(wl.W0, dtype=torch.float64, device="cuda")
    sol.init(W0)
    if args.warmup > 0:
        sol.iterate(args.warmup, stop_at_tol=False)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st = sol.iterate(args.steps, stop_at_tol=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
        pg.barrier()
    value = world * args.steps / (ms / 1e3)

    # per-phase device times (CUDA events on the solver stream, eager launches)
    ph = sol.profile_phases(10)
    hbm_peak, peak_kind = measured_peaks()
    local_gbs = info["bytes_local_step"] / (ph["ms_local"] / 1e3) / 1e9
    wstep_gbs = args.sweeps * info["bytes_global_sweep"] / (ph["ms_wstep"] / 1e3) / 1e9
    # dominant kernel: the triangular passes of the W step (forward + backward per sweep)
    ms_pass = 0.5 * (ph["ms_solve_forward"] + ph["ms_solve_backward"])
    solve_gbs = info["bytes_solve_pass"] / (ms_pass / 1e3) / 1e9
    traffic = (profiled_solve_traffic() if args.cells == 64 and args.precision == "fp32" and
               info["top_inverse_levels"] == 0 else None)
    resid = sol.wstep_residual()

    # end to end through the public API with host buffers: init from pinned host W0,
    # iterate, read W back to pinned host memory
    W0h = torch.tensor(wl.W0, dtype=torch.float64).pin_memory()
    Wout = torch.empty_like(W0h).pin_memory()
    e2e_steps = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sol.init(W0h)
    sol.iterate(e2e_steps, stop_at_tol=False)
    sol.W(Wout)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * e2e_steps / e2e_s
    nbytes = wl.n * 3 * 8

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "elem_updates_per_s": value * wl.m,
        "config": bench_config(args, wl.m, wl.n, wl.rho, world),
        "roofline": {"bound": "hbm", "achieved": solve_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": solve_gbs / hbm_peak,
                     "traffic": None if traffic is None else 0.5 * (traffic[0] + traffic[1]),
                     "kernel": "k_solve_dynamic (W-step triangular passes, forward and backward)",
                     "bytes_per_launch": info["bytes_solve_pass"], "ms_per_launch": ms_pass,
                     "launches_per_step": 2 * args.sweeps, "peak_kind": peak_kind},
        "kernels": {
            "k_solve_dynamic_forward": {"ms": ph["ms_solve_forward"],
                                        "gbs": info["bytes_solve_pass"] / ph["ms_solve_forward"] / 1e6},
            "k_solve_dynamic_backward": {"ms": ph["ms_solve_backward"],
                                         "gbs": info["bytes_solve_pass"] / ph["ms_solve_backward"] / 1e6},
            "k_local_step": {"ms": ph["ms_local"], "gbs": local_gbs, "frac": local_gbs / hbm_peak,
                             "bytes": info["bytes_local_step"]},
        },
        "top_inverse": None if info["top_inverse_levels"] == 0 else {
            "levels": info["top_inverse_levels"], "cols": info["top_inverse_cols"],
            "ms": ph["ms_top_product"], "bytes": info["bytes_top_product"],
            "gbs": info["bytes_top_product"] / ph["ms_top_product"] / 1e6,
            "frac": info["bytes_top_product"] / ph["ms_top_product"] / 1e6 / hbm_peak,
            "setup_s": info["setup_seconds_top_inverse"]},
        "phases_ms": {k: v for k, v in ph.items() if k != "reps"},
        "wstep": {"achieved_gbs": wstep_gbs, "frac": wstep_gbs / hbm_peak,
                  "factor_entries": info["factor_entries"], "rel_residual": resid},
        "gpu_launches": int(args.steps * info["kernels_per_iteration"] +
                            math.ceil(args.steps / args.check_every) * info["kernels_per_check"]),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes / e2e_steps,
                "d2h_bytes_per_step": (nbytes + 96) / e2e_steps,
                "note": f"one solve call: init from host W0, {e2e_steps} iterations, W read back"},
        "clocks": clk,
        "final": {"e_prim": st["e_prim"], "e_dual": st["e_dual"], "n_flipped": st["n_flipped"]},
        "setup_s": {"analyze": info["setup_seconds_analyze"], "factor": info["setup_seconds_factor"],
                    "factor_on": args.factor},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(wl.m, wl.n, args.cpu_sample_cells, args.cpu_seconds, args.growth_cells, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sol.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
