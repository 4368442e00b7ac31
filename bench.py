#!/usr/bin/env python3
"""Benchmark of the CAV-multigrid-preconditioned FGMRES solve on one B300.

Metric: solves/s to a 1e-10 relative residual (||r||/||b||), one step = one FGMRES solve
of the elliptic-membrane system on a built hierarchy (the whole hot path: residuals,
patch gathers, batched patch-inverse applies, weighted scatters, transfers, coarse solve,
Arnoldi and Givens).  Set-up (E_E assembly, Galerkin levels, CAV sets, batched LU) is
timed separately and reported as setup_ms (cav_setup on an assembled system, the median of
three calls after the first; setup_ms_first_call adds ib_setup and the process's first-call
costs) and setup_plus_solve_per_s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own independently seeded system (replicas:
the path has no exchange step); value = all solves / max over ranks of the timed span.
`--impl reference` times the FP64 CPU oracle on the same workload (rank 0 only).
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ib_workloads as W  # noqa: E402

METRIC = "solves/s to 1e-10 rel. residual (mixed+learned vs plain FP64); sweep HBM GB/s"
DEFAULT_NU = 2
# coloured smoother on the finest level only: sweeps per side of the additive smoother below it
# (the coarse levels are cheap; 4 took the N=256 membrane from 30 to 21 iterations)
NU_COARSE_ADDITIVE = 4
# the N=256 membrane headline sweeps its coloured finest level once, after the coarse correction
# only: 26 FGMRES iterations against 19 with a sweep on each side (the oracle's counts), but a
# V-cycle of 0.92 ms against 1.42 ms, 40.6 against 36.6 solves/s
HEADLINE_FINEST_NU = (0, 1)
DEFAULT_ALPHA = 0.85
# the membrane workloads' coarsest grid: a 32 x 32 level solved directly (its dense inverse
# applied as one GEMV) took the N=256 headline from 21 to 19 FGMRES iterations and 28.3 to
# 35.7 solves/s against the 8 x 8 grid of the paper's tests, for about 100 ms more set-up
DEFAULT_COARSEST = 32
MAXIT = 150

# DRAM traffic of the roofline's unit from an ncu capture of the same bench command
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel source it was taken
# on (keyed by the smoother, precision, N and the hash of the kernel's source file); null once
# that source changes.
NCU_TRAFFIC = {
    # coloured: the 105 k_colour_step launches of one finest-level sweep, 422.50 MB read, 0 MB
    # written back within them (the iterate's writes stay in L2)
    "coloured:fp32:256:colour.cu:3f8ca244c58eae2c": 422.51e6,
    # additive: one finest-level patch-apply launch (k_patch_apply_tma<float, 4, 8192>),
    # 289.65 MB read + 5.05 MB written (taken at sweep.cu 63b9c19db8897f36; the file has since
    # changed only in the V-cycle's host code, the kernel not at all)
    "additive:fp32:256:sweep.cu:694b9d8267ec265e": 294.70e6,
}


def max_over_ranks(value: float, dist, device=None) -> float:
    """The largest per-rank timed span (all ranks wait for the slowest): an all-reduce MAX
    over the process group, or the value itself without one."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, span_s: float) -> float:
    """Units all ranks processed divided by the slowest rank's timed span."""
    return world * units_per_rank / span_s


def workload(seed_offset: int = 0, N: int = 256):
    # config 2's membrane at N = 256; the same law and ellipse at N = 512 for the scale check
    rec = W.config2(256, 1e4) if N == 256 else W.membrane_ellipse(N, 1e4)
    if seed_offset:
        rec.seed += 7919 * seed_offset
    return rec


def workload_desc(rec) -> str:
    return (f"elliptic membrane (semi-axes 0.3, 0.2), N={rec.N}, M={rec.M} markers, kappa_s=1e4, "
            f"rho=1, mu=1e-2, dt=h/2, seeded uniform[-1,1] RHS")


S_BYTES = {"fp64": 8, "fp32": 4, "bf16": 2}


def apply_bytes(li: dict, precision: str) -> int:
    """Algorithmic bytes of one finest-level patch apply: the stored inverses and, per slot, the
    index, the gathered residual, the two scales and the correction written."""
    return li["enlarged_sum_n2"] * S_BYTES[precision] + li["enlarged_sum_n"] * 36


def sweep_bytes(li: dict, N: int, precision: str, mean: bool = True) -> int:
    """Algorithmic bytes of one whole additive sweep (Eq. additive_cav_saddle) on a level: the
    enlarged inverses and their per-slot data, the residual pass (read w, b; write r), the
    scatter pass (read w, r; write w), the E_E rows, the transpose incidence, and with `mean`
    the mean removal (read and write p)."""
    NN = N * N
    return (li["enlarged_sum_n2"] * S_BYTES[precision] + li["enlarged_sum_n"] * (4 + 8 + 8 + 8 + 8 + 4 + 8)
            + 3 * NN * 8 * 3 + 3 * NN * 8 * 3 + li["ee_nnz"] * 12 + 3 * NN * 8 + (2 * NN * 8 if mean else 0))


def headline_config(args, rec, world: int) -> dict:
    """The workload the headline line measures, the same dict on both arms (this GPU arm and the
    oracle's reference arm): the system, its V-cycle and the solve's stopping rule."""
    return {"workload": workload_desc(rec), "smoother": smoother_desc(args), "nu_pre": args.nu_pre,
            "nu_post": args.nu_post, "alpha": args.alpha, "coarsest_N": args.coarsest, "rtol": 1e-10, "maxit": MAXIT,
            "l2": "flushed (256 MB write) before every timed GPU solve",
            "parallelism": f"replicas x{world}"}


def kernel_hash(name: str = "sweep.cu") -> str:
    with open(os.path.join(ROOT, "paper_2608_14310_b300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(device_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_cycle(args, n_smooth: int):
    """The oracle's V-cycle arguments for the bench's smoother on a hierarchy with n_smooth
    smoothing levels: per-level modes, pre-sweeps and post-sweeps."""
    if args.smoother == "coloured" and args.coloured_levels == 1:
        below = [args.nu_additive] * (n_smooth - 1)
        return ["coloured"] + ["additive"] * (n_smooth - 1), [args.nu_pre] + below, [args.nu_post] + below
    if args.smoother == "coloured":
        return "coloured", args.nu_pre, args.nu_post
    return "additive", args.nu_pre, args.nu_post


def golden_for(args):
    """The oracle's own iteration count for the bench's V-cycle (tests/golden), or None."""
    g = golden_iters()
    if not g:
        return None
    if args.coarsest != 8:
        g = g.get(f"coarsest_{args.coarsest}")
        if not g:
            return None
    if args.smoother == "coloured" and args.coloured_levels == 1 and args.nu_additive == 4:
        gkey = {(1, 1): g.get("coloured_finest"), (0, 1): g.get("coloured_finest_post_only")}.get(
            (args.nu_pre, args.nu_post))
    elif args.smoother == "additive" and args.nu_pre == args.nu_post == 2:
        gkey = g
    else:
        gkey = None
    return gkey.get("iters") if gkey else None


def cpu_baseline_sample(iters: int, args, timeout_s: int = 900):
    """The oracle as it stands, single-threaded, on a bounded sample of the same workload: one
    oracle V-cycle (timed alone), and the oracle's own FGMRES run for `iters` iterations with
    the identity in place of the V-cycle (Arnoldi with modified Gram-Schmidt, Givens, the
    K_E products and the final update at the solve's real Krylov dimensions; rtol 0 so it
    runs all of them).  A solve is then iters x V-cycle + that FGMRES run."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
import numpy as np
import ib_workloads as W
from oracle import fgmres as fg, multigrid as mg
rec = W.config2(256, 1e4)
t0 = time.perf_counter()
levels = mg.build_hierarchy(rec, %d, "cav")
modes, pre, post = %s, %s, %s
if "coloured" in str(modes):
    mg.level_colours(levels[0])  # the colour classes are set-up, not timed
t_setup = time.perf_counter() - t0
b = rec.rhs()
K = levels[0].KE
t0 = time.perf_counter()
z = mg.vcycle(levels, b, pre, post, modes, %r)
t_vcycle = time.perf_counter() - t0
t0 = time.perf_counter()
fg.fgmres(lambda v: K @ v, b, lambda r: r, rtol=0.0, maxit=%d)
t_rest = time.perf_counter() - t0
print(json.dumps({"t_setup": t_setup, "t_vcycle": t_vcycle, "t_rest": t_rest}))
""" % (ROOT, args.coarsest, *(repr(v) for v in oracle_cycle(args, n_smooth_levels(256, args.coarsest))),
       DEFAULT_ALPHA, iters)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             timeout=timeout_s, env=env)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # pragma: no cover
        return {"error": str(e)}


def n_smooth_levels(N: int, coarsest: int) -> int:
    """Smoothing levels of the hierarchy (halve while N / 2 >= coarsest, as cav_setup does)."""
    n = 0
    while N // 2 >= coarsest and N % 2 == 0:
        N //= 2
        n += 1
    return n


def golden_iters():
    p = os.path.join(ROOT, "tests", "golden", "bench_oracle_iterations.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return None


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle.fgmres as fg
    import oracle.multigrid as mg
    rec = workload()
    set_sweeps(args)
    t0 = time.perf_counter()
    levels = mg.build_hierarchy(rec, args.coarsest, "cav")
    modes, pre, post = oracle_cycle(args, len(levels) - 1)
    if "coloured" in str(modes):
        mg.level_colours(levels[0])
    t_setup = time.perf_counter() - t0
    b = rec.rhs()
    K = levels[0].KE
    iters = golden_for(args) or 77
    # the oracle's FGMRES without its V-cycles (identity preconditioner, all `iters` iterations):
    # Arnoldi, Givens, K_E products and the final update at the solve's Krylov dimensions
    t0 = time.perf_counter()
    fg.fgmres(lambda v: K @ v, b, lambda r: r, rtol=0.0, maxit=iters)
    t_rest = time.perf_counter() - t0

    def step():
        return mg.vcycle(levels, b, pre, post, modes, DEFAULT_ALPHA)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        step()
        times.append(time.perf_counter() - t)
    t_iter = statistics.mean(times) + t_rest / iters
    value = 1.0 / (t_iter * iters)
    sample = (f"each step = one oracle V-cycle ({smoother_desc(args)}) on the full "
              f"N=256 system; solves/s = 1 / ({iters} x mean step time + {t_rest:.2f} s, the oracle's own "
              f"FGMRES run for {iters} iterations with the identity in place of the V-cycle: Arnoldi, "
              f"Givens, K_E products); {iters} = the oracle's own iteration count (tests/golden); "
              f"hierarchy set-up {t_setup:.1f} s untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_iter, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": headline_config(args, rec, world),
            "measures": "the FP64 CPU oracle (single thread) on the same system and V-cycle",
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def set_sweeps(args) -> None:
    """Sweeps per side where not given: 2 for the additive smoother; 1 on the coloured levels,
    whose pre-sweeps (--nu-pre) and post-sweeps (--nu-post) may differ; on the N=256 membrane
    headline's form (coloured finest level, additive below) none before the coarse correction
    and one after it."""
    if (args.nu is None and args.workload == "membrane256" and args.smoother == "coloured"
            and args.coloured_levels == 1):
        if args.nu_pre is None:
            args.nu_pre = HEADLINE_FINEST_NU[0]
        if args.nu_post is None:
            args.nu_post = HEADLINE_FINEST_NU[1]
    if args.nu is None:
        args.nu = 1 if args.smoother == "coloured" else DEFAULT_NU
    if args.nu_pre is None:
        args.nu_pre = args.nu
    if args.nu_post is None:
        args.nu_post = args.nu


def smoother_kw(args) -> dict:
    return {"smoother": args.smoother, "coloured_levels": args.coloured_levels, "nu_additive": args.nu_additive}


def smoother_desc(args) -> str:
    if args.smoother == "additive":
        return f"weighted additive CAV (alpha {args.alpha}), {args.nu_pre}+{args.nu_post} sweeps on every level"
    lv = "every level" if args.coloured_levels == 0 else f"the {args.coloured_levels} finest level(s)"
    extra = "" if args.coloured_levels == 0 else f", additive {args.nu_additive}+{args.nu_additive} below"
    return f"coloured multiplicative CAV, {args.nu_pre}+{args.nu_post} sweeps on {lv}{extra}"


def run_batch(args, api, torch, dist, rank, world, local):
    """64 uneven systems (grid, force law, stiffness drawn per system) solved together by
    fgmres_solve_batched; one step = one batched solve of all 64; value = systems/s.  With
    --batch-loop device (the default) a batched solve is one CUDA graph launch, the 64 systems'
    FGMRES loops running on the device side by side; the host-driven lockstep is timed beside it."""
    recs = W.config4(64)
    if rank:
        for r in recs:
            r.seed += 7919 * rank
    dev = torch.device("cuda", local)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    t0 = time.perf_counter()
    syss = [api.ib_setup(r) for r in recs]
    hs = [api.cav_setup(s, nu_pre=args.nu_pre, nu_post=args.nu_post, alpha=args.alpha, precision="fp32", autotune=True,
                        **smoother_kw(args))
          for s in syss]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    bs = [torch.from_numpy(r.rhs()).to(dev) for r in recs]
    xs = [torch.zeros_like(b) for b in bs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def solve(loop=args.batch_loop):
        for x in xs:
            x.zero_()
        return api.fgmres_solve_batched(syss, hs, bs, xs, rtol=1e-10, maxit=MAXIT, loop=loop)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    launches0 = api.ib_launch_count()
    times, last = [], None
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        last = solve()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    launches = api.ib_launch_count() - launches0
    clk = clocks.stop()
    total = max_over_ranks(sum(times), dist, dev)
    # the other loop on the same batch, for comparison (untimed by the headline)
    other = "host" if args.batch_loop == "device" else "device"
    solve(other)
    ot = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        solve(other)
        torch.cuda.synchronize()
        ot.append(time.perf_counter() - t)
    its = [i["iters"] for i in last]
    flagged = [i["converged"] for i in last]
    # a system counts as solved only when its true residual (recomputed in FP64 after the solve)
    # reached 1e-10; FGMRES's own estimate can reach it while the true residual does not (the
    # stiffest draws, where FP64 evaluation of K_E w loses the last digits); attempted systems
    # and the estimate's count are reported beside
    conv = [1 if (i["relres_true"] <= 1e-10) else 0 for i in last]
    value = whole_job_rate(int(sum(conv)) * args.steps, world, total)
    attempted = whole_job_rate(len(recs) * args.steps, world, total)
    kappa = [r.k_bend if r.law == W.LAW_BEAM else (r.k_stretch if r.law == W.LAW_MEMBRANE else r.k_target)
             for r in recs]  # each system's drawn stiffness (the law's primary coefficient)
    stiff = sorted(range(len(recs)), key=lambda q: -kappa[q])
    stiff_conv = int(sum(conv[q] for q in stiff[:len(recs) // 2]))
    variants = {}
    for h in hs:
        for l in range(api.cav_num_levels(h) - 1):
            v = api.cav_get_level_info(h, l)["apply_variant"]
            variants[v] = variants.get(v, 0) + 1
    line = {"metric": METRIC, "value": value, "unit": "systems solved to 1e-10 per s (64-system batches)",
            "attempted_systems_per_s": attempted,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "64 uneven IB systems: N from {64,96,128,192,256}, law from {target, membrane, "
                                   "beam}, stiffness log-uniform [1e2,1e6], M=4N, seeded RHS; FP32 inverses, "
                                   "autotuned patch-apply variants, fgmres_solve_batched",
                       "nu_pre": args.nu_pre, "nu_post": args.nu_post, "alpha": args.alpha, "maxit": MAXIT,
                       "smoother": smoother_desc(args),
                       "converged": int(sum(conv)), "converged_by_fgmres_estimate": int(sum(flagged)),
                       "converged_of_stiffest_half": stiff_conv, "iters_median": int(statistics.median(its)),
                       "iters_max": int(max(its)), "autotuned_variant_counts": variants,
                       "l2": "flushed (256 MB write) before every timed batch"},
            "batch_loop": args.batch_loop,
            "other_loop": {"loop": other, "ms_per_step": 1e3 * statistics.mean(ot)},
            "systems": [{"N": r.N, "law": {W.LAW_BEAM: "beam", W.LAW_MEMBRANE: "membrane"}.get(r.law, "target"),
                         "kappa": kappa[q], "iters": last[q]["iters"], "converged": conv[q],
                         "relres_true": last[q]["relres_true"]} for q, r in enumerate(recs)],
            "setup_s_all_64": setup_s, "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def additive_sweep_entry(li: dict, N: int, precision: str, ms: float) -> dict:
    """The finest-level additive sweep (Eq. additive_cav_saddle) as measured through cav_sweep."""
    nb = sweep_bytes(li, N, precision)
    return {"level": 0, "form": "fused cooperative kernel" if li["sweep_form"] else "separate kernels",
            "ms": ms, "algorithmic_bytes": nb, "gbs": nb / (ms * 1e-3) / 1e9,
            "frac_of_hbm": nb / (ms * 1e-3) / 1e9 / peaks()[0], "autotuned_us_separate_fused": li["sweep_us"],
            "note": "one cav_sweep (residual, patch apply, scatter, mean removal) of the weighted additive CAV "
                    "smoother on the finest level: 10 sweeps captured in a CUDA graph, median of 3 replays / 10 "
                    "(the inverses exceed L2, so each sweep streams them from HBM)"}


def graph_sweep_ms(api, torch, hier, b, reps: int = 10) -> float:
    """Device time of one finest-level cav_sweep: `reps` sweeps captured into one CUDA graph
    (cav_sweep skips its host-side status check while captured), replayed three times, the
    median replay / reps.  The finest level's inverses (hundreds of MB) exceed L2, so every
    sweep streams them from HBM."""
    w = torch.zeros_like(b)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            api.cav_sweep(hier, 0, b, w)  # warm-up outside capture (checks the status word)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            api.cav_sweep(hier, 0, b, w)
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / reps)
    api.cav_sweep(hier, 0, b, w)  # reads the status word the replays may have set
    return statistics.median(ts)


def run_beam512(args, api, torch, rank):
    """The stretched beam on a 512 x 512 grid (2048 markers, kappa_b 1e3, kappa_s 1e5): finest-level
    sweep and patch-apply bandwidth with BF16 and with FP64 inverses, and the FGMRES attempt (the
    system is beyond FP64's reach at 1e-10; reported, not claimed)."""
    if rank:
        return 0
    rec = W.config3()
    dev = torch.device("cuda", 0)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    sysm = api.ib_setup(rec)
    b = torch.from_numpy(rec.rhs()).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    peak, kind = peaks()
    res = {}
    for prec in ("bf16", "fp64"):
        t0 = time.perf_counter()
        h = api.cav_setup(sysm, nu_pre=args.nu, nu_post=args.nu, alpha=args.alpha, precision=prec, autotune=True)
        setup_s = time.perf_counter() - t0
        li = api.cav_get_level_info(h, 0)
        s_b = {"fp64": 8, "bf16": 2}[prec]
        alg = li["enlarged_sum_n2"] * s_b + li["enlarged_sum_n"] * 36
        w = torch.zeros_like(b)
        for _ in range(3):
            api.cav_sweep(h, 0, b, w)
        api.cav_profile(h, True)
        for _ in range(10):
            api.cav_sweep(h, 0, b, w)
        n_apply, apply_ms = api.cav_profile_read(h)
        api.cav_profile(h, False)
        sw = [graph_sweep_ms(api, torch, h, b)]
        api.cav_profile(h, False)
        x = torch.zeros_like(b)
        t1 = time.perf_counter()
        info = api.fgmres_solve(sysm, h, b, x, rtol=1e-10, maxit=60, history=False)
        solve_s = time.perf_counter() - t1
        achieved = alg / (apply_ms / n_apply * 1e-3) / 1e9
        res[prec] = {"setup_s": setup_s, "inverse_bytes": li["inverse_bytes"], "enlarged_patches": li["n_enlarged"],
                     "max_n": li["max_n"], "apply_variant": li["apply_variant"],
                     "apply_us": 1e3 * apply_ms / n_apply, "apply_gbs": achieved, "apply_frac": achieved / peak,
                     "sweep_ms": statistics.median(sw),
                     "fgmres_60": {"iters": info["iters"], "converged": info["converged"],
                                   "relres_true": info["relres_true"], "seconds": solve_s}}
        h.close()
    line = {"workload": "stretched beam N=512, 2048 markers, kappa_b 1e3, kappa_s 1e5 (config 3)",
            "peak_gbs": peak, "peak_kind": kind, "results": res}
    print(json.dumps(line), flush=True)
    return 0


# Sec. 5.3's refinement study (Table 3): averages over the paper's whole run
PAPER_FIBER = {16: (8.65, 13, 2.00), 32: (9.02, 14, 1.48), 64: (9.15, 15, 1.45), 128: (9.53, 16, 1.60)}


def run_fiber(args, api, torch, rank):
    """The flow-past-a-fiber benchmark (Sec. 5.3) in its channel: `nsteps` time steps from rest,
    each solved by Newton's method with every Newton system solved by CAV-preconditioned
    FGMRES (coloured multiplicative smoother, 1 + 1 sweeps, hierarchy rebuilt per system).
    One step = one time step (ib_setup at X^n, the step's right-hand side, then per Newton
    iterate: E_E at X_k, Newton right-hand side and residual, cav_setup, fgmres_solve).
    value = Newton-system solves per second (set-up included)."""
    from paper_2608_14310_b300.fiber_channel import FiberChannel
    if rank:
        return 0
    rec = W.fiber_channel(args.fiber_n)
    prec = "fp64" if args.precision == "bf16" else args.precision
    fc = FiberChannel(rec, cav=dict(kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured",
                                    precision=prec), fgmres_rtol=args.fiber_rtol)
    n = 3 * rec.N * rec.N
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    t = 0.0
    newton, its, secs, nonconv = [], [], [], 0
    launches0 = api.ib_launch_count()
    clocks = ClockSampler(0)
    for s in range(args.nsteps):
        t += rec.dt
        w, X, hist, infos, sec = fc.step(w, t)
        if args.trace and s % 50 == 0:
            Xa = np.asarray(X)
            print(f"step {s}: markers y in [{Xa[:, 1].min():.4f}, {Xa[:, 1].max():.4f}], x in "
                  f"[{Xa[:, 0].min():.4f}, {Xa[:, 0].max():.4f}], Newton {len(hist) - 1}, FGMRES "
                  f"{[i['iters'] for i in infos]}", file=sys.stderr, flush=True)
        newton.append(len(hist) - 1)
        its.extend(i["iters"] for i in infos)
        nonconv += sum(1 for i in infos if not i["converged"])
        secs.append(sec)
    clk = clocks.stop()
    launches = api.ib_launch_count() - launches0
    timed = secs[args.warmup:] if len(secs) > args.warmup else secs
    solves_timed = sum(newton[args.warmup:]) if len(secs) > args.warmup else sum(newton)
    paper = PAPER_FIBER.get(args.fiber_n)
    line = {"metric": METRIC, "value": solves_timed / sum(timed), "unit": "Newton-system solves/s (set-up + FGMRES)",
            "n_gpus": 1, "steps": len(timed), "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f64+f32", "data": "synthetic",
            "config": {"workload": (f"flow past a clamped fiber (Sec. 5.3): channel (0,2)^2, {rec.N}x{rec.N} cells, "
                                    f"inflow ramped to U=1 on the top wall, traction outflow with backflow "
                                    f"term, Re=200, {rec.M} markers, dt=0.05h; {args.nsteps} steps from rest"),
                       "smoother": "coloured multiplicative CAV 1+1, hierarchy rebuilt per Newton system",
                       "precision": prec + " patch inverses", "fgmres_rtol": args.fiber_rtol,
                       "newton": "stop at 1e-8 relative to the first Newton residual (or 1e-8 absolute)"},
            "newton_per_step_mean": float(np.mean(newton)), "newton_per_step_max": int(max(newton)),
            "fgmres_per_newton_mean": float(np.mean(its)), "fgmres_per_newton_max": int(max(its)),
            "fgmres_not_converged": nonconv, "ms_per_newton_solve": 1e3 * sum(timed) / max(solves_timed, 1),
            "paper": ({"fgmres_per_newton_mean": paper[0], "fgmres_per_newton_max": paper[1],
                       "newton_per_step_mean": paper[2], "note": "averaged over the paper's whole run, tol 1e-9"}
                      if paper else None),
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_learned_channel(args, api, torch, rank):
    """The learned initial guess on the fiber benchmark (Sec. 5.3, config 5): the series is
    stepped with plain FP64 inverses and the previous step's solution as Newton's start for the
    first 75 % of the steps, the CNN is trained on them, and every remaining step is solved five
    ways from the same state: plain FP64 + previous solution, and FP32 inverses + previous
    solution / linear extrapolation / quadratic extrapolation / the CNN's prediction (which
    corrects the `--learned-base` extrapolation).  Newton stops at 1e-9 of the step's base
    right-hand side and FGMRES at 1e-10 of each Newton system's, references that do not depend
    on the guess.  value = time steps/s of FP32 + learned over the test steps."""
    from paper_2608_14310_b300.learned_guess import ChannelSeries, LearnedGuess
    if rank:
        return 0
    rec = W.fiber_channel(args.fiber_n)
    cs = ChannelSeries(rec, cav=dict(kind="cav", coarsest_N=8, nu_pre=1, nu_post=1, smoother="coloured",
                                     precision="fp64"))
    n_train = int(0.75 * args.nsteps)
    t0 = time.perf_counter()
    for _ in range(n_train):
        cs.step()
    t_series = time.perf_counter() - t0
    lg = LearnedGuess(rec.N, hidden=32, n_hidden=3, base=args.learned_base, history=args.learned_history)
    start = int(args.train_start * n_train)
    n_fit = n_train - max(1, n_train // 10)  # the last tenth of the training range is held out
    lg.fit_scales(cs, n_fit, start=start)
    tinfo = lg.train(cs, n_fit, iters=args.train_iters, batch=16, lr=1e-3, start=start)
    calib = lg.calibrate(cs, n_fit, n_train)
    calib.update(lg.calibrate_residual(cs, n_fit, n_train))
    variants = (("plain_fp64_previous", None, "fp64"),
                ("fp32_previous", None, "fp32"),
                ("fp32_extrapolated", lambda s: lg.extrapolate(s, 1), "fp32"),
                ("fp32_quadratic", lambda s: lg.extrapolate(s, 2), "fp32"),
                ("fp32_learned_uncalibrated", lambda s: lg.predict(s, calibrated=False), "fp32"),
                ("fp32_learned_heldout", lambda s: lg.predict(s), "fp32"),
                ("fp32_learned", lambda s: lg.predict(s, online=True), "fp32"))
    res = {v[0]: [] for v in variants}
    launches0 = api.ib_launch_count()
    clocks = ClockSampler(0)
    lg.start_online(cs, n_fit, n_train)
    gam = []
    for _ in range(args.nsteps - n_train):
        gam.append(lg.online_gamma())
        for lab, inf in cs.step(variants):
            res[lab].append(inf)
        lg.observe(cs)  # the step just solved joins the online scale (past data only)
    clk = clocks.stop()
    launches = api.ib_launch_count() - launches0
    summ = {}
    for lab, v in res.items():
        ns = sum(r["newton"] for r in v)
        summ[lab] = {"steps_per_s": len(v) / sum(r["seconds"] for r in v),
                     "ms_per_step": 1e3 * float(np.mean([r["seconds"] for r in v])),
                     "newton_per_step": ns / len(v),
                     "fgmres_per_step": float(np.mean([r["fgmres_total"] for r in v])),
                     "fgmres_per_newton": sum(r["fgmres_total"] for r in v) / max(ns, 1),
                     "first_residual_geomean": float(np.exp(np.mean(np.log([max(r["r0"], 1e-300) for r in v])))),
                     "all_converged": all(r["converged"] for r in v)}
    line = {"metric": METRIC, "value": summ["fp32_learned"]["steps_per_s"], "unit": "time steps/s (Newton + CAV-FGMRES)",
            "n_gpus": 1, "steps": args.nsteps - n_train, "warmup": n_train, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": (f"flow past a clamped fiber (Sec. 5.3) in its channel, {rec.N}x{rec.N} cells, "
                                    f"Re=200, dt=0.05h, {args.nsteps} steps from rest; CNN (3x3 convolutions, 32 "
                                    f"channels, 3 hidden layers) on the last {args.learned_history} steps' u, v, p and spread force, "
                                    f"correcting the {args.learned_base} extrapolation, trained on steps "
                                    f"{int(args.train_start * n_train)}..{n_fit} ({args.train_iters} Adam iterations, "
                                    f"batch 16), its correction's per-field scale fitted on the held-out steps "
                                    f"{n_fit}..{n_train} (least squares, then a search on the held-out first "
                                    f"Newton residual), tested on the last {args.nsteps - n_train}"),
                       "smoother": "coloured multiplicative CAV 1+1, hierarchy rebuilt per Newton system",
                       "tolerances": "Newton 1e-9 of ||b_step||, FGMRES 1e-10 of ||rhs||"},
            "test_steps": summ, "calibration": calib,
            "online_gamma_first_mean_last": [gam[0], np.mean(gam, axis=0).tolist(), gam[-1]],
            "series_s": t_series, "train_s": tinfo["train_s"],
            "train_loss_first_last": [tinfo["losses"][0][1], tinfo["losses"][-1][1]],
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args, api, torch, rank, world):
    """Time series of a tethered elastic ring in a time-periodic shear forcing (periodic box,
    dt = 0.05 h, one linear solve per step, hierarchy rebuilt per step).  Steps 1..75% use the
    previous-step guess with FP64 inverses and train the CNN; on the remaining steps every
    system is solved three ways: plain FP64 + previous guess, FP32 + previous guess, FP32 +
    learned guess.  value = solves/s of FP32 + learned over the test steps."""
    from paper_2608_14310_b300.learned_guess import LearnedGuess, TimeSeries
    if rank:
        return 0
    rec = W.tethered_ring(args.grid, dt_factor=args.dtfactor)
    ts = TimeSeries(rec, W.shear_forcing, nu=args.nu, alpha=args.alpha, precision="fp64")
    n_train = int(0.75 * args.nsteps)
    t0 = time.perf_counter()
    for _ in range(n_train):
        ts.step()
    t_train_series = time.perf_counter() - t0
    lg = LearnedGuess(rec.N, hidden=32, n_hidden=3)
    lg.fit_scales(ts, n_train)
    tinfo = lg.train(ts, n_train, iters=1500, batch=16, lr=1e-3)
    res = {"plain_fp64": [], "fp32_previous": [], "fp32_extrapolated": [], "fp32_learned": []}
    for _ in range(args.nsteps - n_train):
        out = ts.step(guesses=(("fp32_learned", lambda s: lg.predict(s), "fp32"),
                               ("fp32_extrapolated", lambda s: lg.extrapolate(s), "fp32"),
                               ("fp32_previous", None, "fp32"),
                               ("plain_fp64", None, "fp64")))
        for lab, inf, ms in out:
            res[lab].append((inf["iters"], ms, inf["converged"], inf["relres_true"], inf["r0"]))
    summ = {k: {"iters_mean": float(np.mean([r[0] for r in v])), "solve_ms_mean": float(np.mean([r[1] for r in v])),
                "solves_per_s": 1e3 / float(np.mean([r[1] for r in v])),
                "converged": int(sum(r[2] for r in v)), "relres_max": float(max(r[3] for r in v)),
                "r0_geomean": float(np.exp(np.mean(np.log([max(r[4], 1e-300) for r in v]))))}
            for k, v in res.items()}
    line = {"metric": METRIC, "value": summ["fp32_learned"]["solves_per_s"], "unit": "solves/s",
            "n_gpus": 1, "steps": args.nsteps - n_train, "warmup": n_train, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"tethered elastic ring (radius 0.2, spacing h/2, kappa_s 1, kappa_t 10) in a "
                                   f"time-periodic shear forcing, periodic box N={rec.N}, dt={args.dtfactor}h, "
                                   f"{args.nsteps} steps, "
                                   f"rtol 1e-10 (||b||), hierarchy rebuilt per step; CNN trained on the first "
                                   f"{n_train} steps (1500 Adam iterations, batch 16), tested on the rest",
                       "nu": args.nu, "alpha": args.alpha},
            "test_steps": summ, "train_series_s": t_train_series, "train_s": tinfo["train_s"],
            "train_loss_first_last": [tinfo["losses"][0][1], tinfo["losses"][-1][1]]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--nu", type=int, default=None,
                    help="sweeps per side (default: 2 additive, 1 coloured)")
    ap.add_argument("--nu-pre", type=int, default=None,
                    help="sweeps before the coarse correction (default --nu); with the coloured smoother on "
                         "the finest level only, its sweeps (the additive levels take --nu-additive)")
    ap.add_argument("--nu-post", type=int, default=None, help="sweeps after the coarse correction, as --nu-pre")
    ap.add_argument("--smoother", default=None, choices=["additive", "coloured"],
                    help="additive: Eq. additive_cav_saddle on every level; coloured: the multiplicative "
                         "sweep of Sec. 3.3 visited colour class by colour class (default: coloured on the "
                         "finest level, additive below; on batch64 it stops the stiff beam draws, which no "
                         "preconditioner brings to 1e-10 in FP64, at their first non-finite step instead of "
                         "after maxit iterations)")
    ap.add_argument("--coloured-levels", type=int, default=1,
                    help="coloured smoother: levels (finest first) that use it, 0 = all; coarser ones additive")
    ap.add_argument("--nu-additive", type=int, default=NU_COARSE_ADDITIVE,
                    help="coloured smoother: sweeps per side on its additive levels")
    ap.add_argument("--alpha", type=float, default=DEFAULT_ALPHA)
    ap.add_argument("--coarsest", type=int, default=None,
                    help="coarsest grid of the membrane workloads' hierarchies, solved directly (default 32: a "
                         "3073-unknown dense inverse, factorised on every SM at set-up; the paper's own tests "
                         "use 8)")
    ap.add_argument("--loop", default="device", choices=["device", "host"],
                    help="FGMRES iterations driven on the device (each solve one CUDA graph launch) or by the host")
    ap.add_argument("--connections", type=int, default=32,
                    help="--workload batch64: CUDA_DEVICE_MAX_CONNECTIONS for the run (0: leave as is)")
    ap.add_argument("--batch-loop", default="device", choices=["device", "host"],
                    help="--workload batch64: device = one CUDA graph launch per batched solve (FGMRES loops "
                         "under conditional nodes); host = host-driven lockstep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the plain-FP64 and other-smoother comparisons (a short run, e.g. under a profiler)")
    ap.add_argument("--workload", default="membrane256",
                    choices=["membrane256", "membrane512", "batch64", "learned", "beam512", "fiber",
                             "learned_channel"])
    ap.add_argument("--learned-base", default="quadratic", choices=["linear", "quadratic"],
                    help="--workload learned_channel: the extrapolation the CNN corrects")
    ap.add_argument("--trace", action="store_true", help="--workload fiber: print marker ranges every 50 steps")
    ap.add_argument("--train-iters", type=int, default=1500, help="--workload learned_channel: Adam iterations")
    ap.add_argument("--train-start", type=float, default=0.4,
                    help="--workload learned_channel: train on steps [train_start, 1) x the training range (after "
                         "the inflow ramp)")
    ap.add_argument("--learned-history", type=int, default=4, choices=[3, 4],
                    help="--workload learned_channel: steps of history the CNN sees (4: as time differences)")
    ap.add_argument("--fiber-n", type=int, default=32,
                    help="--workload fiber: the paper's N (channel of 2N x 2N cells): 16, 32, 64, 128")
    ap.add_argument("--fiber-rtol", type=float, default=1e-10, help="--workload fiber: FGMRES tolerance")
    ap.add_argument("--grid", type=int, default=64, help="grid for --workload learned")
    ap.add_argument("--nsteps", type=int, default=2000, help="time steps for --workload learned")
    ap.add_argument("--dtfactor", type=float, default=0.05, help="dt / h for --workload learned")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.coarsest is None:
        args.coarsest = DEFAULT_COARSEST if args.workload in ("membrane256", "membrane512") else 8
    if args.smoother is None:
        args.smoother = "coloured"
    set_sweeps(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch64" and args.connections:
        # 64 systems' streams (or graph branches) in flight at once: more hardware work queues
        # than the default 8, read when the CUDA context is created
        os.environ["CUDA_DEVICE_MAX_CONNECTIONS"] = str(args.connections)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2608_14310_b300 import build
    build.build()
    from paper_2608_14310_b300 import api

    if args.workload == "batch64":
        return run_batch(args, api, torch, dist, rank, world, local)
    if args.workload == "learned":
        return run_learned(args, api, torch, rank, world)
    if args.workload == "beam512":
        return run_beam512(args, api, torch, rank)
    if args.workload == "fiber":
        return run_fiber(args, api, torch, rank)
    if args.workload == "learned_channel":
        return run_learned_channel(args, api, torch, rank)

    rec = workload(rank, 512 if args.workload == "membrane512" else 256)
    n = 3 * rec.N * rec.N
    dev = torch.device("cuda", local)
    b = torch.from_numpy(rec.rhs()).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    sysm = api.ib_setup(rec)
    hier = api.cav_setup(sysm, coarsest_N=args.coarsest, nu_pre=args.nu_pre, nu_post=args.nu_post, alpha=args.alpha,
                         precision=args.precision,
                         autotune=True, **smoother_kw(args))
    e1.record()
    torch.cuda.synchronize()
    setup_first_ms = e0.elapsed_time(e1)
    # the set-up as a program that builds hierarchies repeatedly pays it (a Newton loop):
    # three more cav_setup calls on the same system, the median reported
    warm = []
    torch.cuda.nvtx.range_push("warm_setup")  # lets a profiler select these set-ups
    for _ in range(3):
        e0.record()
        hw = api.cav_setup(sysm, coarsest_N=args.coarsest, nu_pre=args.nu_pre, nu_post=args.nu_post, alpha=args.alpha,
                           precision=args.precision, autotune=True, **smoother_kw(args))
        e1.record()
        torch.cuda.synchronize()
        warm.append(e0.elapsed_time(e1))
        hw.close()
    torch.cuda.nvtx.range_pop()
    setup_ms = statistics.median(warm)

    def solve(bv, xv, loop=args.loop):
        return api.fgmres_solve(sysm, hier, bv, xv, rtol=1e-10, maxit=MAXIT, history=False, loop=loop)

    for _ in range(args.warmup):
        x.zero_()
        solve(b, x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    launches0 = api.ib_launch_count()
    times, iters, conv, relres = [], [], [], []
    torch.cuda.nvtx.range_push("timed_solves")  # lets a profiler select the timed region
    for _ in range(args.steps):
        flush.zero_()
        x.zero_()
        s0, s1 = ev(), ev()
        s0.record()
        info = solve(b, x)
        s1.record()
        torch.cuda.synchronize()
        times.append(s0.elapsed_time(s1))
        iters.append(info["iters"])
        conv.append(info["converged"])
        relres.append(info["relres_true"])
    torch.cuda.nvtx.range_pop()
    launches = api.ib_launch_count() - launches0
    clk = clocks.stop()
    # the roofline's unit timed live: CUDA events around each finest-level record inside
    # further solves of the host-driven loop (the same kernels; the device-driven loop's graph
    # holds no event records)
    api.cav_profile(hier, True)
    for _ in range(max(3, args.steps // 4)):
        flush.zero_()
        x.zero_()
        solve(b, x, loop="host")
    n_apply, apply_ms = api.cav_profile_read(hier)
    api.cav_profile(hier, False)
    total_ms = max_over_ranks(sum(times), dist, dev)
    value = whole_job_rate(args.steps, world, total_ms / 1e3)

    # one whole finest-level sweep through cav_sweep (10 sweeps in a CUDA graph)
    li0 = api.cav_get_level_info(hier, 0)
    head_sweep_ms = graph_sweep_ms(api, torch, hier, b)
    head_sweep = additive_sweep_entry(li0, rec.N, args.precision, head_sweep_ms) if args.smoother == "additive" else None

    # the V-cycle alone (graph replay + its two staging copies), to split a solve's time
    zv = torch.empty_like(b)
    for _ in range(3):
        api.vcycle_apply(hier, b, zv)
    v0, v1 = ev(), ev()
    v0.record()
    for _ in range(20):
        api.vcycle_apply(hier, b, zv)
    v1.record()
    torch.cuda.synchronize()
    vcycle_ms = v0.elapsed_time(v1) / 20

    # end to end through the public call with pinned host buffers (H2D of b and x, D2H of x)
    hb = torch.from_numpy(rec.rhs()).pin_memory()
    hx = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        hx.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        solve(hb, hx, loop="host")  # host buffers: the call copies them in and out
        e2e_times.append(time.perf_counter() - t)
    e2e_value = world / statistics.mean(e2e_times) if e2e_times else None

    # plain FP64 inverses on the same system for the mixed-vs-plain comparison
    plain = None
    if args.precision != "fp64" and not args.no_others:
        hier64 = api.cav_setup(sysm, coarsest_N=args.coarsest, nu_pre=args.nu_pre, nu_post=args.nu_post, alpha=args.alpha,
                               precision="fp64",
                               autotune=True, **smoother_kw(args))
        for _ in range(2):
            x.zero_()
            api.fgmres_solve(sysm, hier64, b, x, rtol=1e-10, maxit=MAXIT, history=False, loop=args.loop)
        pt, pit = [], []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            x.zero_()
            s0, s1 = ev(), ev()
            s0.record()
            inf = api.fgmres_solve(sysm, hier64, b, x, rtol=1e-10, maxit=MAXIT, history=False, loop=args.loop)
            s1.record()
            torch.cuda.synchronize()
            pt.append(s0.elapsed_time(s1))
            pit.append(inf["iters"])
        plain = {"value": 1e3 / statistics.mean(pt), "unit": "solves/s", "iters": int(statistics.median(pit))}
        hier64.close()

    # the other smoothers on the same system and precision: with an additive headline, the
    # coloured multiplicative sweep (one per side) on every level and on the finest level only
    # (additive 2+2 below); with a coloured headline, the additive form
    others = []
    if args.precision != "bf16" and not args.no_others:
        if args.smoother == "additive":
            variants = [("coloured", 1, 0), ("coloured", 1, 1)]
        else:
            variants = [("additive", DEFAULT_NU, 0), ("coloured", 1, 0)]
        for o_sm, o_nu, o_cl in variants:
            ho = api.cav_setup(sysm, coarsest_N=args.coarsest, nu_pre=o_nu, nu_post=o_nu, alpha=args.alpha,
                               precision=args.precision,
                               autotune=True, smoother=o_sm, coloured_levels=o_cl, nu_additive=NU_COARSE_ADDITIVE)
            for _ in range(2):
                x.zero_()
                api.fgmres_solve(sysm, ho, b, x, rtol=1e-10, maxit=MAXIT, history=False, loop=args.loop)
            ot, oit = [], []
            for _ in range(max(3, args.steps // 2)):
                flush.zero_()
                x.zero_()
                s0, s1 = ev(), ev()
                s0.record()
                inf = api.fgmres_solve(sysm, ho, b, x, rtol=1e-10, maxit=MAXIT, history=False, loop=args.loop)
                s1.record()
                torch.cuda.synchronize()
                ot.append(s0.elapsed_time(s1))
                oit.append(inf["iters"])
            api.cav_profile(ho, True)
            for _ in range(3):  # the live timing of the finest level's records (host-driven loop)
                flush.zero_()
                x.zero_()
                api.fgmres_solve(sysm, ho, b, x, rtol=1e-10, maxit=MAXIT, history=False, loop="host")
            o_n, o_ms = api.cav_profile_read(ho)
            api.cav_profile(ho, False)
            o_sweep = graph_sweep_ms(api, torch, ho, b)
            ncol = [api.cav_get_level_info(ho, l)["n_colours"] for l in range(api.cav_num_levels(ho) - 1)]
            oli = api.cav_get_level_info(ho, 0)
            o_alg = apply_bytes(oli, args.precision)
            entry = {"smoother": o_sm, "coloured_levels": o_cl if o_sm == "coloured" else None, "nu": o_nu,
                     "nu_additive_levels": NU_COARSE_ADDITIVE if (o_sm == "coloured" and o_cl) else None,
                     "value": 1e3 / statistics.mean(ot), "unit": "solves/s", "iters": int(statistics.median(oit)),
                     "finest_sweep_ms": o_sweep, "colour_classes": ncol,
                     "us_per_class_step_finest": (1e3 * o_sweep / ncol[0]) if ncol and ncol[0] else None}
            if o_sm == "additive":
                # its whole finest-level sweep, and (separate kernels) its patch apply timed live in its solves
                entry["sweep"] = additive_sweep_entry(oli, rec.N, args.precision, o_sweep)
                if o_n and not oli["sweep_form"]:
                    a_us = 1e3 * o_ms / o_n
                    entry["apply_roofline"] = {"kernel": "k_patch_apply_tma (finest level)", "avg_launch_us": a_us,
                                               "algorithmic_bytes_per_launch": o_alg,
                                               "achieved_gbs": o_alg / a_us / 1e3,
                                               "frac_of_measured_hbm": o_alg / a_us / 1e3 / peaks()[0],
                                               "launches_timed": o_n}
            others.append(entry)
            ho.close()

    li = api.cav_get_level_info(hier, 0)
    peak, peak_kind = peaks()
    if args.smoother == "additive" and li["sweep_form"]:
        # the fused sweep kernel is the sweep: its roofline is the sweep's (cav_sweep, graph-timed)
        rl_kernel = "k_sweep_fused (finest level: residual, patch apply, scatter, mean removal)"
        alg_bytes = sweep_bytes(li, rec.N, args.precision)
        launch_us = 1e3 * head_sweep_ms
        n_timed = 10
    else:
        rl_kernel = ("k_patch_apply_tma (finest level)" if args.smoother == "additive" else
                     "k_colour_step (finest level; one record spans the class steps of one sweep)")
        alg_bytes = apply_bytes(li, args.precision)
        launch_us = (1e3 * apply_ms / n_apply) if n_apply else None
        n_timed = n_apply
    achieved = (alg_bytes / (launch_us * 1e-6) / 1e9) if launch_us else None
    src = "colour.cu" if args.smoother == "coloured" else "sweep.cu"
    traffic = NCU_TRAFFIC.get(f"{args.smoother}:{args.precision}:{rec.N}:{src}:{kernel_hash(src)}")
    add_sweep = head_sweep if head_sweep else next((o.get("sweep") for o in others if o["smoother"] == "additive"), None)
    ncol0 = li["n_colours"]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[args.precision],
        "data": "synthetic",
        "config": headline_config(args, rec, world),
        "measures": (f"{args.precision.upper()} enlarged-patch inverses (FP64 everywhere else), "
                     f"{smoother_desc(args)}, zero initial guess: the mixed-precision form without the "
                     f"learned guess (the learned guess is measured by --workload learned_channel); plain "
                     f"FP64 is reported as plain_fp64; FGMRES loop: {args.loop}-driven"
                     + (" (each solve one CUDA graph launch)" if args.loop == "device" else "")),
        "solve": {"precision": args.precision + " enlarged-patch inverses", "iters": int(statistics.median(iters)),
                  "loop": args.loop,
                  "converged": all(conv), "relres_true_max": max(relres)},
        "plain_fp64": plain,
        "other_smoothers": others,
        "setup_ms": setup_ms,
        "setup_ms_first_call": setup_first_ms,
        "vcycle_ms": vcycle_ms,
        "sweep": add_sweep,
        "coloured_sweep": ({"level": 0, "ms": head_sweep_ms, "colour_classes": ncol0,
                            "us_per_class_step": 1e3 * head_sweep_ms / ncol0} if args.smoother == "coloured" else None),
        "setup_plus_solve_per_s": world / ((setup_ms + total_ms / args.steps) / 1e3),
        "apply_variant_finest": li["apply_variant"], "apply_variant_us_finest": li["apply_us"],
        "roofline": {"bound": "hbm", "kernel": rl_kernel, "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes, "launches_timed": n_timed,
                     "avg_launch_us": launch_us},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 2 * n * 8,
                "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and rec.N == 256:
        it = golden_for(args) or int(statistics.median(iters))
        cb = cpu_baseline_sample(it, args)
        if "t_vcycle" in cb:
            t_solve = it * cb["t_vcycle"] + cb["t_rest"]
            line["cpu_baseline"] = {
                "value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": (f"the oracle's solve of the same N=256 system (the same V-cycle: {smoother_desc(args)}; "
                           f"its own count of {it} iterations) = {it} x one timed oracle V-cycle "
                           f"({cb['t_vcycle']:.2f} s) + the oracle's FGMRES run for {it} iterations with the "
                           f"identity in place of the V-cycle ({cb['t_rest']:.2f} s: Arnoldi, Givens, K_E "
                           f"products); oracle hierarchy set-up {cb['t_setup']:.1f} s not timed")}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": "failed: " + cb.get("error", "?")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
