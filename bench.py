"""Benchmark: one-shot Helmholtz solves per second at relative error 1e-8.

A step is one pass of the whole path for one problem: set-up (hierarchy, leaf
factorisation, interface sketches, coarse bases, Galerkin matrices and their inverses)
followed by the outer iteration to the calibrated FP64 residual tolerance, then the
handle is released.  Workload: the precision form, a 1023 x 1023 interior grid
(1025^2 = 1,050,625 unknowns), k = 100, 3-level binary band hierarchy (8 leaves of 130
to 132 rows), overlap 4 rows, r = 32, p = 10, seeded Gaussian point sources.  The
headline runs the mixed form: complex64 subdomain factors, sweeps, sketches and bases;
FP64 residual, Galerkin matrices (FP64 products of the complex64 basis), their
elimination and the sketch eigenproblem.  The FP64 GPU form runs the same workload on
the same line, and the errors of both against the oracle's direct solution are stated.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this project) on the
same workload and `config`, on rank 0 only.  Under torchrun (N > 1) every rank solves its own independent problems
(weak scaling, no collective on the data path); rank 0 prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Helmholtz solves/sec at rel err 1e-8 (mixed vs FP64 GPU); p50/p99 latency"
UNIT = "solves/s"
WORKLOAD = "helm2d_n1023_k100_L3"
# FP64 relative-residual stopping tolerance for relative error <= 1e-8 against the
# direct solution on this workload, with a margin of at least 10x (the error is checked
# to be <= 1e-9 in both forms by tests/test_gpu_bench_calibration.py; measured about
# 0.13 times the residual on this workload).
TOL = 3e-9
# The batching and serving forms mix grid sizes and wavenumbers that this calibration
# does not cover: they stop at the tighter 1e-10.
TOL_FORMS = 1e-10
MAX_ITER = 400
PROFILED_PASS_STEPS = 2      # untimed steps with every kernel category timed
PROFILE_EVERY = 5            # timed steps per step whose dominant-kernel launches carry events
OUTER = "oras"                      # stationary ORAS iteration (GMRES: outer="gmres")
RESTART = 40
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2: written between timed steps
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SM_COUNT, FP32_LANES = 152, 128


# ------------------------------------------------------------------------ helpers
def peaks():
    try:
        with open(MEASURED_PEAKS) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [t.strip() for t in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_inputs():
    from workloads import WORKLOADS, problem_inputs
    w = WORKLOADS[WORKLOAD]
    f, g = problem_inputs(w)
    return w, f, g


def leaf_bands(w):
    """Rows of every leaf band (the same split rule as the library)."""
    e = w.overlap // 2
    S = w.S
    nodes = [(0, S)]
    for _ in range(w.levels):
        nxt = []
        for oa, ob in nodes:
            mid = oa + (ob - oa) // 2
            nxt += [(oa, mid), (mid, ob)]
        nodes = nxt
    return [min(S, ob + e) - max(0, oa - e) for oa, ob in nodes]


# Bound of each profiler category (the library reports each launch's algorithmic bytes
# and flops; see hh_profile_read in include/hh.h).
CATEGORY_BOUND = {
    "factor": ("latency", "k_eig_roots + k_eig_modes (eigenpairs of the column pencil, scalar Schur recursions)"),
    "sweep_in": ("tensor_tf32x3", "k_tc_transform (f^ = V^T f on the tensor cores, TF32 three-term split; "
                                  "k_eig_gemm2 on the CUDA cores where the autotuner chose it)"),
    "sweep_recur": ("hbm", "k_eig_recur (scalar Schur recursions along the line, warp scans)"),
    "sweep_out": ("tensor_tf32x3", "k_tc_transform (x = V x^ on the tensor cores, TF32 three-term split; "
                                   "k_eig_gemm2 on the CUDA cores where the autotuner chose it)"),
    "residual": ("hbm", "k_residual_cast (FP64 residual b - A u, its norm partials and complex64 copy)"),
    "coarse_project": ("hbm", "k_coarse_batch (one-column coarse corrections: C^H r, A_c^-1, C y; "
                              "one cooperative launch per level)"),
    "galerkin": ("alu64", "k_galerkin_herm + k_galerkin_bdry (A_c = C^H A~ C, Hermitian-packed: the upper "
                          "triangle by FP64 3M products of the stored basis, the impedance terms on the boundary "
                          "points)"),
    "qr": ("latency", "k_qr / k_qr_cluster (sketch orthonormalisation, CGS2 in shared memory, one CTA or a cluster)"),
    "svd": ("latency", "k_heig_tri + k_heig_vec (FP64 Hermitian eigenproblem of the sketch Gram matrix)"),
    "leaf_sweep": ("alu", "k_eig_sweep_fused (f^ = V^T f, scalar recursions, x = V x^; one cluster per leaf)"),
    "coarse_multi": ("hbm", "k_ip_colA_rt (multi-column coarse projections of the set-up's sub-level solves)"),
}
# FP64 peak derived from the DFMA issue rate (2 per SM per cycle, the peak ncu reports for
# sm__sass_thread_inst_executed_op_dfma_pred_on.sum): 152 SMs x 2 x 2 flops x max SM clock.
DFMA_PER_SM_CLK = 2
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel on this workload's shapes (mean of its three launches per step), from the ncu
# capture summarised in profiles/coarse_batch_helm2d_n1023_k100_L3.md.  To be removed
# whenever k_coarse_batch changes.
TRAFFIC_BYTES_PER_LAUNCH = {"coarse_project": 491.7e6}


def whole_job_rate(local_ms, units_per_rank, world, device="cuda"):
    """Whole-job throughput over `world` ranks that each processed `units_per_rank`
    units in `local_ms`: the units of all ranks over the slowest rank's time (a MAX
    all-reduce of the times when world > 1).  Returns (units/s, max ms)."""
    ms = float(local_ms)
    if world > 1:
        import torch
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


# --------------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_12538_gb300 as hh

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    w, f, g = workload_inputs()
    fd = torch.from_numpy(f).cuda()
    gd = torch.from_numpy(g).cuda()
    u = torch.empty_like(fd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def params(prec):
        return hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, w.n_inner, TOL, MAX_ITER,
                              prec, 1 + rank, outer=OUTER, restart=RESTART)

    def one(prec, profile=False):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h, _ = hh.hh_setup(params(prec), stream)
        st = hh.hh_solve(h, fd, gd, u, stream)
        e1.record(stream)
        prof = hh.hh_profile_read(h, work=True) if profile else None
        hh.hh_destroy(h)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st, prof

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        one("mixed")
    if args.fp64_form == "on":
        one("fp64")

    # untimed profiled pass: every kernel category timed with CUDA events on `stream`
    # (the per-category table, and which category dominates)
    prof_all = {}
    hh.hh_profile_enable(None, True)
    for _ in range(PROFILED_PASS_STEPS):
        _, _, prof = one("mixed", profile=True)
        for k, vals in prof.items():
            old = prof_all.get(k, (0.0, 0, 0.0, 0.0))
            prof_all[k] = tuple(x + y for x, y in zip(old, vals))
    dominant = max(prof_all, key=lambda k: prof_all[k][0])

    # timed: mixed form, headline.  The library's event profiler times the dominant
    # category alone here (CUDA events on `stream` around its launches), which gives its
    # average launch duration over the timed region.  Events cost stream time (two per
    # outer step), so they are recorded in one of every PROFILE_EVERY timed steps.
    hh.hh_profile_categories(None, [dominant])
    barrier()
    launches0 = hh.hh_launch_count()
    step_ms, iters, prof_total = [], [], {}
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            sampled = i % PROFILE_EVERY == 0
            hh.hh_profile_enable(None, sampled)
            ms, st, prof = one("mixed", profile=sampled)
            step_ms.append(ms)
            iters.append(st.iters)
            for k, vals in (prof or {}).items():
                old = prof_total.get(k, (0.0, 0, 0.0, 0.0))
                prof_total[k] = tuple(x + y for x, y in zip(old, vals))
        barrier()
        wall = time.perf_counter() - t0
    hh.hh_profile_enable(None, False)
    hh.hh_profile_categories(None, None)
    launches = hh.hh_launch_count() - launches0
    value, total_ms = whole_job_rate(sum(step_ms), args.steps, world)
    u_mixed = u.cpu().numpy()
    setup_split = one("mixed")[1]

    # FP64 GPU form of the same method on the same workload
    fp64_ms = []
    fp64_iters = []
    for _ in range(max(3, args.steps // 2) if args.fp64_form == "on" else 0):
        ms, st, _ = one("fp64")
        fp64_ms.append(ms)
        fp64_iters.append(st.iters)
    fp64_value = whole_job_rate(sum(fp64_ms), len(fp64_ms), world)[0] if fp64_ms else None
    u_fp64 = u.cpu().numpy() if fp64_ms else None

    # end to end through the C-ABI with host buffers (pinned): H2D f, g and D2H u inside
    fh = torch.from_numpy(f).pin_memory()
    gh = torch.from_numpy(g).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h, _ = hh.hh_setup(params("mixed"), stream)
        hh.hh_solve_host(h, fh, gh, uh, stream)
        hh.hh_destroy(h)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    N = w.S * w.S
    e2e = {"value": whole_job_rate(sum(e2e_ms), len(e2e_ms), world)[0], "unit": UNIT,
           "h2d_bytes_per_step": 16 * (N + 4 * w.S), "d2h_bytes_per_step": 16 * N,
           "ms_per_step": statistics.mean(e2e_ms), "timing": "host wall clock around set-up, "
           "hh_solve_host (pinned buffers) and release, no profiler events"}

    batch, batch_u = run_batch_form(hh, torch) if rank == 0 and args.batch_form == "on" else (None, None)
    serving = run_serving(args, hh, torch) if rank == 0 and args.serving_form == "on" else None

    pk, pk_kind = peaks()
    roof = roofline(w, prof_total, prof_all, dominant, pk, pk_kind)
    if roof is not None:
        roof["event_steps"] = f"{len(range(0, args.steps, PROFILE_EVERY))} of {args.steps} timed steps"
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64/f64", "data": "synthetic",
        "config": workload_config(w, "mixed", "inputs larger than L2 (16.8 MB vectors, 2.3 GB factors and bases); "
                                             "L2 also flushed between steps (256 MB write)", f"replicas x{world}"),
        "latency_ms": {"p50": pct(step_ms, 50), "p99": pct(step_ms, 99)},
        "iterations": {"mixed": statistics.median(iters),
                       "fp64": statistics.median(fp64_iters) if fp64_iters else None},
        "setup_ms": {"mixed": setup_split.t_setup_ms, "solve_mixed": setup_split.t_solve_ms},
        "fp64_form": {"value": fp64_value, "unit": UNIT, "dtype": "c128/f64",
                      "ms_per_step": statistics.mean(fp64_ms) if fp64_ms else None,
                      "median_ms_per_step": statistics.median(fp64_ms) if fp64_ms else None,
                      "iterations": statistics.median(fp64_iters) if fp64_iters else None,
                      "step_ms": [round(x, 3) for x in fp64_ms]},
        "mixed_over_fp64": value / fp64_value if fp64_value else None,
        "e2e": e2e, "roofline": roof, "gpu_launches": int(launches), "clocks": clocks,
        "kernels": {k: dict(rate(k, v[0], v[2], v[3], pk, pk_kind), ms_total=v[0], launches=v[1])
                    for k, v in prof_all.items() if v[1] > 0},
        "kernels_from": f"untimed profiled pass of {PROFILED_PASS_STEPS} steps, every category timed",
        "autotune": hh.hh_autotune_report(),
        "wall_s_timed": wall,
    }
    if batch is not None:
        out["batch_form"] = batch
    if serving is not None:
        out["serving_form"] = serving
    if rank == 0 and world == 1 and args.cpu_baseline == "on":
        base, refs = cpu_baseline_leg(w, batch_u)
        out["cpu_baseline"] = base
        # relative errors against the oracle's direct solution u* = A^{-1} b
        out["rel_err"] = {"mixed": rel_err(u_mixed, refs["u_star"]),
                          "fp64": rel_err(u_fp64, refs["u_star"]) if u_fp64 is not None else None,
                          "against": "oracle direct solve (sparse LU) of the same system"}
        if batch is not None and refs.get("batch"):
            errs = [rel_err(batch_u[i], us) for i, us in refs["batch"].items()]
            batch["rel_err_sample"] = {"problems": sorted(refs["batch"]), "max": max(errs),
                                       "against": "oracle direct solves of a seeded subset incl. the largest k h"}
    return out


def rel_err(u, u_star):
    import numpy as np
    u = np.asarray(u).reshape(-1)
    u_star = np.asarray(u_star).reshape(-1)
    return float(np.linalg.norm(u - u_star) / np.linalg.norm(u_star))


BATCH_PROBLEMS = 512
BATCH_ERR_SAMPLE = 8      # problems of the batch compared with the oracle's direct solution


def batch_error_sample(probs):
    """Indices of the batch problems whose errors the line states: the problems with the
    largest k h and a seeded draw of the rest."""
    import numpy as np
    kh = [w.k / (w.n + 1) for (w, f, g) in probs]
    order = sorted(range(len(probs)), key=lambda i: -kh[i])
    pick = order[:BATCH_ERR_SAMPLE // 2]
    rng = np.random.Generator(np.random.PCG64(2512_12538 + 4))
    rest = [i for i in range(len(probs)) if i not in pick]
    pick += [int(i) for i in rng.choice(rest, size=min(len(rest), BATCH_ERR_SAMPLE - len(pick)), replace=False)]
    return sorted(pick)


def run_batch_form(hh, torch, count=BATCH_PROBLEMS):
    """The batching form: `count` independent problems (grid sides 63..255, k h in
    [0.3, 0.6], 2 levels, r = 16, p = 8) set up together (hh_setup_batch) and solved
    together (hh_solve_batch), one warm-up and one timed pass; solves/s over set-up and
    solve.  Returns (result, the solutions of the error sample on the host)."""
    from workloads import batch_problems
    probs = batch_problems(count)
    params = [hh.make_params(2, w.n, w.k, w.levels, w.overlap, w.rank, w.oversample, 1, TOL_FORMS, MAX_ITER, "mixed",
                             1 + i) for i, (w, f, g) in enumerate(probs)]
    fs = [torch.from_numpy(f).cuda() for (w, f, g) in probs]
    gs = [torch.from_numpy(g).cuda() for (w, f, g) in probs]
    us = [torch.empty((w.S, w.S), dtype=torch.complex128, device="cuda") for (w, f, g) in probs]
    res = None
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = hh.hh_setup_batch(params)
        t1 = time.perf_counter()
        sts = hh.hh_solve_batch(hs, fs, gs, us)
        t2 = time.perf_counter()
        for h in hs:
            hh.hh_destroy(h)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        its = [st.iters for st in sts]
        res = {"problems": count, "value": count / (t3 - t0), "unit": UNIT, "setup_ms": 1e3 * (t1 - t0),
               "solve_ms": 1e3 * (t2 - t1), "iterations": {"median": statistics.median(its), "max": max(its)},
               "max_rel_res": max(st.rel_res for st in sts),
               "workload": "batch: grid sides U{63,127,191,255}, k h U[0.3,0.6], L=2, overlap 2, r=16, p=8, "
                           f"mixed form, tol {TOL_FORMS}", "timing": "host wall clock, warm second pass"}
    sample = {i: us[i].cpu().numpy() for i in batch_error_sample(probs)}
    return res, sample


SERVE_SECONDS = 0.5       # length of the serving stream in the default line


def serving_requests(hh, torch, rate, seconds):
    """The serving form's request stream: Poisson arrivals (mean `rate` per second for
    `seconds` seconds), grid sides U{127,255,511,1023}, k ~ U[20, min(150, 0.6/h)], 2 levels
    (r=16, p=10, overlap 2) up to 255 and 3 levels (r=32, p=10, overlap 4) above."""
    import numpy as np
    from workloads import point_source_rhs
    rng = np.random.Generator(np.random.PCG64(2512_12538 + 5))
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        n = int(rng.choice([127, 255, 511, 1023]))
        k = float(rng.uniform(20.0, min(150.0, 0.6 * (n + 1))))
        lv, ov, r = (2, 2, 16) if n <= 255 else (3, 4, 32)
        p = hh.make_params(2, n, k, lv, ov, r, 10, 1, TOL_FORMS, MAX_ITER, "mixed", len(reqs) + 1)
        f = torch.from_numpy(point_source_rhs(n, 2512_12538 + 31 * len(reqs))).cuda()
        g = torch.zeros((4, n + 2), dtype=torch.complex128, device="cuda")
        u = torch.empty_like(f)
        reqs.append((t, n, p, f, g, u))
    return reqs


def run_serving(args, hh, torch, seconds=None):
    """The serving form: the request stream submitted to one hh_server as the requests
    arrive; served solves/s and p50/p99 latency (submission to completion)."""
    seconds = args.serve_seconds if seconds is None else seconds
    reqs = serving_requests(hh, torch, args.rate, seconds)
    torch.cuda.synchronize()
    srv = hh.hh_server_create(160 << 30, 64)
    lat, done, fails, codes = [], {}, 0, {}
    t0 = time.perf_counter()
    tickets = []
    i = 0
    while len(done) < len(reqs):
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            _, n, p, f, g, u = reqs[i]
            tickets.append(hh.hh_server_submit(srv, p, f, g, u))
            i += 1
        for j, tk in enumerate(tickets):
            if j in done:
                continue
            res = hh.hh_server_poll(srv, tk)
            if res is not None:
                st, stats = res
                done[j] = time.perf_counter() - t0
                lat.append(stats.t_total_ms)
                fails += st != hh.HH_OK
                codes[hh.status_string(st)] = codes.get(hh.status_string(st), 0) + 1
        time.sleep(0.0002)
    wall = max(done.values())
    hh.hh_server_destroy(srv)
    return {"metric": "served Helmholtz solves/sec (Poisson stream) at rel err 1e-8; p50/p99 latency",
            "value": len(reqs) / wall, "unit": UNIT, "higher_is_better": True,
            "requests": len(reqs), "failed": fails, "statuses": codes, "offered_rate": args.rate,
            "stream_s": seconds, "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)}, "wall_s": wall,
            "config": {"workload": "serving: sides U{127,255,511,1023}, k U[20, min(150, 0.6/h)], L=2 (r=16,p=10) "
                                   "up to 255, L=3 (r=32,p=10) above; budget 160 GB, 64 slots", "precision": "mixed",
                       "tol_rel_residual": TOL_FORMS},
            "data": "synthetic"}


def run_serving_line(args):
    """--form serve: a longer serving stream on its own line."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_12538_gb300 as hh
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = run_serving(args, hh, torch)
    out["n_gpus"] = 1
    return out


def run_case(args):
    """--form case: one set-up and a few stationary steps of the workload's grid and
    hierarchy at rank --case-rank (oversampling 4), with no timing: the small case the
    profiler captures of single kernels run on (profiles/).  --case-n takes a smaller grid
    (n interior points a side, k scaled to keep the workload's k h) with the same hierarchy."""
    import dataclasses

    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_12538_gb300 as hh
    from workloads import problem_inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w, f, g = workload_inputs()
    if args.case_n and args.case_n != w.n:
        w = dataclasses.replace(w, n=args.case_n, k=w.k * (args.case_n + 1) / (w.n + 1))
        f, g = problem_inputs(w)
    fd = torch.from_numpy(f).cuda()
    gd = torch.from_numpy(g).cuda()
    u = torch.empty_like(fd)
    # the sweep transforms on the tensor cores without timing alternatives: under a
    # profiler every launch is serialised, so the autotuner's timings would mean nothing
    p = hh.make_params(2, w.n, w.k, w.levels, w.overlap, args.case_rank, 4, 1, 1e-3, args.case_steps, "mixed", 1,
                       "eigen", "oras", RESTART, flags=hh.HH_FLAG_TENSOR_CORE_SWEEPS)
    h, fp = hh.hh_setup(p)
    st = hh.hh_solve(h, fd, gd, u, allow_noconv=True)
    torch.cuda.synchronize()
    hh.hh_destroy(h)
    return {"case": WORKLOAD, "n": w.n, "k": w.k, "rank": args.case_rank, "footprint_bytes": fp,
            "iters": st.iters, "rel_res": st.rel_res}


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    lo, hi = int(k), min(int(k) + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def rate(cat, ms, by, fl, pk, pk_kind):
    """Achieved rate of one category against its peak."""
    bound, kname = CATEGORY_BOUND.get(cat, ("latency", cat))
    out = {"kernel": kname, "category": cat, "bound": bound}
    if bound == "hbm" and by > 0:
        a = by / (ms / 1e3) / 1e9
        out.update({"achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": a / pk["hbm_gbs"],
                    "peak_kind": f"{pk_kind} hbm_gbs"})
    elif bound == "alu" and fl > 0:
        peak = SM_COUNT * FP32_LANES * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        a = fl / (ms / 1e3) / 1e12
        out.update({"achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                    "peak_kind": "FP32 FFMA derived: 152 SMs x 128 lanes x 2 flops x max SM clock"})
    elif bound == "tensor_tf32x3" and fl > 0:
        # the transforms run as TF32 MMAs three times over (hi.hi + hi.lo + lo.hi): executed
        # tensor flops = 3 x the algorithmic complex-GEMM flops, against the dense TF32 peak
        # (the measured bf16 GEMM rate x the nominal TF32 / BF16 ratio, 1.1 / 2.25)
        peak = pk["bf16_tflops"] * (1.1 / 2.25)
        a = 3.0 * fl / (ms / 1e3) / 1e12
        out.update({"achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                    "peak_kind": f"{pk_kind} bf16_tflops x 1.1/2.25 (TF32 dense); achieved counts the three "
                                 "TF32 passes"})
    elif bound == "alu64" and fl > 0:
        peak = SM_COUNT * DFMA_PER_SM_CLK * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        a = fl / (ms / 1e3) / 1e12
        out.update({"achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                    "peak_kind": "FP64 DFMA derived: 152 SMs x 2 DFMA/clk x 2 flops x max SM clock"})
    else:
        out.update({"achieved": None, "peak": None, "unit": None, "frac": None})
    return out


def roofline(w, prof, prof_all, cat, pk, pk_kind):
    """The dominant kernel category (largest total device time in the untimed profiled
    pass) with its algorithmic rate against its peak; the rate from its CUDA-event times
    over the timed solves (`prof`, that category alone timed)."""
    if not prof or cat not in prof or prof[cat][1] == 0:
        return None
    ms, launches, by, fl = prof[cat]
    out = rate(cat, ms, by, fl, pk, pk_kind)
    out.update({"launches": launches, "avg_launch_ms": ms / max(launches, 1),
                "share_of_profiled_ms": prof_all[cat][0] / sum(v[0] for v in prof_all.values()),
                "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(cat), "alg_bytes_per_launch": by / max(launches, 1),
                "alg_flops_per_launch": fl / max(launches, 1)})
    return out


def workload_config(w, precision, l2, parallelism):
    """The JSON line's `config`: the workload and the step, shared by both arms."""
    return {"workload": WORKLOAD, "grid": f"{w.S}x{w.S} nodes ({w.n}^2 interior)", "k": w.k,
            "levels": w.levels, "leaves": 2 ** w.levels, "overlap": w.overlap, "rank": w.rank,
            "oversample": w.oversample, "n_inner": w.n_inner, "tol_rel_residual": TOL,
            "precision": precision, "step": "setup+solve+release of one problem per rank", "l2": l2,
            "parallelism": parallelism}


# ------------------------------------------------------------------ CPU baseline
# The oracle (oracle/, FP64 CPU) runs only here: the CPU baseline leg of the GPU arm and
# the reference arm.  Its direct solve u* = A^{-1} b (sparse LU) is the oracle's fastest
# way to a solution of the workload at the metric's accuracy (exact), so it is the timed
# sample; its solutions also state the GPU results' errors.  Workers are spawned (fresh
# interpreters, no CUDA state), single-threaded each.
def _oracle_worker_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _oracle_direct(job):
    """(seconds, u*) of one direct solve; job = (workload name or batch index, keep u*)."""
    from oracle import direct
    from oracle.problem import Problem
    from workloads import WORKLOADS, batch_problems, problem_inputs
    what, keep = job
    if isinstance(what, str):
        w = WORKLOADS[what]
        f, g = problem_inputs(w)
    else:
        w, f, g = batch_problems(what + 1)[what]
    t0 = time.perf_counter()
    u = direct.solve(Problem(2, w.n, w.k), f, g)
    return time.perf_counter() - t0, (u if keep else None)


def _oracle_pool(workers):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers, initializer=_oracle_worker_init)


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


ORACLE_POOL_MAX = 16


def cpu_baseline_leg(w, batch_u=None):
    """The oracle on the host cores: one direct solve single-threaded (its u* also gives
    the GPU results' errors), then one solve per core on all cores at once (throughput).
    With `batch_u`, the direct solutions of those batch problems as well.  Returns
    (cpu_baseline object, {"u_star": u*, "batch": {index: u*}})."""
    cores, model = host_cpu()
    nw = max(1, min(cores, ORACLE_POOL_MAX))
    with _oracle_pool(nw) as pool:
        t1, u_star = pool.apply(_oracle_direct, ((WORKLOAD, True),))
        t0 = time.perf_counter()
        pool.map(_oracle_direct, [(WORKLOAD, False)] * nw, chunksize=1)
        t_all = time.perf_counter() - t0
        batch = {}
        if batch_u:
            idx = sorted(batch_u)
            for i, (_, ub) in zip(idx, pool.map(_oracle_direct, [(i, True) for i in idx], chunksize=1)):
                batch[i] = ub
    base = {"value": nw / t_all, "unit": UNIT, "cores": nw, "kind": "oracle",
            "sample": f"{nw} direct solves (oracle sparse LU, minimum-degree ordering; exact, so within the metric's "
                      f"1e-8) of {WORKLOAD}, one per core at once, single-threaded each",
            "single_thread": {"value": 1.0 / t1, "unit": UNIT, "cores": 1, "seconds_per_solve": t1},
            "cpu_model": model, "host_logical_cores": cores,
            "note": "the oracle's stepwise method (O-method) on this workload is slower than its direct solve"}
    return base, {"u_star": u_star, "batch": batch}


def run_reference(args, rank, world):
    """The reference arm: the oracle (FP64 CPU) on this workload, timed on the host cores.
    A step is one direct solve of the workload; the steps run one per core at once
    (single-threaded each), warm-up steps first."""
    if rank != 0:
        return None
    w, f, g = workload_inputs()
    cores, model = host_cpu()
    nw = max(1, min(cores, ORACLE_POOL_MAX, max(args.steps, args.warmup, 1)))
    with _oracle_pool(nw) as pool:
        if args.warmup > 0:
            pool.map(_oracle_direct, [(WORKLOAD, False)] * args.warmup, chunksize=1)
        t0 = time.perf_counter()
        times = pool.map(_oracle_direct, [(WORKLOAD, False)] * args.steps, chunksize=1)
        dt = time.perf_counter() - t0
    value = args.steps / dt
    per = [t for t, _ in times]
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(w, "fp64 (CPU oracle)", "host run", "rank 0 only"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(nw, args.steps), "kind": "oracle",
                             "sample": f"{args.steps} direct solves (oracle sparse LU, minimum-degree ordering) of "
                                       f"{WORKLOAD}, up to {nw} at once, single-threaded each",
                             "seconds_per_solve": statistics.mean(per), "cpu_model": model,
                             "host_logical_cores": cores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="single", choices=["single", "serve", "case"],
                    help="serve: the serving-form stream instead of the headline workload; case: the small "
                         "case profiler captures run on (--case-rank, --case-steps)")
    ap.add_argument("--case-rank", type=int, default=16)
    ap.add_argument("--case-steps", type=int, default=12)
    ap.add_argument("--case-n", type=int, default=0, help="case: interior points a side (0: the workload's)")
    ap.add_argument("--batch-form", default="on", choices=["on", "off"],
                    help="also measure the batching form (512 problems) after the headline")
    ap.add_argument("--serving-form", default="on", choices=["on", "off"],
                    help="also run a short serving stream after the headline")
    ap.add_argument("--fp64-form", default="on", choices=["on", "off"],
                    help="also time the FP64 GPU form of the same workload")
    ap.add_argument("--cpu-baseline", default="on", choices=["on", "off"],
                    help="time the oracle on the host cores and state the errors against its solution")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=SERVE_SECONDS,
                    help="serving: length of the arrival stream")
    args = ap.parse_args()
    if args.form == "serve":
        print(json.dumps(run_serving_line(args)), flush=True)
        return
    if args.form == "case":
        print(json.dumps(run_case(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
