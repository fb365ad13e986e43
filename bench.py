"""Benchmark: multi-shift CG solves/s on a 32^4 lattice (15 shifts, m = 0.01,
tol 1e-10, FP64), plus the FP64 D_eo ns/site and HBM GB/s sweep and the
mixed-precision speed-up, through the C ABI of liblqcd.

One "step" = one complete multi-shift solve (every kernel of the path:
D_oe, D_eo with the normal-operator epilogue, the deterministic FP64
reductions, the shifted updates, the FP64 true-residual check).  Inputs are
resident in HBM when the timed region starts and are larger than L2 (links
604 MB, Krylov vectors 0.8 GB), so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the plain C FP64 oracle (the reference arm of this
build) on bounded samples of the same workload on the host cores.
Multi-GPU: replicas only (every rank solves its own source; no collective
on the data path); value = solves of all ranks / max-over-ranks time.
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

METRIC = "D_eo ns/site & HBM GB/s; mshift-CG solves/s at 1e-10 (mixed/batched vs FP64)"
DIMS = (32, 32, 32, 32)
MASS = 0.01
N_SHIFT = 15
TOL = 1e-10
WORKLOAD = "mscg 32^4, m=0.01, 15 shifts log-spaced 1e-5..1e2, tol 1e-10, FP64 (hot random SU(3) links)"
COUNTS_KEY = "mscg_32x32x32x32_m0.01_15shifts_tol1e-10"


# DRAM traffic of the dominant kernel (k_it_deo2_st, the staged FP64 D_eo with
# the normal-operator epilogue) from one ncu capture of the staged iteration
# kernels on a 24^4 lattice:
# dram__bytes_read.sum + dram__bytes_write.sum of one launch / (V/2).  It scales
# with the even sites (links stream from HBM at both sizes, spinors hit L2), so
# a launch at V/2 sites moves bytes_per_site * V/2.  Reported only while the
# kernel sources still hash to the captured version.
K2_TRAFFIC = {"bytes_per_site": 1257.7, "src_sha256_16": "1c46e0f51e652eed",
              "sources": ["solver_kernels.cuh", "stencil_staged.cuh", "bulk.cuh", "deo_core.cuh", "common.cuh", "iteration.h"]}


def k2_traffic_per_site():
    import hashlib
    h = hashlib.sha256()
    for f in K2_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_1701_00426_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return K2_TRAFFIC["bytes_per_site"] if h.hexdigest()[:16] == K2_TRAFFIC["src_sha256_16"] else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    return 6800.0, "fallback 6.8 TB/s"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- distributed
def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps: int, t_ms_local: float, world: int):
    """Replicas: every rank ran `steps` solves; the job's time is the slowest
    rank's.  Returns (solves/s of the whole job, max-over-ranks ms)."""
    t_max = max_over_ranks(t_ms_local, world)
    return world * steps / (t_max * 1e-3), t_max


# ---------------------------------------------------------------- oracle (CPU)
def oracle_counts():
    """The oracle's own iteration counts for this workload (written by
    tests/golden/make_oracle_counts.py from a full oracle solve)."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_counts.json")
    if os.path.exists(p):
        d = json.load(open(p)).get(COUNTS_KEY)
        if d:
            return d
    return None


def oracle_sample(U, b, shifts, k_lo=2, k_hi=12, dims=None, reps=3):
    """Bounded sample of the oracle on the same workload.  Its multi-shift CG
    runs stopped after k_lo and k_hi iterations, once with every shift and
    once with the first shift alone; the differences give the cost of one
    iteration with n and with 1 active shift, hence the per-iteration base
    cost (A application, base residual and direction) and the cost per active
    shift.  fixed = the k_lo run with every shift minus its k_lo iterations
    (set-up and the final true residuals).  Medians over reps repeats.
    Returns (base s/iteration, s per active shift per iteration, fixed s,
    threads, seconds spent)."""
    from oracle import oracle
    dims = DIMS if dims is None else dims
    orc = oracle()
    threads = orc.set_threads(0)
    n = len(shifts)
    t_start = time.time()
    cn, c1, fx = [], [], []
    for _ in range(reps):
        t0 = time.time()
        orc.mscg(dims, U, MASS, shifts, b, TOL, max_iter=k_lo)
        t1 = time.time()
        orc.mscg(dims, U, MASS, shifts, b, TOL, max_iter=k_hi)
        t2 = time.time()
        orc.mscg(dims, U, MASS, shifts[:1], b, TOL, max_iter=k_lo)
        t3 = time.time()
        orc.mscg(dims, U, MASS, shifts[:1], b, TOL, max_iter=k_hi)
        t4 = time.time()
        it_n = ((t2 - t1) - (t1 - t0)) / (k_hi - k_lo)
        cn.append(it_n)
        c1.append(((t4 - t3) - (t3 - t2)) / (k_hi - k_lo))
        fx.append(max((t1 - t0) - k_lo * it_n, 0.0))
    it_n, it_1, fixed = float(np.median(cn)), float(np.median(c1)), float(np.median(fx))
    per_shift = max(it_n - it_1, 0.0) / (n - 1) if n > 1 else 0.0
    base = max(it_1 - per_shift, 0.0)
    return base, per_shift, fixed, threads, time.time() - t_start


def oracle_deo_sample(inputs, sizes=(16, 32)):
    """The oracle's D_eo (one application, odd -> even) in ns per even site,
    single-threaded and on all host cores, on the sweep's lattices."""
    from oracle import oracle
    orc = oracle()
    out = {}
    for L in sizes:
        dims = (L,) * 4
        U = inputs.random_links(dims)
        x = inputs.gaussian_field(dims)
        Vh = L ** 4 // 2
        res = {}
        for n in (1, 0):
            got = orc.set_threads(n)
            orc.deo(dims, 0, U, x)
            t0 = time.perf_counter()
            reps = 0
            while reps < 3 or time.perf_counter() - t0 < 1.0:
                orc.deo(dims, 0, U, x)
                reps += 1
            res[f"{got}_threads"] = round((time.perf_counter() - t0) / reps * 1e9 / Vh, 2)
        out[f"{L}^4"] = res
        del U
    orc.set_threads(0)
    return out


def cpu_solve_seconds(base, per_shift, fixed, counts):
    """Whole-solve time of the oracle from the sample: every iteration costs
    the base part, plus the per-shift part for each shift still active; the
    iteration counts (and each shift's last iteration) are the oracle's own."""
    return fixed + counts["iters"] * base + sum(counts["shift_iters"]) * per_shift


def validate_cpu_model(L=16):
    """Checks the whole-solve model of the CPU baseline against a measured
    solve: on an L^4 lattice (same mass, shifts and tolerance; 16^4 takes
    ~10 s on the host cores) the oracle runs one full multi-shift solve, and
    the model prices the same solve from a bounded sample (the stopped runs
    and one A application, as on the timed workload) and the solve's own
    iteration counts.  Returns both times and their ratio."""
    from oracle import oracle
    from paper_1701_00426_gb300 import inputs
    dims = (L,) * 4
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=0)
    shifts = inputs.log_shifts(N_SHIFT)
    orc = oracle()
    base, per_shift, fixed, thr, _ = oracle_sample(U, b, shifts, dims=dims)
    t0 = time.time()
    _, info = orc.mscg(dims, U, MASS, shifts, b, TOL)
    measured = time.time() - t0
    counts = {"iters": info["iters"] + info["refine_iters"], "shift_iters": list(info["shift_iters"])}
    modelled = cpu_solve_seconds(base, per_shift, fixed, counts)
    return {"lattice": f"{L}^4", "measured_s": round(measured, 3), "modelled_s": round(modelled, 3),
            "measured_over_modelled": round(measured / modelled, 3), "iters": info["iters"],
            "refine_iters": info["refine_iters"], "threads": thr}


def run_reference(args, rank, world):
    """Reference arm: the plain C oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_1701_00426_gb300 import inputs
    U = inputs.random_links(DIMS)
    b = inputs.gaussian_field(DIMS, k=0)
    shifts = inputs.log_shifts(N_SHIFT)
    counts = oracle_counts()
    src = "the oracle's own full-solve counts (tests/golden/oracle_counts.json)"
    if counts is None:
        counts = {"iters": 3000, "shift_iters": [3000] * N_SHIFT}
        src = "assumed 3000 iterations with every shift active (count file missing)"
    validation = validate_cpu_model()
    for _ in range(args.warmup):
        oracle_sample(U, b, shifts, 1, 2, reps=1)
    vals, wall, thr = [], time.time(), 1
    for _ in range(args.steps):
        base, per_shift, fixed, thr, _ = oracle_sample(U, b, shifts, reps=1)
        vals.append(1.0 / cpu_solve_seconds(base, per_shift, fixed, counts))
    wall = time.time() - wall
    v = float(np.median(vals))
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": thr, "kind": "oracle",
                             "sample": "each step: oracle multi-shift CG stopped after 2 and 12 iterations, with "
                                       "all 15 shifts and with one; whole solve = set-up + iterations x base "
                                       f"cost + shift-iterations x per-shift cost, with {src}"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "modelled": True, "model_validation": validation,
            "recorded_full_solve": {k: counts.get(k) for k in ("seconds", "threads")} if "seconds" in counts else None,
            "sample_wall_s": round(wall, 1),
            "note": "value and ms_per_step are the modelled whole-solve time, not time spent in this run; "
                    "sample_wall_s is the real wall time of the timed samples"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- extra configs
def batched_bench(lqcd, inputs, torch, hbm_peak):
    """24^4: multi-RHS D_eo (ns per field-site, link loads shared by 1/4/8/16
    fields) and the batched CG (m = 0.1, one shift, FP32 iterations with FP64
    reliable updates) against n single-field solves."""
    dims = (24, 24, 24, 24)
    U = inputs.random_links(dims)
    out = {"lattice": list(dims), "deo_fp32_12r": {}, "cg": {}}
    with lqcd.Context(dims, prec=lqcd.PREC_FP32, recon=12) as c:
        c.links_upload(U)
        del U
        s = torch.cuda.current_stream()
        flush = L2Flush(torch)
        for n in (1, 4, 8, 16):
            x = torch.randn((3, c.Vh, n), dtype=torch.complex64, device="cuda")
            o = torch.empty_like(x)
            for _ in range(3):
                c.deo_apply_mrhs(0, n, 12, x, o, s)
            ts = []
            for _ in range(10):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                c.deo_apply_mrhs(0, n, 12, x, o, s)
                e1.record(s)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            med = float(np.median(ts))
            bps = 384.0 + 48.0 * n
            out["deo_fp32_12r"][str(n)] = {"ns_per_field_site": round(med * 1e6 / (c.Vh * n), 4),
                                           "GB_s": round(bps * c.Vh / (med * 1e-3) / 1e9, 1)}
        b = np.stack([inputs.gaussian_field(dims, k=j) for j in range(16)])
        t0 = time.perf_counter()
        for j in range(4):
            c.cg_solve_mrhs(0.1, 0.0, 1e-10, b[j:j + 1])
        t1 = time.perf_counter()
        x16, inf16 = c.cg_solve_mrhs(0.1, 0.0, 1e-10, b)
        t2 = time.perf_counter()
        single = 4 / (t1 - t0)
        out["cg"] = {"single_solves_per_s": round(single, 2), "batched16_solves_per_s": round(16 / (t2 - t1), 2),
                     "speedup": round((16 / (t2 - t1)) / single, 2),
                     "max_true_resid": max(i["true_resid"][0] for i in inf16),
                     "iters": max(i["iters"] for i in inf16)}
    return out


def packed_bench(lqcd, inputs):
    """8^4, 12^4, 16^4, 20^4 solved together in shared launches vs one after
    another (15 shifts, m = 0.01, tol 1e-10, FP64); results compared bitwise."""
    sizes = [(8,) * 4, (12,) * 4, (16,) * 4, (20,) * 4]
    shifts = inputs.log_shifts(15)
    ctxs, bs = [], []
    for k, d in enumerate(sizes):
        c = lqcd.Context(d)
        c.links_upload(inputs.random_links(d))
        ctxs.append(c)
        bs.append(inputs.gaussian_field(d, k=k))
    for c, b in zip(ctxs, bs):  # warm
        c.mscg_solve(MASS, shifts, TOL, b)
    t0 = time.perf_counter()
    solo = [c.mscg_solve(MASS, shifts, TOL, b)[0] for c, b in zip(ctxs, bs)]
    t1 = time.perf_counter()
    xs, infos = lqcd.mscg_solve_packed(ctxs, [MASS] * 4, [shifts] * 4, [TOL] * 4, bs)
    t2 = time.perf_counter()
    same = all(np.array_equal(a, b) for a, b in zip(xs, solo))
    for c in ctxs:
        c.close()
    return {"lattices": ["8^4", "12^4", "16^4", "20^4"], "separate_s": round(t1 - t0, 4),
            "packed_s": round(t2 - t1, 4), "speedup": round((t1 - t0) / (t2 - t1), 3),
            "bitwise_equal_to_separate": same, "max_true_resid": max(max(i["true_resid"]) for i in infos)}


def serving_bench(lqcd, inputs, n_req=40, loads=(0.5, 0.8, 0.95), budget=16 << 30, mixed=False, sequential=True,
                  sides=(8, 16, 24, 32)):
    """Poisson stream of multi-shift requests over resident 8^4/16^4/24^4/32^4
    fields (1..16 shifts log-spaced in [1e-5, 1e2], tol 1e-8 or 1e-10,
    m = 0.01) under an HBM budget.  A burst run (all requests at t = 0)
    measures capacity; Poisson runs at the given fractions of it measure
    latency.  Peak admitted bytes and slots are sampled during each run.
    mixed: requests run in mixed precision (FP32 12-real links, FP64 phase
    to 3e-4, FP64 reliable updates).  sequential: also time the same requests
    solved one after another by the plain FP64 solver (device-resident
    sources, no host copies)."""
    sizes = [(L,) * 4 for L in sides]
    rng = np.random.default_rng(inputs.ARRIVAL_SEED)
    reqs = []
    for k in range(n_req):
        f = int(rng.integers(0, len(sizes)))
        ns = int(rng.integers(1, 17))
        tol = [1e-8, 1e-10][int(rng.integers(0, 2))]
        reqs.append((f, ns, tol, k))
    res = {"requests": n_req, "hbm_budget": budget, "prec": "fp32_12r (FP64 phase to 3e-4)" if mixed else "fp64"}
    with lqcd.Server(budget, max_slots=16, max_queue=4096) as srv:
        if mixed:
            srv.set_opts(prec=1, recon=12, fp64_until=3e-4)
        fids = [srv.register_field(d, inputs.random_links(d)) for d in sizes]
        srcs = {f: inputs.gaussian_field(sizes[f], k=100 + f) for f in range(len(sizes))}
        res["fields"] = [f"{d[0]}^4" for d in sizes]

        def run(arrivals):
            """Submit at the given offsets; returns (wall, latencies, peak bytes, peak slots, worst residual)."""
            t0 = time.perf_counter()
            pend, lat = [], []
            peak_b = peak_s = peak_q = 0
            worst = 0.0
            i = 0
            while i < len(reqs) or pend:
                now = time.perf_counter() - t0
                while i < len(reqs) and arrivals[i] <= now:
                    f, ns, tol, k = reqs[i]
                    pend.append((srv.submit(fids[f], MASS, inputs.log_shifts(ns), tol, srcs[f]), f, ns, tol,
                                 time.perf_counter()))
                    i += 1
                keep = []
                for t, f, ns, tol, ts in pend:
                    r = srv.poll(t, fids[f], ns)
                    if r is None:
                        keep.append((t, f, ns, tol, ts))
                    else:
                        lat.append(time.perf_counter() - ts)
                        worst = max(worst, max(r[1]["true_resid"]) / tol)
                        assert worst <= 1.0
                pend = keep
                st = srv.stats()
                peak_b = max(peak_b, st["hbm_in_use"])
                peak_s = max(peak_s, st["active_slots"])
                peak_q = max(peak_q, st["queued"])
                time.sleep(0.0005)
            return time.perf_counter() - t0, np.array(lat), peak_b, peak_s, peak_q, worst

        def summary(wall, lat, peak_b, peak_s, peak_q, worst):
            return {"solves_per_s": round(len(reqs) / wall, 3), "wall_s": round(wall, 2),
                    "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
                    "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
                    "peak_admitted_bytes": int(peak_b), "peak_active_slots": int(peak_s),
                    "peak_queued": int(peak_q), "max_true_resid_over_tol": round(worst, 3)}

        out = run(np.zeros(len(reqs)))
        cap = len(reqs) / out[0]
        res["burst"] = summary(*out)
        for load in loads:
            rate = load * cap
            out = run(inputs.poisson_arrivals(rate, len(reqs)))
            res[f"poisson_{load:g}"] = {"rate_hz": round(rate, 3), **summary(*out)}
        st = srv.stats()
        res["ticks"] = st["ticks"]
        res["rejected"] = st["rejected"]
    if not sequential:
        return res
    # the same requests solved one after another by the plain FP64 solver
    import torch
    ctxs, bds = [], []
    for f, d in enumerate(sizes):
        c = lqcd.Context(d)
        c.links_upload(inputs.random_links(d))
        ctxs.append(c)
        bds.append(lqcd.to_device_spinor(inputs.gaussian_field(d, k=100 + f)))
    for f in range(len(sizes)):  # graphs and workspaces
        ctxs[f].mscg_solve_dev(MASS, inputs.log_shifts(16), 1e-10, bds[f],
                               torch.empty((16, 3, ctxs[f].Vh), dtype=torch.complex128, device="cuda"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    by_size = [0.0] * len(sizes)
    for f, ns, tol, k in reqs:
        xd = torch.empty((ns, 3, ctxs[f].Vh), dtype=torch.complex128, device="cuda")
        t1 = time.perf_counter()
        ctxs[f].mscg_solve_dev(MASS, inputs.log_shifts(ns), tol, bds[f], xd)  # returns when solved
        by_size[f] += time.perf_counter() - t1
    torch.cuda.synchronize()
    seq = len(reqs) / (time.perf_counter() - t0)
    for c in ctxs:
        c.close()
    res["sequential_fp64_solves_per_s"] = round(seq, 3)
    res["sequential_s_by_lattice"] = {f"{d[0]}^4": round(t, 3) for d, t in zip(sizes, by_size)}
    # Packing can hide the launch-bound small lattices behind the large ones,
    # but the 24^4 and 32^4 solves already stream at HBM speed alone: the
    # burst cannot beat the sequential time of those.
    big = sum(t for d, t in zip(sizes, by_size) if d[0] >= 24)
    if big > 0:
        res["bound_burst_vs_sequential_if_large_lattices_stay_bandwidth_bound"] = round(sum(by_size) / big, 3)
    res["speedup_burst_vs_sequential_fp64"] = round(res["burst"]["solves_per_s"] / seq, 3)
    return res


# ---------------------------------------------------------------- ours
def rel_diff_per_shift(x, xref):
    """max over shifts of ||x_i - xref_i|| / ||xref_i|| (device complex128 [n][3][Vh])."""
    d = (x - xref).reshape(x.shape[0], -1).abs().pow(2).sum(1).sqrt()
    n = xref.reshape(x.shape[0], -1).abs().pow(2).sum(1).sqrt()
    return float((d / n).max())


def mixed_48_bench(lqcd, inputs, torch, with_oracle=False):
    """Mixed precision on 48^4 (same mass and shifts): FP32 12-real links with an
    FP64 phase to 3e-4, and FP16 12-real links, both with FP64 reliable updates
    and per-shift refinement, against the FP64 solver on the same lattice.  The
    oracle recomputes the true residual of the smallest, a middle and the largest
    shift of every result.  with_oracle: one full FP64 oracle solve (all host
    cores, minutes) gives every shift's error of every result against it."""
    dims = (48, 48, 48, 48)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=0)
    shifts = inputs.log_shifts(N_SHIFT)
    ctx = lqcd.Context(dims)
    ctx.links_upload(U)
    bd = lqcd.to_device_spinor(b)
    xd = torch.empty((N_SHIFT, 3, ctx.Vh), dtype=torch.complex128, device="cuda")
    out = {"lattice": list(dims)}
    from oracle import oracle
    orc = oracle()
    orc.set_threads(0)
    sample = (0, 7, N_SHIFT - 1)
    results = {}
    x64 = None
    for name, kw in [("fp64", dict(prec=0, recon=18)), ("fp32_12r", dict(prec=1, recon=12, fp64_until=3e-4)),
                     ("fp16_12r", dict(prec=2, recon=12, fp64_until=0.0))]:
        ctx.set_opts(**kw)
        ctx.mscg_solve_dev(MASS, shifts, TOL, bd, xd)  # warm-up (graph capture, workspaces)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = ctx.mscg_solve_dev(MASS, shifts, TOL, bd, xd)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"solves_per_s": round(1.0 / dt, 4), "s": round(dt, 3), "iters": info["iters"],
                     "refine_iters": info["refine_iters"], "reliable_updates": info["reliable_updates"],
                     "max_true_resid": max(info["true_resid"])}
        if x64 is None:
            x64 = xd.clone()
        else:
            out[name]["max_rel_diff_vs_fp64_solution"] = rel_diff_per_shift(xd, x64)
        out[name]["oracle_true_resid_sampled"] = {
            f"{shifts[i]:.3g}": orc.true_residual(dims, U, MASS, shifts[i], b, lqcd.from_device_spinor(xd[i]))
            for i in sample}
        if with_oracle:
            results[name] = lqcd.from_device_spinor(xd)
    for name in ("fp32_12r", "fp16_12r"):
        out[f"speedup_{name}_vs_fp64"] = round(out["fp64"]["s"] / out[name]["s"], 3)
    if with_oracle:
        t0 = time.perf_counter()
        xo, oinfo = orc.mscg(dims, U, MASS, shifts, b, TOL)
        out["oracle_solve"] = {"s": round(time.perf_counter() - t0, 1), "iters": oinfo["iters"],
                               "threads": orc.set_threads(0), "status": oinfo["status"]}
        for name, x in results.items():
            out[name]["rel_err_vs_oracle_per_shift"] = [
                float(np.linalg.norm(x[i] - xo[i]) / np.linalg.norm(xo[i])) for i in range(N_SHIFT)]
            out[name]["bound_2_kappa_tol"] = [2 * (MASS ** 2 + sg + 16) / (MASS ** 2 + sg) * TOL for sg in shifts]
    out["note"] = "second of two solves of each kind (the first captures graphs and allocates workspaces)"
    ctx.close()
    return out


def fma_rates_bench(lqcd, sweep):
    """Measured FP64 / FP32 FMA issue rates and the native-FP64 D_eo against
    the FP64 one: 288 DFMA + 54 DMUL per output site (8 half-hops of a 3x3
    complex mat-vec, the hop signs and the 1/2)."""
    r = lqcd.measure_fma_rates()
    out = {k: round(v / 1e12, 4) for k, v in r.items()}
    out["unit"] = "T FMA/s"
    for L, v in sweep.items():
        nat = v.get("fp64_native_dfma")
        if nat:
            ops = (288 + 54) / (nat["ns_per_site"] * 1e-9)
            out[f"native_fp64_deo_{L}"] = {"T_fp64_op_per_s": round(ops / 1e12, 4),
                                           "frac_of_measured_fp64_rate": round(ops / r["fp64_fma_per_s"], 3)}
    return out


class L2Flush:
    """Flush between timed launches: write a 256 MB buffer (twice L2), then read
    another 256 MB, so that L2 holds clean lines of the read buffer.  A write
    alone leaves ~129 MB of dirty lines whose write-back the next kernel would
    pay for (measured: +9 % on a 32^4 D_eo)."""

    def __init__(self, torch):
        self.w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def fill_(self, v):
        self.w.fill_(v)
        self.r.sum()


# Table md-norm (gauge part of the MD step, ns per lattice site), 32^4 column;
# other hardware, quoted as context only.
PAPER_MD_NS_32 = {"P100": 51.72, "GK210": 201.82, "E5-2697v4": 944.40, "E5-2630v3": 1719.97}


def gauge_md_bench(lqcd, inputs, L=32, beta=5.5, eps=0.01):
    """One gauge MD step (momentum update with the tree-level Symanzik force,
    then the link update) per lattice site on L^4, FP32 and FP64, as in
    Table md-norm; flop count per site from the kernels' SU(3) products."""
    dims = (L,) * 4
    V = L ** 4
    U = inputs.random_links(dims)
    H = inputs.random_momenta(dims)
    ctx = lqcd.Context(dims)
    ctx.links_upload(U)
    ctx.mom_upload(H)
    del U, H
    # per link: 67 SU(3) products in the staple sum, 1 for U A, about 16 in the
    # exponential and 1 for exp(i eps H) U, 198 flops each; 4 links per site
    flops_site = 4 * (67 + 1 + 16 + 1) * 198
    out = {"lattice": list(dims), "beta": beta, "eps": eps, "flops_per_site_approx": flops_site,
           "paper_ns_per_site_32^4_context": PAPER_MD_NS_32}
    for name, prec, n in (("fp32", 1, 20), ("fp64", 0, 4), ("fp64_native", 3, 4)):
        ctx.gauge_md_steps(beta, eps, 1, prec)  # warm-up (copies to the precision)
        t0 = time.perf_counter()
        ctx.gauge_md_steps(beta, eps, n, prec)
        dt = (time.perf_counter() - t0) / n
        out[name] = {"ns_per_site": round(dt * 1e9 / V, 3), "ms_per_step": round(dt * 1e3, 3),
                     "tflops": round(flops_site * V / dt / 1e12, 3),
                     "speedup_vs_paper_P100": round(PAPER_MD_NS_32["P100"] / (dt * 1e9 / V), 2)}
    ctx.close()
    return out


def fermion_force_bench(lqcd, inputs):
    """Fermion force of phi^dag r(A) phi on the 32^4 workload (15 quadrature
    poles of x^(-1/2), m = 0.01, tol 1e-10): one momentum update against the
    rational application alone (the difference is the 15 D_oe applications
    and the force kernel)."""
    from paper_1701_00426_gb300 import rational
    a0, a, sg = rational.inverse_sqrt_poles(N_SHIFT, MASS * MASS, MASS * MASS + 16.0)
    U = inputs.random_links(DIMS)
    phi = inputs.gaussian_field(DIMS, k=0)
    ctx = lqcd.Context(DIMS)
    ctx.links_upload(U)
    ctx.mom_upload(inputs.random_momenta(DIMS))
    del U
    ctx.fermion_force_update(MASS, a0, a, sg, TOL, phi, 0.0)  # warm-up (graphs, workspaces)
    t0 = time.perf_counter()
    act, info = ctx.fermion_force_update(MASS, a0, a, sg, TOL, phi, 0.01)
    dt_f = time.perf_counter() - t0
    t1 = time.perf_counter()
    ctx.rational_apply(MASS, a0, a, sg, TOL, phi)
    dt_r = time.perf_counter() - t1
    ctx.close()
    V = int(np.prod(DIMS))
    return {"poles": N_SHIFT, "force_updates_per_s": round(1.0 / dt_f, 4), "s": round(dt_f, 4),
            "rational_apply_s": round(dt_r, 4), "force_beyond_solve_ms": round(1e3 * (dt_f - dt_r), 2),
            "force_beyond_solve_ns_per_site": round(1e9 * (dt_f - dt_r) / V, 2), "action": act,
            "iters": info["iters"], "max_true_resid": max(info["true_resid"][:N_SHIFT])}


def stout_bench(lqcd, inputs, rho=0.15, levels=2):
    """Stout smearing on the 32^4 workload (native FP64): smearing the links
    `levels` times, the force chain through the levels (lqcd_stout_force: a
    host call that uploads the force on the smeared links and downloads the
    one on the thin links, 2 x 604 MB of transfers included), and the fermion
    force update on the smeared links (solve, force and chain)."""
    from paper_1701_00426_gb300 import rational
    V = int(np.prod(DIMS))
    U = inputs.random_links(DIMS)
    ctx = lqcd.Context(DIMS)
    ctx.links_upload(U)
    ctx.mom_upload(inputs.random_momenta(DIMS))
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        ctx.stout_smear(rho, levels)
        ts.append(time.perf_counter() - t0)
        ctx.stout_restore()
    ctx.stout_smear(rho, levels)
    F = np.asarray(inputs.random_momenta(DIMS, seed=5))
    ctx.stout_force(F)  # warm-up (scratch buffers)
    t0 = time.perf_counter()
    ctx.stout_force(F)
    dt_chain = time.perf_counter() - t0
    del F, U
    a0, a, sg = rational.inverse_sqrt_poles(N_SHIFT, MASS * MASS, MASS * MASS + 16.0)
    phi = inputs.gaussian_field(DIMS, k=0)
    ctx.fermion_force_update(MASS, a0, a, sg, TOL, phi, 0.0)  # warm-up
    t0 = time.perf_counter()
    act, info = ctx.fermion_force_update(MASS, a0, a, sg, TOL, phi, 0.01)
    dt_f = time.perf_counter() - t0
    ctx.close()
    smear = min(ts)
    return {"rho": rho, "levels": levels, "smear_ms": round(1e3 * smear, 2),
            "smear_ns_per_site_per_level": round(1e9 * smear / V / levels, 2),
            "force_chain_host_call_s": round(dt_chain, 4),
            "force_chain_ns_per_site_per_level_incl_transfers": round(1e9 * dt_chain / V / levels, 2),
            "fermion_force_update_smeared_s": round(dt_f, 4), "iters_on_smeared_links": info["iters"],
            "max_true_resid": max(info["true_resid"][:N_SHIFT])}


def rational_bench(lqcd, inputs, torch):
    """RHMC rational function on the 32^4 workload: y = r(A) b with the 15
    quadrature poles of x^(-1/2) on [m^2, m^2 + 16] and the action Re <b, y>,
    through the device call (inputs resident) and the host call; the host call
    returns one spinor (25 MB) where the multi-shift host call returns 15."""
    from paper_1701_00426_gb300 import rational
    a0, a, sg = rational.inverse_sqrt_poles(N_SHIFT, MASS * MASS, MASS * MASS + 16.0)
    U = inputs.random_links(DIMS)
    b = inputs.gaussian_field(DIMS, k=0)
    ctx = lqcd.Context(DIMS)
    ctx.links_upload(U)
    del U
    bd = lqcd.to_device_spinor(b)
    yd = torch.empty_like(bd)
    ctx.rational_apply_dev(MASS, a0, a, sg, TOL, bd, yd)  # warm-up (graph capture, workspaces)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    act, info = ctx.rational_apply_dev(MASS, a0, a, sg, TOL, bd, yd)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    y, act_h, _ = ctx.rational_apply(MASS, a0, a, sg, TOL, b)
    dth = time.perf_counter() - t1
    t2 = time.perf_counter()
    ctx.mscg_solve(MASS, sg, TOL, b)
    dtm = time.perf_counter() - t2
    ctx.close()
    n3 = 3 * (int(np.prod(DIMS)) // 2)
    return {"poles": N_SHIFT, "function": "x^(-1/2), Gauss-Legendre quadrature poles on [m^2, m^2+16]",
            "rational_error_on_interval": rational.max_rel_error(a0, a, sg, MASS * MASS, MASS * MASS + 16.0),
            "device_applies_per_s": round(1.0 / dt, 4), "host_applies_per_s": round(1.0 / dth, 4),
            "host_mscg_solves_per_s_same_poles": round(1.0 / dtm, 4),
            "d2h_bytes_host_apply": n3 * 16, "d2h_bytes_host_mscg": N_SHIFT * n3 * 16,
            "action": act, "action_host_call": act_h, "iters": info["iters"],
            "max_true_resid": max(info["true_resid"][:N_SHIFT])}


def deo_sweep(lqcd, inputs, torch, flush, hbm_peak, sizes):
    """ns/site and algorithmic GB/s of one D_eo (odd -> even, library-tuned launch
    shape), median and best of reps with L2 flushed before each (L2Flush);
    fractions of the measured copy bandwidth and of the 7.9 TB/s nominal."""
    out = {}
    variants = [("fp64", 0, 18, torch.complex128, 1248.0), ("fp64_12r", 0, 12, torch.complex128, 864.0),
                ("fp64_native_dfma", 3, 18, torch.complex128, 1248.0), ("fp32_18r", 1, 18, torch.complex64, 624.0),
                ("fp32_12r", 1, 12, torch.complex64, 432.0), ("fp16_12r", 2, 12, torch.complex64, 240.0)]
    for L in sizes:
        dims = (L,) * 4
        U = inputs.random_links(dims)
        with lqcd.Context(dims) as c:
            c.links_upload(U)
            del U
            res = {}
            for name, prec, recon, dt, bps in variants + [("fp16_12r_fp16_spinors_site_norm", None, 12, None, 224.0)]:
                s = torch.cuda.current_stream()
                if prec is None:  # FP16 spinors with a per-site norm (lqcd_deo_apply_h16)
                    hx, nx = lqcd.to_device_h16(inputs.gaussian_field(dims))
                    ho, no = torch.empty_like(hx), torch.empty_like(nx)

                    def apply():
                        c.deo_apply_h16(0, hx, nx, ho, no, s)
                else:
                    x = lqcd.to_device_spinor(inputs.gaussian_field(dims), dtype=dt)
                    o = torch.empty_like(x)

                    def apply():
                        c.deo_apply_ex(0, prec, recon, x, o, s)
                for _ in range(3):
                    apply()
                ts = []
                reps = 10 if L >= 48 else 20
                for _ in range(reps):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    apply()
                    e1.record(s)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                med = float(np.median(ts))
                gbs = bps * c.Vh / (med * 1e-3) / 1e9
                code = c.deo_tuned_config(prec, recon) if prec is not None else 5120 + 128
                res[name] = {"ns_per_site": round(med * 1e6 / c.Vh, 4),
                             "tuned": {"kind": ["per-thread", "2 threads/site", "4 threads/site", "staged",
                                                "8 threads/site", "per-thread unrolled"][code >> 10],
                                       "threads": code & 1023},
                             "best_ns_per_site": round(min(ts) * 1e6 / c.Vh, 4), "GB_s": round(gbs, 1),
                             "frac_hbm": round(gbs / hbm_peak, 3), "frac_nominal_7900": round(gbs / 7900.0, 3),
                             "bytes_per_site": bps}
                if prec is None:
                    del hx, nx, ho, no
                else:
                    del x, o
        out[f"{L}^4"] = res
        torch.cuda.empty_cache()
    return out


KERNEL_VARIANTS = {"f32_12": ("PREC_FP32", 12, "complex64"), "f16_12": ("PREC_FP16", 12, "complex64"),
                   "f64_12": ("PREC_FP64", 12, "complex128"), "f64": ("PREC_FP64", 18, "complex128")}


def kernels_probe(lqcd, inputs, torch, L, which, mrhs_n):
    """Fixed launch sequence for ncu captures of single kernels on L^4.
    D_eo variants (which): every variant is called once (the autotuner's
    timing, unless LQCD_TUNE_CACHE already holds its choice, plus one
    launch), then twice more.  Multi-RHS (mrhs_n > 0, FP32 12-real): in the
    site-major and then the field-major layout, one call (tuning plus one
    launch), then five launches after a 256 MB buffer write.  The repeated
    launches sit in NVTX ranges ("deo_timed", "mrhs_site_major",
    "mrhs_field_major") that ncu --nvtx-include selects.  Returns the tuned
    launch codes and the event-timed launches."""
    dims = (L,) * 4
    out = {"lattice": list(dims), "deo": {}, "mrhs": {}}
    with lqcd.Context(dims) as c:
        c.links_upload(inputs.random_links(dims))
        s = torch.cuda.current_stream()
        bufs = {}
        for w in which:
            pname, recon, dt = KERNEL_VARIANTS[w]
            x = lqcd.to_device_spinor(inputs.gaussian_field(dims), dtype=getattr(torch, dt))
            o = torch.empty_like(x)
            c.deo_apply_ex(0, getattr(lqcd, pname), recon, x, o, s)
            bufs[w] = (x, o)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("deo_timed")
        for w in which:
            pname, recon, _ = KERNEL_VARIANTS[w]
            ts = []
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                c.deo_apply_ex(0, getattr(lqcd, pname), recon, *bufs[w], s)
                e1.record(s)
                e1.synchronize()
                ts.append(round(e0.elapsed_time(e1) * 1e3, 1))
            out["deo"][w] = {"tuned_code": c.deo_tuned_config(getattr(lqcd, pname), recon), "us": ts}
        torch.cuda.nvtx.range_pop()
        del bufs
        if mrhs_n > 0:
            flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
            for layout in (0, 1):
                shape = (3, c.Vh, mrhs_n) if layout == 0 else (3, mrhs_n, c.Vh)
                x = torch.randn(shape, dtype=torch.complex64, device="cuda")
                o = torch.empty_like(x)
                c.deo_apply_mrhs(0, mrhs_n, 12, x, o, s, layout=layout)
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push(["mrhs_site_major", "mrhs_field_major"][layout])
                ts = []
                for _ in range(5):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    c.deo_apply_mrhs(0, mrhs_n, 12, x, o, s, layout=layout)
                    e1.record(s)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e3)
                torch.cuda.nvtx.range_pop()
                med = float(np.median(ts))
                out["mrhs"][["site_major", "field_major"][layout]] = {
                    "n": mrhs_n, "us": round(med, 1), "ns_per_field_site": round(med * 1e3 / (c.Vh * mrhs_n), 4)}
                del x, o
    return out


def run_ours(args, rank, world, local):
    global DIMS, WORKLOAD
    if args.lattice != 32:
        DIMS = (args.lattice,) * 4
        WORKLOAD = WORKLOAD.replace("32^4", f"{args.lattice}^4")
    import torch
    from paper_1701_00426_gb300 import build, inputs, lqcd
    torch.cuda.set_device(local)
    # one rank per node compiles (the others would write the same objects);
    # every rank loads the library after the barrier
    if local == 0:
        build.build()
    barrier(world)
    lqcd.load()
    hbm_peak, peak_src = peaks()
    if args.only_kernels is not None:
        if rank == 0:
            which = [w for w in args.only_kernels.split(",") if w]
            print(json.dumps({"metric": METRIC, "config": {"only_kernels": which, "mrhs_n": args.mrhs_n},
                              "kernels_probe": kernels_probe(lqcd, inputs, torch, args.lattice, which,
                                                             args.mrhs_n)}), flush=True)
        return
    if args.only_md:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": "ns/site", "config": {"only_md": True},
                              "gauge_md": gauge_md_bench(lqcd, inputs, L=args.lattice)}), flush=True)
        return
    if args.only_serving:
        if rank == 0:
            b = int(args.serving_budget_gb * (1 << 30))
            n = args.serving_requests
            out = {"serving": serving_bench(lqcd, inputs, n_req=n, budget=b),
                   "serving_mixed": serving_bench(lqcd, inputs, n_req=n, loads=(0.8,), budget=b, mixed=True,
                                                  sequential=False),
                   "serving_2gb": serving_bench(lqcd, inputs, n_req=n, loads=(0.95,), budget=2 << 30,
                                                sequential=False, sides=(8, 16, 24))}
            print(json.dumps({"metric": METRIC, "unit": "solves/s", "config": {"only_serving": True}, **out}),
                  flush=True)
        return
    if args.only_mixed_48:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": "solves/s", "config": {"only_mixed_48": True},
                              "mixed_48": mixed_48_bench(lqcd, inputs, torch, with_oracle=args.with_oracle_48)}),
                  flush=True)
        return
    if args.only_deo:
        if rank == 0:
            flush = L2Flush(torch)
            print(json.dumps({"metric": METRIC, "unit": "ns/site", "config": {"only_deo": True},
                              "deo": deo_sweep(lqcd, inputs, torch, flush, hbm_peak, args.sweep)}), flush=True)
        return
    U = inputs.random_links(DIMS)
    b = inputs.gaussian_field(DIMS, k=rank)
    shifts = inputs.log_shifts(N_SHIFT)
    ctx = lqcd.Context(DIMS)
    ctx.links_upload(U)
    if args.solve_prec == "fp32":
        ctx.set_opts(prec=1, recon=12, fp64_until=3e-4)
    if args.stencils == "per-thread":
        ctx.set_opts(staged=0)
    bd = lqcd.to_device_spinor(b)
    xd = torch.empty((N_SHIFT, 3, ctx.Vh), dtype=torch.complex128, device="cuda")
    info = None
    for _ in range(args.warmup):
        info = ctx.mscg_solve_dev(MASS, shifts, TOL, bd, xd)
    torch.cuda.synchronize()
    barrier(world)
    s = torch.cuda.current_stream()
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            infos.append(ctx.mscg_solve_dev(MASS, shifts, TOL, bd, xd, stream=s))
        e1.record(s)
        torch.cuda.synchronize()
    barrier(world)
    t_ms = e0.elapsed_time(e1)
    value, t_max = job_throughput(args.steps, t_ms, world)
    clocks = clk.summary()
    launches = int(sum(i["kernel_launches"] for i in infos))
    worst_res = float(max(max(i["true_resid"]) for i in infos))
    it = infos[-1]
    if args.only_solve:
        if rank == 0:
            # per-kernel ms of the iteration (kernels launched one by one, CUDA events)
            kms, _ = ctx.profile_iteration(MASS, shifts, bd, tol=TOL, iters=it["iters"])
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                              "iters": it["iters"], "max_true_resid": worst_res, "gpu_launches": launches,
                              "kernel_ms": [round(m, 4) for m in kms],
                              "config": {"workload": WORKLOAD, "only_solve": True, "prec": args.solve_prec,
                                         "stencils": args.stencils}}),
                  flush=True)
        ctx.close()
        return

    # end to end through the host API (numpy buffers, copies inside); the
    # output array is allocated and touched once, as a caller's loop reuses it
    # host buffers in pinned (page-locked) memory, so the copies run at the
    # link's speed without staging through a bounce buffer
    e2e_steps = max(1, args.steps)
    b_pin = torch.from_numpy(np.ascontiguousarray(b)).pin_memory().numpy()
    xh = torch.zeros((N_SHIFT, ctx.Vh, 3), dtype=torch.complex128).pin_memory().numpy()
    b = b_pin
    xh, _ = ctx.mscg_solve(MASS, shifts, TOL, b, out=xh)  # untimed warm-up of the host path
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        xh, _ = ctx.mscg_solve(MASS, shifts, TOL, b, out=xh)
    torch.cuda.synchronize()
    e2e_t = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": world * e2e_steps / e2e_t, "unit": "solves/s", "host_buffers": "pinned",
           "h2d_bytes_per_step": int(b.nbytes),
           "d2h_bytes_per_step": int(xh.nbytes)}
    if rank != 0:
        ctx.close()
        return

    # per-kernel times of the iteration (same kernels, launched one by one)
    n_it = it["iters"]
    ms, nact = ctx.profile_iteration(MASS, shifts, bd, tol=TOL, iters=n_it)
    Vh = ctx.Vh
    kbytes = [Vh * 1248.0, Vh * 1296.0, Vh * 144.0, Vh * (48.0 + 192.0 * nact)]
    knames = ["D_oe (t = D_oe p)", "D_eo + normal-operator epilogue + <p,q>", "r -= alpha q, ||r||^2",
              "shifted updates x_i, p_i"]
    shares = [m / sum(ms) for m in ms]
    kdom = int(np.argmax(ms))
    achieved = kbytes[kdom] / (ms[kdom] * 1e-3) / 1e9
    tps = k2_traffic_per_site() if kdom == 1 else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 3),
                "traffic": None if tps is None else round(tps * Vh / 1e9, 4),
                "traffic_unit": "GB per launch", "algorithmic": round(kbytes[kdom] / 1e9, 4),
                "kernel": knames[kdom],
                "peak_source": peak_src, "note": "of measured"}
    kernels = {knames[k]: {"ms": round(ms[k], 4), "share": round(shares[k], 3),
                           "GB_s": round(kbytes[k] / (ms[k] * 1e-3) / 1e9, 1)} for k in range(4)}

    # mixed precision on the same workload
    mixed = {}
    x64 = xd.clone()
    for name, prec, recon, fu in [("fp32_12r", 1, 12, 3e-4), ("fp32_18r", 1, 18, 3e-4),
                                  ("fp32_12r_no_fp64_phase", 1, 12, 0.0), ("fp16_12r", 2, 12, 0.0)]:
        try:
            ctx.set_opts(prec=prec, recon=recon, fp64_until=fu)
            ctx.mscg_solve_dev(MASS, shifts, TOL, bd, xd)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mi = ctx.mscg_solve_dev(MASS, shifts, TOL, bd, xd)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            mixed[name] = {"solves_per_s": round(1.0 / dt, 4), "speedup_vs_fp64": round((1.0 / dt) / value, 3),
                           "max_true_resid": max(mi["true_resid"]), "iters": mi["iters"],
                           "refine_iters": mi["refine_iters"], "reliable_updates": mi["reliable_updates"],
                           "fp64_until": fu,
                           "max_rel_diff_vs_fp64_solution": rel_diff_per_shift(xd, x64)}
            # the low-precision iteration's kernels, first iterations (before any reliable update)
            mms, _ = ctx.profile_iteration(MASS, shifts, bd, tol=TOL, iters=30)
            mixed[name]["kernels_ms"] = [round(m, 4) for m in mms]
        except Exception as exc:  # reported, never hidden
            mixed[name] = {"error": repr(exc)}
    ctx.set_opts(prec=0, recon=18, fp64_until=3e-4)
    ctx.close()
    del bd, xd
    torch.cuda.empty_cache()

    flush = L2Flush(torch)
    sweep = deo_sweep(lqcd, inputs, torch, flush, hbm_peak, args.sweep)
    del flush
    torch.cuda.empty_cache()
    extras = {}
    for name, fn in [("rational", lambda: rational_bench(lqcd, inputs, torch)),
                     ("gauge_md", lambda: gauge_md_bench(lqcd, inputs)),
                     ("fermion_force", lambda: fermion_force_bench(lqcd, inputs)),
                     ("stout", lambda: stout_bench(lqcd, inputs)),
                     ("mixed_48", lambda: mixed_48_bench(lqcd, inputs, torch, with_oracle=args.with_oracle_48)),
                     ("fma_rates", lambda: fma_rates_bench(lqcd, sweep)),
                     ("batched", lambda: batched_bench(lqcd, inputs, torch, hbm_peak)),
                     ("packed", lambda: packed_bench(lqcd, inputs)),
                     ("serving", lambda: serving_bench(lqcd, inputs, n_req=args.serving_requests,
                                                       budget=int(args.serving_budget_gb * (1 << 30)))),
                     ("serving_mixed", lambda: serving_bench(lqcd, inputs, n_req=args.serving_requests, loads=(0.8,),
                                                             budget=int(args.serving_budget_gb * (1 << 30)),
                                                             mixed=True, sequential=False)),
                     ("serving_2gb", lambda: serving_bench(lqcd, inputs, n_req=args.serving_requests, loads=(0.95,),
                                                           budget=2 << 30, sequential=False, sides=(8, 16, 24)))]:
        if name in args.skip:
            continue
        try:
            extras[name] = fn()
        except Exception as exc:  # reported, never hidden
            extras[name] = {"error": repr(exc)}
        torch.cuda.empty_cache()

    sm, sf = extras.get("serving_mixed", {}), extras.get("serving", {})
    if "burst" in sm and "sequential_fp64_solves_per_s" in sf:
        sm["speedup_burst_vs_sequential_fp64"] = round(sm["burst"]["solves_per_s"] / sf["sequential_fp64_solves_per_s"], 3)

    # CPU baseline: the oracle on a bounded sample of the same workload
    counts = oracle_counts()
    src = "the oracle's own full-solve counts (tests/golden/oracle_counts.json)"
    if counts is None:
        counts = {"iters": it["iters"], "shift_iters": [s_ or it["iters"] for s_ in it["shift_iters"]]}
        src = "the GPU solve's counts"
    base, per_shift, fixed, thr, sample_s = oracle_sample(U, b, shifts)
    cpu_v = 1.0 / cpu_solve_seconds(base, per_shift, fixed, counts)
    deo_cpu = oracle_deo_sample(inputs)
    cpu = {"value": cpu_v, "unit": "solves/s", "cores": thr, "kind": "oracle", "deo_ns_per_site": deo_cpu,
           "modelled": True, "model_validation": validate_cpu_model(),
           "recorded_full_solve": {k: counts.get(k) for k in ("seconds", "threads")} if "seconds" in counts else None,
           "sample_wall_s": round(sample_s, 1),
           "sample": "oracle multi-shift CG on the same 32^4 workload stopped after 2 and 12 iterations, with all "
                     "15 shifts and with one (median of 3); whole solve = set-up + iterations x base cost + "
                     "shift-iterations x per-shift cost, with " + src}

    line = {"metric": METRIC, "value": round(value, 5), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "mass": MASS, "n_shift": N_SHIFT, "tol": TOL,
                       "prec": "fp64 (df64 iteration, IEEE FP64 true residual)", "parallelism": "replicas",
                       "l2": "inputs larger than L2 (links 604 MB, vectors 0.8 GB); no flush"},
            "iters": it["iters"], "refine_iters": it["refine_iters"], "max_true_resid": worst_res,
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
            "cpu_baseline": cpu, "kernels": kernels, "n_active_avg": round(nact, 2),
            "mixed": mixed, "deo": sweep, **extras}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sweep", type=int, nargs="*", default=[16, 24, 32, 48])
    ap.add_argument("--lattice", type=int, default=32, help="side of the solve lattice (default 32)")
    ap.add_argument("--skip", nargs="*", default=[], help="extra sections to skip: rational gauge_md fermion_force stout mixed_48 fma_rates batched "
                         "packed serving serving_mixed serving_2gb")
    ap.add_argument("--only-solve", action="store_true",
                    help="time the solves only (no e2e, profile, mixed, sweep, CPU legs); for ncu launch lists")
    ap.add_argument("--only-md", action="store_true",
                    help="only the gauge MD step timing at --lattice (for profiling)")
    ap.add_argument("--only-deo", action="store_true",
                    help="run the D_eo sweep only (sizes from --sweep); for ncu captures of the stencil")
    ap.add_argument("--only-kernels", default=None, metavar="VARIANTS",
                    help="fixed launch sequence for ncu captures on --lattice: D_eo variants, comma-separated, "
                         "from " + ",".join(KERNEL_VARIANTS) + " (may be empty), then multi-RHS with --mrhs-n")
    ap.add_argument("--mrhs-n", type=int, default=0, help="with --only-kernels: fields of the multi-RHS D_eo")
    ap.add_argument("--with-oracle-48", action="store_true",
                    help="mixed_48 section: also one full FP64 oracle solve on 48^4 (minutes on the host cores) "
                         "for every shift's error of the GPU results")
    ap.add_argument("--only-mixed-48", action="store_true", help="run the 48^4 mixed-precision section only")
    ap.add_argument("--only-serving", action="store_true",
                    help="run the serving sections only (FP64 with the sequential baseline, mixed, tight 2 GB)")
    ap.add_argument("--serving-requests", type=int, default=40, help="requests per serving run (default 40)")
    ap.add_argument("--serving-budget-gb", type=float, default=16.0, help="HBM budget of the serving runs")
    ap.add_argument("--solve-prec", choices=["fp64", "fp32"], default="fp64",
                    help="with --only-solve: precision of the timed solves (fp32: 12-real links, FP64 phase "
                         "to 3e-4, FP64 reliable updates)")
    ap.add_argument("--stencils", choices=["staged", "per-thread"], default="staged",
                    help="with --only-solve: the FP64 iteration's D_oe / D_eo kernels (per-thread: opts.staged = 0)")
    args = ap.parse_args()
    if args.solve_prec != "fp64" and not args.only_solve:
        ap.error("--solve-prec applies to --only-solve runs")
    if args.stencils != "staged" and not args.only_solve:
        ap.error("--stencils applies to --only-solve runs")
    if args.impl == "reference":
        # the oracle runs on the host; ranks other than 0 exit without work
        run_reference(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank, world, local = dist_setup(args.gpus)
    run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
