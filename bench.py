#!/usr/bin/env python3
"""Throughput of the E-A-HALS outer loop on GB300 (one JSON line on stdout).

A step is one outer iteration of Algorithm 2 (all kernels of the hot path:
Grams, W^T X, H sweeps + extrapolation, X H^T, W sweeps + error + restart
decision + Algorithm 3, finalize) on the dense noisy low-rank workload
m = 10000, n = 4000, r = 50 (FP32 path, paper defaults hp = 3, beta0 = 0.5,
eta = 1.5, gamma = 1.01, gamma_bar = 1.005, A-HALS sweep budget L_W = 40,
L_H = 100).  X (160 MB) is larger than the 129 MB L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own instance (independent problems, no
collective on the data path, weak scaling); the timed region is bracketed by
a barrier and synchronisation and the slowest rank's time is used.
``--impl reference`` times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "E-A-HALS outer iters/s & time-to-rel-err on 1 GB300; % of HBM roofline"
UNIT = "iter/s"
WORKLOAD = "dense_noisy_10000x4000_r50"
FP32_LANES_PER_SM = 128
NUM_SMS = 152


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the image-like, batched and document-like workload lines")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip e2e / time-to-target / phase profile (quick runs)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.out.read())) if len(r) >= 9]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(seed: int):
    from paper_1805_06604_gb300 import workloads as wl
    return wl.dense_noisy(seed)


def phase_work(P, lw, lh):
    """Algorithmic (flops, bytes) of one launch of every phase (FP32 data)."""
    m, n, r = P.m, P.n, P.r
    f4 = 4
    return {
        "gram_w": (2 * m * r * r, f4 * m * r),
        "wtx": (2 * m * n * r, f4 * (m * n + m * r + r * n)),
        "hals_h": (2 * r * r * lh * n, f4 * 5 * r * n),
        "gram_h": (2 * n * r * r, f4 * r * n),
        "xht": (2 * m * n * r, f4 * (m * n + r * n + m * r)),
        "hals_w": (2 * r * r * (lw + 1) * m, f4 * 3 * m * r),
        "finalize": (0, f4 * 4 * (m * r + r * n)),
    }


def load_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(kernel)
    if not ent:
        return None
    import hashlib
    h = hashlib.sha256()
    for rel in ent.get("sources", []):
        p = os.path.join(ROOT, rel)
        if not os.path.exists(p):
            return None
        with open(p, "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != ent.get("digest"):
        return None
    return ent.get("bytes_per_launch")


def sgemm_tflops(n: int = 8192, reps: int = 5) -> float:
    """A measured FP32 rate for the ALU roofline's context: cuBLAS SGEMM with
    TF32 off (the FMA pipes, as the CUDA-core kernels use them)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        g = torch.Generator(device="cuda").manual_seed(0)
        a = torch.rand((n, n), device="cuda", generator=g)
        b = torch.rand((n, n), device="cuda", generator=g)
        c = a @ b
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            c = a @ b
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1000.0 / reps
        del a, b, c
        return 2.0 * n ** 3 / s / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def l2_copy_gbs(mb: int = 24, reps: int = 200) -> float:
    """A measured L2 rate for the sparse products' gathers: device-to-device
    copies of a 24 MB buffer (source and destination stay in the 129 MB L2),
    read plus written bytes per second."""
    import torch
    n = mb * (1 << 20) // 4
    a = torch.rand(n, device="cuda")
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        b.copy_(a)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1000.0
    del a, b
    return 2.0 * 4 * n * reps / s / 1e9


def timed_steps(solver, steps, stream):
    """Seconds for `steps` graph replays of `solver`, on the device clock."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    solver.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0


def other_workloads(nmf, torch, stream):
    """The benchmark description's other single-GPU workloads, each measured
    briefly: the image-like precision study, the batched instances and the
    sparse document-like matrix."""
    import numpy as np
    from paper_1805_06604_gb300 import workloads as wl
    out = {}
    # Image-like 10304 x 4000, r = 64: FP32 / TF32 / BF16X3 products.
    P = wl.image_like(0)
    Xd = torch.from_numpy(P.X).cuda()
    W0d, H0d = torch.from_numpy(P.W0).cuda(), torch.from_numpy(P.H0).cuda()
    steps = 200
    img = {"workload": P.name, "steps": steps}
    for name, prec in (("fp32", nmf.NMF_PREC_FP32), ("tf32", nmf.NMF_PREC_TF32),
                       ("bf16x3", nmf.NMF_PREC_BF16X3)):
        sv = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream, precision=prec)
        sv.step(3)
        t = timed_steps(sv, steps, stream)
        W, H = sv.factors()
        img[name] = {"iters_per_s": steps / t, "relerr_direct": direct_relerr(Xd, W, H)}
        sv.close()
    out["image_like_precision_study"] = img
    del Xd, W0d, H0d
    # Batched: 512 uneven instances, one graph per iteration vs a launch loop.
    probs = wl.batch(count=512, seed=0)
    b = nmf.Batch([(Q.X, Q.r, Q.W0, Q.H0) for Q in probs])
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn in (("graph", b.step), ("loop", b.step_loop)):
        fn(1)
        torch.cuda.synchronize()
        e0.record()
        fn(20)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / 20.0
    pl = b.plan()
    plan = {"grouped": pl.grouped, "branches": pl.branches, "h_cols_per_cta": pl.h_cols_per_cta,
            "launches_per_iter": pl.launches_per_iter}
    if pl.grouped:
        # The per-instance chains on 64 branches, for comparison.
        b.set_plan(0, 64, 0)
        b.step(1)
        torch.cuda.synchronize()
        e0.record()
        b.step(20)
        e1.record()
        torch.cuda.synchronize()
        res["chains_64"] = e0.elapsed_time(e1) / 20.0
    b.close()
    out["batched_512"] = {"instances": 512, "plan": plan,
                          "graph_ms_per_iter": res["graph"], "loop_ms_per_iter": res["loop"],
                          "chains_graph_ms_per_iter": res.get("chains_64"),
                          "speedup": res["loop"] / res["graph"],
                          "instance_iters_per_s": 512 * 1000.0 / res["graph"]}
    # Document-like CSR 50000 x 20000, r = 30: E-A-HALS and A-HALS.
    P = wl.document_like(0)
    csr = (P.rowptr, P.colidx, P.val.astype(np.float32))
    doc = {"workload": P.name, "nnz": int(P.nnz), "steps": 300}
    for name, kw in (("eahals", {}), ("ahals", {"beta0": 0.0})):
        sv = nmf.Solver(None, P.r, P.W0.astype(np.float32), P.H0.astype(np.float32), csr=csr,
                        m=P.m, n=P.n, stream=stream, **kw)
        sv.step(3)
        t = timed_steps(sv, 300, stream)
        doc[name] = {"iters_per_s": 300 / t, "relerr": sv.info().relerr}
        sv.close()
    # The CSR products against HBM (stored entries: 4 B value + 4 B index
    # per nonzero, read once per product) and the factor rows they gather
    # (r floats per nonzero, served mostly from L2).
    sv = nmf.Solver(None, P.r, P.W0.astype(np.float32), P.H0.astype(np.float32), csr=csr,
                    m=P.m, n=P.n, stream=stream)
    sv.step(3)
    pm = sv.profile_phases(10)
    sv.close()
    hbm_gbs = peaks()[0]
    l2_gbs = l2_copy_gbs()
    doc["l2_copy_gbs_measured"] = l2_gbs
    nnz = float(P.nnz)
    for k in ("wtx", "xht"):
        s_ = pm[k] / 1000.0
        stored = 8.0 * nnz + 4.0 * P.r * (P.m + P.n)
        gathered = 4.0 * P.r * nnz
        doc[k] = {"us": pm[k] * 1000.0, "stored_gbs": stored / s_ / 1e9,
                  "frac_of_hbm": stored / s_ / 1e9 / hbm_gbs,
                  "gathered_gbs": gathered / s_ / 1e9,
                  "gathered_frac_of_l2": gathered / s_ / 1e9 / l2_gbs if l2_gbs else None}
    out["document_like_csr"] = doc
    # E-ANLS (exact NNLS subproblems, nmf_params.exact_nnls) and the A-HALS
    # inner stopping rule (delta = 0.1) on the dense noisy workload.
    Pd = wl.dense_noisy(0)
    Xd = torch.from_numpy(Pd.X).cuda()
    W0d, H0d = torch.from_numpy(Pd.W0).cuda(), torch.from_numpy(Pd.H0).cuda()
    extra = {}
    for name, kw, steps in (("eanls", {"exact_nnls": 1}, 50), ("delta_0.1", {"delta": 0.1}, 100)):
        sv = nmf.Solver(Xd, Pd.r, W0d, H0d, stream=stream, **kw)
        sv.step(3)
        t = timed_steps(sv, steps, stream)
        info = sv.info()
        ent = {"iters_per_s": steps / t, "steps": steps, "relerr_pair": sv.eval_error()[1],
               "sweeps_last_iter": [int(info.lh_used), int(info.lw_used)],
               "exact_failed": int(info.exact_failed)}
        ph = sv.profile_phases(3)
        ent["phase_us"] = {k: v * 1000.0 for k, v in ph.items()}
        extra[name] = ent
        sv.close()
    out["dense_noisy_variants"] = extra
    del Xd, W0d, H0d
    # The parameter study of Sec. 4.2 (reduced: one data set, two
    # initialisations, all 109 variants in batched graphs).
    from paper_1805_06604_gb300 import sweep
    study = {}
    for kind in ("low_rank", "full_rank"):
        summ, _, secs = sweep.run(kind, datasets=1, inits=2, iters=500)
        per = summ["per_variant"]
        study[kind] = {"seconds": secs, "variants": len(per), "runs": summ["runs"],
                       "iters": 500, "shape": "200x200 r=20",
                       "mean_E": {v: per[v]["mean_E"] for v in summ["ranking"]},
                       "ranking": summ["ranking"]}
    out["parameter_study"] = study
    # Sec. 3's line-search step beta* of every W-update (diagnostic trace) on
    # the low-rank synthetic data: the paper observes it near zero for most
    # iterations once near a stationary point.
    P = wl.low_rank(200, 200, 20, seed=1000)
    sv = nmf.Solver(P.X, P.r, P.W0, P.H0, line_search_trace=1)
    sv.step(500)
    bs = np.abs(sv.line_search_trace())
    sv.close()
    tail = bs[100:]
    out["line_search_beta_star"] = {"workload": "low_rank_200x200_r20", "iters": 500,
                                    "median_abs_after_100": float(np.median(tail)),
                                    "frac_abs_below_0.1_after_100": float(np.mean(tail < 0.1)),
                                    "median_abs_first_10": float(np.median(bs[:10]))}
    return out


def time_to_direct(sv, Xd, target, stream, max_iters=3000, chunk=10):
    """Device seconds and iterations until the returned factors' direct
    relative error is <= target (checked every `chunk` iterations, checks
    untimed).  The direct error is the common yardstick of the precision
    modes: the tensor-core modes' own e(k) carries a small offset from the
    tensor core's in-stage accumulation."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    secs, iters, rel = 0.0, 0, None
    while iters < max_iters:
        torch.cuda.synchronize()
        e0.record(stream)
        sv.step(chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        secs += e0.elapsed_time(e1) / 1000.0
        iters += chunk
        W, H = sv.factors()
        rel = direct_relerr(Xd, W, H)
        if rel <= target:
            return {"seconds": secs, "iters": iters, "reached": True, "relerr_direct": rel}
    return {"seconds": secs, "iters": iters, "reached": False, "relerr_direct": rel}


def restarts(sv):
    """Iterations whose restart test of Algorithm 2 rejected the step."""
    import numpy as np
    _, _, acc = sv.trace()
    return int(len(acc) - int(np.sum(acc)))


def direct_relerr(Xd, W, H):
    """||X - W H||_F / ||X||_F of returned factors, evaluated directly in FP64
    on the device in row blocks (a check beside the solver's own e(k))."""
    import torch
    Wd = torch.as_tensor(W, device=Xd.device, dtype=torch.float64)
    Hd = torch.as_tensor(H, device=Xd.device, dtype=torch.float64)
    num = 0.0
    den = 0.0
    for i in range(0, Xd.shape[0], 1024):
        Xb = Xd[i:i + 1024].double()
        num += float(((Xb - Wd[i:i + 1024] @ Hd) ** 2).sum())
        den += float((Xb ** 2).sum())
    return (num / den) ** 0.5


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for key in ("Model name", "Vendor ID"):
            for line in out.splitlines():
                if line.startswith(key + ":"):
                    return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_oracle(P, lw, lh, iters: int, threads: int):
    """The FP64 oracle as it stands, `iters` outer iterations of the
    workload on `threads` host threads; (iterations/s, seconds)."""
    import numpy as np
    import oracle as O
    O.build()
    O.set_threads(threads)
    p = O.Params(hp=3, lw=lw, lh=lh)
    X = O.Matrix(P.X.astype(np.float64))
    st = O.eahals_init(X, P.W0, P.H0, p)
    f2 = O.fro2(X)
    t0 = time.perf_counter()
    for _ in range(iters):
        O.eahals_step(X, st, p, fro2_x=f2)
    dt = time.perf_counter() - t0
    return iters / dt, dt


def run_reference(args, world, rank):
    if rank != 0:
        return None
    from paper_1805_06604_gb300 import nmf as _unused  # noqa: F401  (package importable)
    import numpy as np
    import oracle as O
    O.build()
    P = make_workload(args.seed)
    ncores = os.cpu_count() or 1
    O.set_threads(ncores)
    lw, lh = O.sweep_counts(P.m, P.n, P.nnz, P.r)
    p = O.Params(hp=3, lw=lw, lh=lh)
    X = O.Matrix(P.X.astype(np.float64))
    st = O.eahals_init(X, P.W0, P.H0, p)
    f2 = O.fro2(X)
    warm = min(args.warmup, 1)
    t0 = time.perf_counter()
    for _ in range(max(warm, 1)):
        O.eahals_step(X, st, p, fro2_x=f2)
    per = time.perf_counter() - t0
    budget = 150.0
    steps = max(1, min(args.steps, int(budget / max(per, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(steps):
        O.eahals_step(X, st, p, fro2_x=f2)
    dt = time.perf_counter() - t0
    value = steps / dt
    sample = (f"{steps} full outer iterations of {WORKLOAD} (FP64 oracle, OpenMP on all "
              f"{ncores} host cores, {cpu_model()}), after {max(warm, 1)} untimed; steps capped "
              f"to keep the run near {budget:.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": steps, "steps_requested": args.steps, "warmup": max(warm, 1),
            "ms_per_step": 1000.0 * dt / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": P.m, "n": P.n, "r": P.r, "lw": lw, "lh": lh,
                       "hp": 3, "beta0": 0.5, "eta": 1.5, "gamma": 1.01, "gamma_bar": 1.005},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model(), "nproc": ncores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    return line


def rank_max_seconds(t: float, dist, device) -> float:
    """The slowest rank's timed-region seconds (max over ranks; t itself on
    one process).  Every rank times its own independent instance."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(world: int, steps: int, t_max: float) -> float:
    """Iterations per second of the whole job: every rank ran `steps`
    iterations of its own instance within the slowest rank's time."""
    return world * steps / t_max


def instance_seed(seed: int, rank: int) -> int:
    """Each rank solves a different instance (weak scaling, no collective
    on the data path)."""
    return seed + rank


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1805_06604_gb300 import build as nb
    from paper_1805_06604_gb300 import nmf

    nb.build()
    nmf.load()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    P = make_workload(instance_seed(args.seed, rank))
    lw, lh = nmf.nmf_sweep_counts(P.m, P.n, P.nnz, P.r)
    stream = torch.cuda.current_stream()
    Xd = torch.from_numpy(P.X).cuda()
    W0d = torch.from_numpy(P.W0).cuda()
    H0d = torch.from_numpy(P.H0).cuda()
    solver = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream)
    solver.step(args.warmup)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    t = rank_max_seconds(e0.elapsed_time(e1) / 1000.0, dist, "cuda")
    info = solver.info()
    value = whole_job_value(world, args.steps, t)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": P.m, "n": P.n, "r": P.r, "lw": lw, "lh": lh,
                       "hp": 3, "beta0": 0.5, "eta": 1.5, "gamma": 1.01, "gamma_bar": 1.005,
                       "precision": "fp32", "parallelism": f"independent instance per GPU x{world}",
                       "l2": "inputs larger than L2 (X is 160 MB), no flush"},
            "clocks": clocks,
            "gpu_launches": int(info.launches_per_iter) * args.steps,
            "relerr_after_timed": info.relerr}
    if rank != 0:
        solver.close()
        return None
    if args.no_extras:
        solver.close()
        return line

    hbm_gbs, sm_max_mhz, peak_src = peaks()
    alu_tflops = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    # Per-phase device time: an event-instrumented pass over the same step.
    prof_iters = min(max(args.steps // 10, 5), 50)
    ms = solver.profile_phases(prof_iters)
    work = phase_work(P, lw, lh)
    phases = {}
    for k, v in ms.items():
        fl, by = work[k]
        s = v / 1000.0
        t_alu = fl / (alu_tflops * 1e12)
        t_hbm = by / (hbm_gbs * 1e9)
        phases[k] = {"us": 1000.0 * v, "gflop": fl / 1e9, "mb": by / 1e6,
                     "bound": "alu" if t_alu >= t_hbm else "hbm",
                     "frac": (max(t_alu, t_hbm) / s) if s > 0 else None}
    dom = max(ms, key=ms.get)
    fl, by = work[dom]
    s = ms[dom] / 1000.0
    if phases[dom]["bound"] == "alu":
        achieved, peak, unit = fl / s / 1e12, alu_tflops, "TFLOP/s"
    else:
        achieved, peak, unit = by / s / 1e9, hbm_gbs, "GB/s"
    line["roofline"] = {"kernel": dom, "bound": phases[dom]["bound"], "achieved": achieved,
                        "peak": peak, "unit": unit, "frac": achieved / peak,
                        "traffic": load_traffic(dom),
                        "peak_source": (f"{peak_src} HBM copy {hbm_gbs} GB/s; FP32 FMA peak = "
                                        f"152 SMs x 128 lanes x 2 x {sm_max_mhz:.0f} MHz"),
                        "algorithmic_per_launch": {"flops": fl, "bytes": by},
                        "profiled_iters": prof_iters}
    if unit == "TFLOP/s":
        sg = sgemm_tflops()
        line["roofline"]["measured_fp32"] = {
            "sgemm_tflops": sg, "frac": achieved / sg if sg else None,
            "what": "cuBLAS FP32 SGEMM 8192^3 (TF32 off), CUDA events, on this GPU"}
    # The X-streaming products against HBM (the metric's roofline).
    xbytes = {k: work[k][1] for k in ("wtx", "xht")}
    line["x_products_hbm"] = {k: {"gbs": xbytes[k] / (ms[k] / 1000.0) / 1e9,
                                  "frac_of_hbm": xbytes[k] / (ms[k] / 1000.0) / 1e9 / hbm_gbs}
                              for k in xbytes}
    # Whole-iteration roofline: the slower of the X bytes at HBM bandwidth and
    # all flops at the FP32 peak, against the measured step time.
    it_bytes = 2 * 4 * P.m * P.n
    it_flops = sum(w[0] for w in work.values())
    bound_s = max(it_bytes / (hbm_gbs * 1e9), it_flops / (alu_tflops * 1e12))
    line["iteration_roofline"] = {"bound_us": bound_s * 1e6, "frac": bound_s / (t / args.steps),
                                  "x_bytes": it_bytes, "flops": it_flops}
    line["phases"] = phases

    # The tensor-core precision modes on the same workload (X products on
    # tcgen05 from a packed copy of X): iteration rate, the X products
    # against HBM, and the relative error beside the FP32 run's.
    modes = {}
    Wf, Hf = solver.factors()
    fp32_direct = direct_relerr(Xd, Wf, Hf)
    line["relerr_direct"] = fp32_direct
    # Same final error: every mode (FP32 included) runs from the same start
    # until its returned factors reach 1.001 x the FP32 path's direct error
    # after 500 iterations.
    ref = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream)
    ref.step(500)
    Wr, Hr = ref.factors()
    same_target = 1.001 * direct_relerr(Xd, Wr, Hr)
    ref.close()
    same = {"target_relerr_direct": same_target,
            "definition": "1.001 x the FP32 path's direct relerr after 500 iterations"}
    for name, prec in (("fp32", nmf.NMF_PREC_FP32), ("tf32", nmf.NMF_PREC_TF32),
                       ("bf16x3", nmf.NMF_PREC_BF16X3)):
        sv = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream, precision=prec)
        same[name] = time_to_direct(sv, Xd, same_target, stream)
        same[name]["restarts"] = restarts(sv)
        sv.close()
    modes["same_final_error"] = same
    for name, prec in (("tf32", nmf.NMF_PREC_TF32), ("bf16x3", nmf.NMF_PREC_BF16X3)):
        sv = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream, precision=prec)
        sv.step(args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        sv.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        tm = e0.elapsed_time(e1) / 1000.0
        pm = sv.profile_phases(prof_iters)
        Wm, Hm = sv.factors()
        modes[name] = {
            "iters_per_s": args.steps / tm, "ms_per_step": 1000.0 * tm / args.steps,
            "relerr_direct": direct_relerr(Xd, Wm, Hm), "fp32_relerr_direct": fp32_direct,
            "relerr_from_e_k": sv.info().relerr, "restarts": restarts(sv),
            "fp32_restarts": restarts(solver),
            "x_products_hbm": {k: {"us": 1000.0 * pm[k],
                                   "gbs": xbytes[k] / (pm[k] / 1000.0) / 1e9,
                                   "frac_of_hbm": xbytes[k] / (pm[k] / 1000.0) / 1e9 / hbm_gbs}
                               for k in xbytes}}
        sv.close()
    line["precision_modes"] = modes

    # End to end through the public API from pinned host buffers: create
    # (X, W0, H0 uploaded), `steps` iterations, factors read back.
    Xh = torch.from_numpy(P.X).pin_memory()
    W0h = torch.from_numpy(P.W0).pin_memory()
    H0h = torch.from_numpy(P.H0).pin_memory()
    Wout = torch.empty((P.m, P.r), dtype=torch.float32).pin_memory()
    Hout = torch.empty((P.r, P.n), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s2 = nmf.Solver(Xh, P.r, W0h, H0h, stream=stream)
    s2.step(args.steps)
    nmf.nmf_get_factors(s2.h, Wout, Hout)
    inf2 = s2.info()
    t_e2e = time.perf_counter() - t0
    s2.close()
    h2d = 4 * (P.m * P.n + P.m * P.r + P.r * P.n)
    d2h = 4 * (P.m * P.r + P.r * P.n) + 128
    line["e2e"] = {"value": args.steps / t_e2e, "unit": UNIT,
                   "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                   "seconds": t_e2e, "relerr": inf2.relerr,
                   "includes": "nmf_create (upload, validation, ||X||^2, e(0), graph capture), "
                               "nmf_step x steps, nmf_get_factors, nmf_get_info"}

    # Time to a target relative error: E-A-HALS vs un-extrapolated A-HALS,
    # both judged on the error of the pair (W, H) they return
    # (nmf_eval_error, checked every 10 iterations inside nmf_solve; the
    # checks' cost is inside the time).
    ref = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream)
    ref.step(500)
    target = 1.001 * ref.eval_error()[1]
    ref.close()
    ttt = {"target_relerr": target,
           "definition": "1.001 x the relative error of E-A-HALS's returned pair after 500 "
                         "iterations; nmf_solve checks the returned pair's error every 10"}
    for name, kw in (("eahals", {}), ("ahals", {"beta0": 0.0})):
        sv = nmf.Solver(Xd, P.r, W0d, H0d, stream=stream, **kw)
        torch.cuda.synchronize()
        res = sv.solve(5000, target_relerr=target, check_every=10)
        ttt[name] = {"seconds": res.seconds, "iters": res.iters, "reached": bool(res.reached),
                     "relerr": res.relerr, "relerr_last": res.relerr_last}
        sv.close()
    line["time_to_relerr"] = ttt
    solver.close()

    if not args.no_workloads:
        line["workloads"] = other_workloads(nmf, torch, stream)

    if world == 1 and not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        v1, dt1 = cpu_baseline_oracle(P, lw, lh, 2, 1)
        vn, dtn = cpu_baseline_oracle(P, lw, lh, 8, ncores)
        model = cpu_model()
        line["cpu_baseline"] = {
            "value": vn, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "cpu_model": model, "nproc": ncores,
            "sample": f"8 outer iterations of {WORKLOAD}, FP64 oracle on all {ncores} host "
                      f"cores (OpenMP over independent columns / rows), {dtn:.1f} s",
            "one_thread": {"value": v1, "unit": UNIT, "cores": 1,
                           "sample": f"2 outer iterations, one thread, {dt1:.1f} s"}}
    return line


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_ours(args, world, rank, local)
    if line is not None and rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
