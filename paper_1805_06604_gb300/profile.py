"""Per-phase device time of E-A-HALS outer iterations on a synthetic workload.

    python -m paper_1805_06604_gb300.profile --workload dense_noisy --iters 2

Creates a solver on cuda:0 for the workload, runs `--warm` graphed
iterations, then `--iters` ungraphed iterations through nmf_profile_phases
(a CUDA event between consecutive phases on the solver's stream) and prints
the mean microseconds of every phase.  Under a profiler, the ungraphed
iterations launch each kernel of the path once per iteration.
"""
from __future__ import annotations

import argparse
import json

from . import nmf
from . import workloads as wl

WORKLOADS = {
    "dense_noisy": lambda: wl.dense_noisy(0),
    "image_like": lambda: wl.image_like(0),
    "document_like": lambda: wl.document_like(0),
    "oracle_scale": lambda: wl.oracle_scale(0),
}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dense_noisy")
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--warm", type=int, default=0)
    ap.add_argument("--precision", choices=["fp32", "tf32", "bf16x3"], default="fp32")
    ap.add_argument("--batch", type=int, default=0,
                    help="time COUNT uneven instances (m, n ~ U{64..2048}, r ~ U{4..32}): "
                         "batched graph vs per-instance launch loop")
    ap.add_argument("--plan", default="",
                    help="with --batch: GROUPED,BRANCHES,COLS -- set this schedule and run "
                         "--iters iterations only (for a profiler's launch list)")
    args = ap.parse_args(argv)
    if args.batch:
        return batch_main(args)
    import numpy as np
    import torch
    nmf.load()
    P = WORKLOADS[args.workload]()
    st = torch.cuda.current_stream()
    prec = {"fp32": nmf.NMF_PREC_FP32, "tf32": nmf.NMF_PREC_TF32,
            "bf16x3": nmf.NMF_PREC_BF16X3}[args.precision]
    if P.is_csr:
        s = nmf.Solver(None, P.r, P.W0.astype(np.float32), P.H0.astype(np.float32),
                       csr=(P.rowptr, P.colidx, P.val.astype(np.float32)), m=P.m, n=P.n,
                       stream=st)
    else:
        X = torch.from_numpy(P.X.astype(np.float32)).cuda()
        s = nmf.Solver(X, P.r, torch.from_numpy(P.W0.astype(np.float32)).cuda(),
                       torch.from_numpy(P.H0.astype(np.float32)).cuda(), stream=st,
                       precision=prec)
    if args.warm:
        s.step(args.warm)
    ms = s.profile_phases(args.iters)
    info = s.info()
    s.close()
    print(json.dumps({"workload": P.name, "precision": args.precision, "lw": info.lw,
                      "lh": info.lh, "device_status": info.device_status,
                      "phase_us": {k: round(v * 1000.0, 2) for k, v in ms.items()},
                      "iteration_us": round(sum(ms.values()) * 1000.0, 2)}))


def batch_main(args):
    import time
    import torch
    nmf.load()
    probs = wl.batch(count=args.batch, seed=0)
    t0 = time.perf_counter()
    b = nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs])
    t_create = time.perf_counter() - t0
    if args.plan:
        g, br, cols = (int(v) for v in args.plan.split(","))
        b.set_plan(g, br, cols)
        b.step(max(args.iters, 1))
        torch.cuda.synchronize()
        pl = b.plan()
        b.close()
        print(json.dumps({"instances": args.batch, "grouped": pl.grouped, "branches": pl.branches,
                          "h_cols": pl.h_cols_per_cta, "launches_per_iter": pl.launches_per_iter,
                          "iters": max(args.iters, 1)}))
        return
    branches, tuned = b.schedule()
    K = max(args.iters, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, fn in (("graph", b.step), ("loop", b.step_loop)):
        fn(1)
        torch.cuda.synchronize()
        e0.record()
        fn(K)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / K
    pl = b.plan()
    chosen = {"grouped": pl.grouped, "branches": pl.branches, "h_cols": pl.h_cols_per_cta,
              "launches_per_iter": pl.launches_per_iter}
    # Every schedule the tuner considers, timed the same way.
    plans = {}
    for g, br, cols in ((0, 64, 0), (0, 16, 0), (1, 1, 32), (1, 16, 32), (1, 1, 16),
                        (1, 16, 16), (1, 16, 8)):
        b.set_plan(g, br, cols)
        b.step(1)
        torch.cuda.synchronize()
        e0.record()
        b.step(K)
        e1.record()
        torch.cuda.synchronize()
        plans[f"{'grouped' if g else 'chains'}_b{br}_c{cols}"] = round(e0.elapsed_time(e1) / K, 3)
    flops = sum(4.0 * P.m * P.n * P.r for P in probs)
    b.close()
    print(json.dumps({"instances": args.batch, "sum_mn": int(sum(P.m * P.n for P in probs)),
                      "plan": chosen, "plans_ms_per_iter": plans,
                      "branches": branches, "autotune_ms_per_iter": round(tuned, 3),
                      "create_s": round(t_create, 2), "iters": K,
                      "graph_ms_per_iter": round(res["graph"], 3),
                      "loop_ms_per_iter": round(res["loop"], 3),
                      "speedup": round(res["loop"] / res["graph"], 2),
                      "product_gflop_per_iter": round(flops / 1e9, 2)}))


if __name__ == "__main__":
    main()
