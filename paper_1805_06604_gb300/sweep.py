"""The paper's parameter study (Sec. 4.2, "Tuning parameters") on the GPU.

E-A-HALS runs for every combination of hp in {1, 2, 3}, beta0 in {0.25,
0.5, 0.75}, eta in {1.5, 2, 3} and (gamma, gamma_bar) in {(1.01, 1.005),
(1.05, 1.01), (1.1, 1.05), (1.005, 1.001)} -- the values Sec. 4.2 lists,
with the extra pair it adds for A-HALS -- plus the original A-HALS
(beta0 = 0), on the synthetic data of Sec. 4.1 (m = n = 200, r = 20).  All
variants of one data set and one initialisation are solved together: one
batched graph (nmf_batch_create_params) whose instances share X, W0 and H0
and differ only in their parameters.

Reported per variant: the error measure E(K) = relerr - e_min of Sec. 4.2
(e_min = 0 for the exactly low-rank data, otherwise the lowest relative
error reached by any variant from any initialisation of that data set),
averaged over the data sets and initialisations, with its standard
deviation; for each hp the best and the worst parameter set by mean E (the
two curves per hp that the paper's figures show); and, as in Tables 3-6,
how often each of those and A-HALS produced the i-th best solution.

    python -m paper_1805_06604_gb300.sweep --data low_rank --datasets 2 --inits 2 --iters 500

The relative errors are evaluated directly in FP64 from the returned
factors.  Only the GPU solve runs through the library; everything here is
bookkeeping.
"""
from __future__ import annotations

import argparse
import itertools
import json
import time

import numpy as np

HP = (1, 2, 3)
BETA0 = (0.25, 0.5, 0.75)
ETA = (1.5, 2.0, 3.0)
GAMMAS = ((1.01, 1.005), (1.05, 1.01), (1.1, 1.05), (1.005, 1.001))
AHALS = "A-HALS"


def variant_name(hp, beta0, eta, gamma, gamma_bar) -> str:
    return f"hp={hp} beta0={beta0} eta={eta} gamma={gamma} gamma_bar={gamma_bar}"


def variants(hp=HP, beta0=BETA0, eta=ETA, gammas=GAMMAS):
    """(name, hp, parameter overrides) for the grid, A-HALS first."""
    out = [(AHALS, 0, {"beta0": 0.0})]
    for h, b, e, (g, gb) in itertools.product(hp, beta0, eta, gammas):
        out.append((variant_name(h, b, e, g, gb), h,
                    {"hp": h, "beta0": b, "eta": e, "gamma": g, "gamma_bar": gb}))
    return out


def summarize(relerr: dict, hp_of: dict, exact_low_rank: bool) -> dict:
    """relerr[(dataset, init)][variant] -> relative error after K iterations.

    e_min per data set: 0 for exactly low-rank X (Sec. 4.2), else the lowest
    relative error over every variant and initialisation of that data set.
    Returns per-variant mean / std of E, the best and worst variant of each
    hp (by mean E), and the rank histogram of A-HALS and those variants
    over the runs (entry i: how often the variant had the (i+1)-th smallest
    E among them; ties share the better rank)."""
    runs = sorted(relerr)
    names = sorted({v for r in runs for v in relerr[r]})
    datasets = sorted({d for d, _ in runs})
    e_min = {}
    for d in datasets:
        e_min[d] = 0.0 if exact_low_rank else min(
            relerr[r][v] for r in runs if r[0] == d for v in relerr[r])
    E = {v: np.array([relerr[r][v] - e_min[r[0]] for r in runs]) for v in names}
    per = {v: {"mean_E": float(E[v].mean()), "std_E": float(E[v].std()), "hp": hp_of[v]}
           for v in names}
    best, worst = {}, {}
    for h in sorted({hp_of[v] for v in names if hp_of[v] > 0}):
        cand = [v for v in names if hp_of[v] == h]
        best[h] = min(cand, key=lambda v: (per[v]["mean_E"], v))
        worst[h] = max(cand, key=lambda v: (per[v]["mean_E"], v))
    shown = [AHALS] if AHALS in names else []
    for h in sorted(best):
        for v in (best[h], worst[h]):
            if v not in shown:
                shown.append(v)
    ranks = {v: [0] * len(shown) for v in shown}
    for i in range(len(runs)):
        vals = {v: E[v][i] for v in shown}
        for v in shown:
            ranks[v][sum(1 for u in shown if vals[u] < vals[v])] += 1
    return {"e_min": {str(d): e_min[d] for d in datasets}, "per_variant": per,
            "best": {str(h): best[h] for h in best}, "worst": {str(h): worst[h] for h in worst},
            "ranking": ranks, "runs": len(runs)}


def make_data(kind: str, dataset: int, m: int, n: int, r: int):
    from . import workloads as wl
    if kind == "low_rank":
        return wl.low_rank(m, n, r, seed=1000 + dataset).X
    if kind == "full_rank":
        return wl.full_rank(m, n, r, seed=1000 + dataset).X
    raise ValueError(kind)


def run(kind="low_rank", datasets=2, inits=2, iters=500, m=200, n=200, r=20, grid=None):
    """Runs the study on cuda:0; returns (summary, relerr table, seconds)."""
    from . import nmf
    from . import workloads as wl
    nmf.load()
    vs = variants(**(grid or {}))
    hp_of = {name: h for name, h, _ in vs}
    table = {}
    t0 = time.perf_counter()
    for d in range(datasets):
        X = make_data(kind, d, m, n, r)
        Xd = X.astype(np.float64)
        nx = np.linalg.norm(Xd)
        for i in range(inits):
            W0, H0 = wl.init_factors(m, n, r, seed=5000 + 97 * d + i)
            b = nmf.Batch([(X, r, W0, H0)] * len(vs), per_instance=[ov for _, _, ov in vs])
            b.step(iters)
            row = {}
            for j, (name, _, _) in enumerate(vs):
                W, H = b.factors(j)
                row[name] = float(np.linalg.norm(Xd - W.astype(np.float64) @ H) / nx)
            b.close()
            table[(d, i)] = row
    secs = time.perf_counter() - t0
    return summarize(table, hp_of, kind == "low_rank"), table, secs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", choices=["low_rank", "full_rank"], default="low_rank")
    ap.add_argument("--datasets", type=int, default=2)
    ap.add_argument("--inits", type=int, default=2)
    ap.add_argument("--iters", type=int, default=500)
    args = ap.parse_args(argv)
    summ, _, secs = run(args.data, args.datasets, args.inits, args.iters)
    per = summ["per_variant"]
    print(f"# {args.data} 200x200 r=20, {summ['runs']} runs x {len(per)} variants, "
          f"{args.iters} iterations, {secs:.1f} s")
    for v in summ["ranking"]:
        print(f"{v:60s} E {per[v]['mean_E']:.3e} +- {per[v]['std_E']:.1e}  ranks {summ['ranking'][v]}")
    print(json.dumps({"data": args.data, "iters": args.iters, "seconds": secs, **summ}))


if __name__ == "__main__":
    main()
