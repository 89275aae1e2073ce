"""Writes the stored oracle runs at the benchmark workloads' full sizes
(tests/golden/fullsize_*.json), used by tests/test_gpu_fullsize_k.py.

It calls only the FP64 oracle (oracle/) and the seeded input generators
(paper_1805_06604_gb300/workloads.py, which draw data and hold none of the
method's arithmetic).  For each workload it runs Algorithm 2 with
Algorithm 3 and the A-HALS sweep budget from the float32 inputs the GPU
path sees (widened to float64), and stores the e(k) trace, the beta_k used,
the accept/restart decisions and the relative error ||X - WH||_F / ||X||_F
of the returned pair, evaluated entry by entry.

    python tests/golden/make_fullsize.py [names...]

Runs take minutes per workload (OpenMP over the host cores).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1805_06604_gb300 import workloads as wl  # noqa: E402


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def problem(name: str):
    if name.startswith("dense_noisy"):
        return wl.dense_noisy(0)
    if name.startswith("image_like"):
        return wl.image_like(0)
    if name.startswith("document_like"):
        return wl.document_like(0)
    raise KeyError(name)


# (file tag, workload, iterations, beta0): the dense noisy workload runs
# E-A-HALS and un-extrapolated A-HALS (beta0 = 0), as the benchmark compares.
RUNS = [
    ("dense_noisy_10000x4000_r50_eahals", "dense_noisy", 500, 0.5),
    ("dense_noisy_10000x4000_r50_ahals", "dense_noisy", 500, 0.0),
    ("image_like_10304x4000_r64_eahals", "image_like", 200, 0.5),
    ("document_like_50000x20000_r30_eahals", "document_like", 300, 0.5),
]


def run(tag: str, kind: str, iters: int, beta0: float) -> dict:
    P = problem(kind)
    lw, lh = O.sweep_counts(P.m, P.n, P.nnz, P.r)
    p = O.Params(hp=3, beta0=beta0, lw=lw, lh=lh)
    W0 = P.W0.astype(np.float32)
    H0 = P.H0.astype(np.float32)
    if P.is_csr:
        val = P.val.astype(np.float32)
        X = O.Matrix(m=P.m, n=P.n, rowptr=P.rowptr, colidx=P.colidx, val=val.astype(np.float64))
        xdig = digest(P.rowptr, P.colidx, val)
    else:
        Xf = P.X.astype(np.float32)
        X = O.Matrix(Xf.astype(np.float64))
        xdig = digest(Xf)
    t0 = time.time()
    st = O.eahals_init(X, W0, H0, p)
    e0 = st.s.e_last
    te, tb, ta = O.eahals_run(X, st, p, iters)
    fro2 = O.fro2(X)
    rel = float(np.sqrt(O.err2_direct(X, st.W, st.H) / fro2))
    secs = time.time() - t0
    # Samples of the returned factors (32 evenly spaced rows of W and columns
    # of H, and (W H)_ij on the 32 x 32 grid of those), for the precision
    # study's factor comparison; 9 significant digits.
    rows = np.linspace(0, P.m - 1, 32).astype(np.int64)
    cols = np.linspace(0, P.n - 1, 32).astype(np.int64)

    def r9(a):
        return [[float(f"{v:.9g}") for v in row] for row in np.atleast_2d(a)]

    samples = {"rows": rows.tolist(), "cols": cols.tolist(),
               "W_rows": r9(st.W[rows]), "H_cols": r9(st.H[:, cols]),
               "WH": r9(st.W[rows] @ st.H[:, cols])}
    return {
        "tag": tag, "workload": P.name, "m": P.m, "n": P.n, "r": P.r, "nnz": int(P.nnz),
        "params": {"hp": 3, "beta0": beta0, "eta": 1.5, "gamma": 1.01, "gamma_bar": 1.005,
                   "lw": lw, "lh": lh, "compare_prev": 1},
        "iters": iters, "inputs_sha256": xdig, "factors_sha256": digest(W0, H0),
        "fro2": fro2, "e0": e0, "relerr_direct": rel,
        "e": [float(f"{v:.15g}") for v in te], "beta": [float(f"{v:.15g}") for v in tb],
        "accepted": [int(v) for v in ta],
        "restarts": int((~ta).sum()), "samples": samples,
        "oracle_seconds": secs, "oracle_threads": O.get_threads(),
        "written_by": "tests/golden/make_fullsize.py (FP64 oracle)",
    }


def main(argv):
    want = set(argv[1:])
    for tag, kind, iters, beta0 in RUNS:
        if want and tag not in want:
            continue
        res = run(tag, kind, iters, beta0)
        path = os.path.join(HERE, f"fullsize_{tag}.json")
        with open(path, "w") as f:
            json.dump(res, f)
        print(f"{tag}: relerr {res['relerr_direct']:.9e}, restarts {res['restarts']}, "
              f"{res['oracle_seconds']:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv)
