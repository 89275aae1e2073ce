"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (the same library, graph and kernels).

* Dense noisy 10000 x 4000, r = 50 and image-like 10304 x 4000, r = 64:
  one full step from an identical mid-run state, every output element
  compared with the FP64 oracle (one oracle step takes seconds here).
* Properties that hold at any size, on 60 GPU iterations of the dense
  workload: accepted errors never increase, H_y >= 0 for hp = 3, and the
  tracked error equals ||X - W H_y|| computed directly for the last accepted
  iterate.
"""
import numpy as np
import pytest

import oracle as O
from paper_1805_06604_gb300 import nmf
from paper_1805_06604_gb300 import workloads as wl

from gpu_helpers import make_solver, normwise, oracle_params, single_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1805_06604_gb300 import build
    build.build()
    O.build()
    nmf.load()


@pytest.fixture(scope="module")
def dense_noisy():
    return wl.dense_noisy(0)


def _assert_step(res):
    g, o = res["gpu"], res["orc"]
    assert g["acc"] == o["acc"]
    for name in ("W", "H", "Wy", "Hy"):
        err = normwise(g[name], o[name])
        assert err <= res["tol"], f"{name}: {err:.3e} > {res['tol']:.2e} (kappa {res['kappa']:.0f})"
    assert abs(g["e"] ** 2 - o["e"] ** 2) <= 2e-6 * res["fro2"]


def test_full_size_dense_single_step(dense_noisy):
    P = dense_noisy
    _assert_step(single_step(P, oracle_params(P), warm=1))


def test_full_size_image_like_single_step():
    P = wl.image_like(0)
    _assert_step(single_step(P, oracle_params(P), warm=1))


def test_full_size_properties(dense_noisy):
    P = dense_noisy
    p = oracle_params(P)
    with make_solver(P, p) as s:
        e0 = s.info().e_last
        s.step(60)
        te, tb, ta = s.trace()
        info = s.info()
        W, H = s.factors()
        Wy, Hy = s.extrapolated()
    acc = np.concatenate([[e0], te[ta]])
    assert np.all(np.diff(acc) <= 0.0)
    assert np.all(Hy >= 0.0)
    assert (~ta).sum() < 30
    assert info.relerr < 1e-2 and te[ta][-1] < 0.2 * e0
    if ta[-1]:
        # after an accepted step H_y is the H the W-update used, so e(k) is
        # ||X - W H_y|| (Algorithm 2 step 15)
        X = P.X.astype(np.float64)
        direct = np.linalg.norm(X - W.astype(np.float64) @ Hy.astype(np.float64))
        assert direct == pytest.approx(info.e_last, rel=1e-3)
