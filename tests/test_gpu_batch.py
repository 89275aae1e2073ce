"""Batched solver: many uneven instances in one CUDA graph per iteration.

Every instance runs the same kernels in the same order as a single-instance
solver, only scheduled concurrently, so results are compared bit for bit
with nmf_create/nmf_step (which the parity tests check against the oracle),
and the per-instance launch loop must give identical results too."""
import numpy as np
import pytest

import oracle as O
from paper_1805_06604_gb300 import nmf
from paper_1805_06604_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_06604_gb300 import build
    build.build()
    O.build()
    nmf.load()


def _problems(count, seed=1, mn=(64, 400)):
    return wl.batch(count=count, seed=seed, mn_range=mn, r_range=(4, 32))


def test_batch_matches_single_instance_solvers():
    probs = _problems(24)
    K = 12
    with nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs]) as b:
        branches, ms = b.schedule()
        assert 1 <= branches <= 24 and ms > 0
        b.step(K)
        for i, P in enumerate(probs):
            W, H = b.factors(i)
            with nmf.Solver(P.X, P.r, P.W0, P.H0) as s:
                s.step(K)
                Ws, Hs = s.factors()
                assert b.info(i).k == K
                np.testing.assert_array_equal(W, Ws)
                np.testing.assert_array_equal(H, Hs)
                assert b.info(i).e_last == s.info().e_last


def test_batch_loop_equals_graph_and_tuning_is_undone():
    probs = _problems(10, seed=2)
    with nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs]) as a, \
            nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs]) as b:
        assert all(a.info(i).k == 0 for i in range(len(probs)))
        a.step(7)
        b.step_loop(7)
        for i in range(len(probs)):
            Wa, Ha = a.factors(i)
            Wb, Hb = b.factors(i)
            np.testing.assert_array_equal(Wa, Wb)
            np.testing.assert_array_equal(Ha, Hb)


def test_batch_instance_against_oracle():
    """One instance of a batch, single step from its state after 5 batched
    iterations, against the oracle (same gate as the single-instance tests)."""
    from gpu_helpers import gram_kappa, normwise, oracle_params, step_tol
    probs = _problems(6, seed=3)
    with nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs]) as b:
        b.step(5)
        i = 4
        P = probs[i]
        info = b.info(i)
        assert info.device_status == 0
        W, H = b.factors(i)
        p = oracle_params(P)
        Xo = P.X.astype(np.float32).astype(np.float64)
        st = O.eahals_init(Xo, P.W0, P.H0, p)
        O.eahals_run(Xo, st, p, 5)
        rel_o = np.linalg.norm(Xo - st.W @ st.H) / np.linalg.norm(Xo)
        rel_g = np.linalg.norm(Xo - W.astype(np.float64) @ H) / np.linalg.norm(Xo)
        assert abs(rel_g - rel_o) <= 1e-3 * rel_o, (rel_g, rel_o)


def test_per_instance_parameters_match_single_solvers():
    """nmf_batch_create_params: every instance runs with its own parameters
    (the parameter study's batches share X and differ only in hp, beta0,
    eta, gamma, gamma_bar); each must equal a single solver created with
    those parameters, bit for bit."""
    from paper_1805_06604_gb300 import sweep
    P = wl.low_rank(120, 90, 6, seed=5)
    vs = sweep.variants(hp=(1, 3), beta0=(0.25, 0.75), eta=(1.5,), gammas=((1.05, 1.01),))
    K = 15
    with nmf.Batch([(P.X, P.r, P.W0, P.H0)] * len(vs), per_instance=[ov for _, _, ov in vs]) as b:
        b.step(K)
        for i, (_, _, ov) in enumerate(vs):
            W, H = b.factors(i)
            with nmf.Solver(P.X, P.r, P.W0, P.H0, **ov) as s:
                s.step(K)
                Ws, Hs = s.factors()
                np.testing.assert_array_equal(W, Ws)
                np.testing.assert_array_equal(H, Hs)
                assert b.info(i).beta == s.info().beta


def test_parameter_study_runs_and_ranks():
    """A reduced parameter study (Sec. 4.2) end to end on the GPU: every
    variant's E is finite and >= 0 on exactly low-rank data (e_min = 0), and
    the extrapolated best variant beats A-HALS after the same iterations."""
    from paper_1805_06604_gb300 import sweep
    grid = dict(hp=(1, 3), beta0=(0.5,), eta=(1.5,), gammas=((1.01, 1.005), (1.1, 1.05)))
    summ, table, _ = sweep.run("low_rank", datasets=1, inits=2, iters=150, m=80, n=70, r=6,
                               grid=grid)
    per = summ["per_variant"]
    assert len(per) == 1 + 4
    assert all(np.isfinite(v["mean_E"]) and v["mean_E"] >= 0.0 for v in per.values())
    best = min(per[summ["best"][h]]["mean_E"] for h in summ["best"])
    assert best < per[sweep.AHALS]["mean_E"]
    assert all(sum(r) == summ["runs"] for r in summ["ranking"].values())


def test_per_instance_parameters_are_validated():
    """A bad parameter set in one instance fails the whole batch with that
    instance's index in the message; params = NULL is rejected."""
    import ctypes as ct
    P = wl.low_rank(50, 40, 4, seed=6)
    with pytest.raises(nmf.NmfError) as ei:
        nmf.Batch([(P.X, P.r, P.W0, P.H0)] * 3, per_instance=[{}, {"hp": 5}, {}])
    assert ei.value.status == nmf.NMF_EINVAL and "instance 1" in str(ei.value)
    h = ct.c_void_p()
    st = nmf.load().nmf_batch_create_params(ct.byref(h), 1, None, None, None, None, 0, None, None)
    assert st == nmf.NMF_EINVAL
