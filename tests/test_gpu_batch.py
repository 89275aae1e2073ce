"""Batched solver: many uneven instances in one CUDA graph per iteration.

Every instance runs the same kernels, with the same tiles, splits and CTAs,
as a single-instance solver -- grouped into one launch per phase and kernel
variant, or as per-instance chains on concurrent branches -- so results are
compared bit for bit with nmf_create/nmf_step (which the parity tests check
against the oracle), and the per-instance launch loop must give identical
results too."""
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
    """An instance run inside a batch (grouped launches, beside five uneven
    instances) for K = 800 iterations on noisy low-rank X: the relative
    error of its returned pair matches the FP64 oracle's within 1e-4
    relative -- the K-iteration gate of the single solver, on the same
    problem."""
    from gpu_helpers import oracle_X, oracle_params, f32
    P = wl.low_rank(300, 200, 8, seed=11, noise=0.05)
    others = _problems(5, seed=3)
    K = 800
    p = oracle_params(P)
    Xo = oracle_X(P)
    st = O.eahals_init(Xo, f32(P.W0), f32(P.H0), p)
    O.eahals_run(Xo, st, p, K)
    rel_o = np.linalg.norm(Xo - st.W @ st.H) / np.linalg.norm(Xo)
    with nmf.Batch([(Q.X, Q.r, Q.W0, Q.H0) for Q in others[:2]] + [(P.X, P.r, P.W0, P.H0)] +
                   [(Q.X, Q.r, Q.W0, Q.H0) for Q in others[2:]]) as b:
        b.set_plan(1, 4, 0)
        b.step(K)
        info = b.info(2)
        assert info.device_status == 0 and info.k == K
        W, H = b.factors(2)
    rel_g = np.linalg.norm(Xo - W.astype(np.float64) @ H) / np.linalg.norm(Xo)
    assert abs(rel_g - rel_o) <= 1e-4 * rel_o, (rel_g, rel_o)


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


def _mixed_problems():
    """Instances of every variant class the grouped launches key on: r from
    1 to 40 (one to five 8-wide column groups, lane slot counts 2..20), a
    tall instance whose products split their reduction, ragged m and n."""
    out = _problems(14, seed=11, mn=(40, 600))
    out.append(wl.low_rank(3100, 260, 40, seed=12, noise=0.01))
    out.append(wl.low_rank(300, 2900, 13, seed=13, noise=0.01))
    out.append(wl.low_rank(90, 70, 1, seed=14, noise=0.01))
    return out


@pytest.mark.parametrize("grouped,branches,cols", [(1, 1, 32), (1, 16, 16), (1, 4, 7),
                                                   (0, 4, 0)])
def test_every_plan_matches_single_solvers(grouped, branches, cols):
    """Grouped launches (one per phase and kernel variant over all instances)
    and per-instance chains: each instance bit-identical to its single
    solver after K iterations, whatever the schedule."""
    probs = _mixed_problems()
    K = 9
    with nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs]) as b:
        b.set_plan(grouped, branches, cols)
        pl = b.plan()
        assert pl.grouped == grouped and pl.branches == branches
        if grouped:
            assert pl.launches_per_iter < 9 * len(probs) // 2, pl.launches_per_iter
        else:
            assert pl.launches_per_iter == 9 * len(probs)
        b.step(K)
        for i, P in enumerate(probs):
            W, H = b.factors(i)
            with nmf.Solver(P.X, P.r, P.W0, P.H0) as s:
                s.step(K)
                Ws, Hs = s.factors()
                np.testing.assert_array_equal(W, Ws, err_msg=f"instance {i}")
                np.testing.assert_array_equal(H, Hs, err_msg=f"instance {i}")
                bi, si = b.info(i), s.info()
                assert bi.e_last == si.e_last and bi.beta == si.beta and bi.k == K
                assert bi.device_status == 0


def test_grouped_plan_with_per_instance_parameters():
    """The parameter-study form (same X, hp and the beta schedule varying per
    instance) under grouped launches equals single solvers bit for bit."""
    from paper_1805_06604_gb300 import sweep
    P = wl.low_rank(150, 110, 9, seed=15)
    vs = sweep.variants(hp=(1, 2, 3), beta0=(0.25, 0.75), eta=(1.5,), gammas=((1.05, 1.01),))
    K = 12
    with nmf.Batch([(P.X, P.r, P.W0, P.H0)] * len(vs), per_instance=[ov for _, _, ov in vs]) as b:
        b.set_plan(1, 8, 0)
        b.step(K)
        for i, (_, _, ov) in enumerate(vs):
            W, H = b.factors(i)
            with nmf.Solver(P.X, P.r, P.W0, P.H0, **ov) as s:
                s.step(K)
                Ws, Hs = s.factors()
                np.testing.assert_array_equal(W, Ws)
                np.testing.assert_array_equal(H, Hs)


def test_plan_is_validated():
    """Out-of-range fields give NMF_EINVAL; grouped launches for a batch with
    a tensor-core instance give NMF_ENOTSUP, and the batch keeps working with
    its tuned schedule."""
    probs = _problems(3, seed=16)
    with nmf.Batch([(P.X, P.r, P.W0, P.H0) for P in probs],
                   per_instance=[{}, {"precision": nmf.NMF_PREC_TF32}, {}]) as b:
        before = b.plan()
        assert before.grouped == 0
        for bad in [(2, 1, 0), (1, 0, 0), (0, 65, 0), (1, 1, 33), (1, 1, -1)]:
            with pytest.raises(nmf.NmfError) as ei:
                b.set_plan(*bad)
            assert ei.value.status == nmf.NMF_EINVAL
        with pytest.raises(nmf.NmfError) as ei:
            b.set_plan(1, 1, 0)
        assert ei.value.status == nmf.NMF_ENOTSUP
        b.step(3)
        assert all(b.info(i).k == 3 and b.info(i).device_status == 0 for i in range(3))
