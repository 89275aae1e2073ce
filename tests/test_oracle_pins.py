"""Pins for the FP64 oracle: each routine is checked against something other
than itself -- a library routine it reduces to, brute force on tiny inputs, a
closed form, an invariant the paper states, or a hand-derived example.

Which pin covers which oracle routine:
  orc_fro2, orc_wtx, orc_xht, orc_gram_*   numpy / scipy products (library)
  orc_hals_row_h, orc_hals_col_w           1-D brute-force minimisation of the
                                           direct objective (Sec. 1 closed form)
  orc_hals_sweeps_*                        convergence to brute-force NNLS
                                           (all 2^r active sets), monotone decrease
  orc_err2_expanded / orc_err2_direct      Remark 1 identity + numpy direct error
  orc_sweep_counts                         hand-evaluated budgets
  orc_line_search_beta                     vertex of the parabola through three
                                           direct errors (Sec. 3), zero cases,
                                           the step's own W, W_n, H_y
  orc_nnls, orc_nnls_h / _w (E-ANLS)       brute-force NNLS over every free set,
                                           scipy.optimize.nnls, KKT, zero column;
                                           ANLS monotone and exact per column;
                                           E-ANLS beats ANLS on low-rank data
  orc_beta_update                          hand-derived Algorithm 3 sequences
  orc_eahals_*                             hand-worked 2x2 examples (accepted
                                           steps; a restart; hp = 1; hp = 2),
                                           beta0 = 0
                                           reduces to A-HALS, accepted errors
                                           monotone, hp=3 feasibility, exact
                                           power-of-two scaling equivariance,
                                           row / column permutation equivariance,
                                           low-rank recovery, KKT, acceleration
                                           over A-HALS (Table 3's claim)
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1805_06604_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed):
    return wl.rng(seed).random(shape)


def _csr(X):
    rp, ci, v = wl.csr_from_dense(X)
    return O.Matrix(m=X.shape[0], n=X.shape[1], rowptr=rp, colidx=ci, val=v)


def _sparse_dense(m, n, density, seed):
    g = wl.rng(seed)
    X = g.random((m, n)) * (g.random((m, n)) < density)
    X[3, :] = 0.0            # an empty row
    return X


# ---------------------------------------------------------------- products

@pytest.mark.parametrize("m,n,r", [(7, 5, 3), (37, 23, 6), (64, 41, 17)])
def test_products_match_numpy(m, n, r):
    X = _rand((m, n), 1) - 0.3        # X may be negative (X in R^{m x n})
    W = _rand((m, r), 2)
    H = _rand((r, n), 3)
    np.testing.assert_allclose(O.wtx(X, W), W.T @ X, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.xht(X, H), X @ H.T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.gram_w(W), W.T @ W, rtol=1e-13)
    np.testing.assert_allclose(O.gram_h(H), H @ H.T, rtol=1e-13)
    assert O.fro2(X) == pytest.approx(np.linalg.norm(X) ** 2, rel=1e-14)


def test_csr_products_match_scipy():
    X = _sparse_dense(53, 31, 0.1, 4)
    S = sp.csr_matrix(X)
    W = _rand((53, 5), 5)
    H = _rand((5, 31), 6)
    M = _csr(X)
    np.testing.assert_allclose(O.wtx(M, W), (S.T @ W).T, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(O.xht(M, H), S @ H.T, rtol=1e-13, atol=1e-14)
    assert O.fro2(M) == pytest.approx(sp.linalg.norm(S) ** 2, rel=1e-14)
    assert O.err2_direct(M, W, H) == pytest.approx(np.linalg.norm(X - W @ H) ** 2, rel=1e-12)


# ---------------------------------------------------------------- Remark 1

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_expanded_error_equals_direct(seed):
    m, n, r = 31, 19, 4
    X = _rand((m, n), seed) * 3 - 1
    W = _rand((m, r), seed + 10)
    H = _rand((r, n), seed + 20)
    direct = np.linalg.norm(X - W @ H) ** 2            # library, independent
    assert O.err2_direct(X, W, H) == pytest.approx(direct, rel=1e-12)
    C = X @ H.T
    D = H @ H.T
    assert O.err2_expanded(O.fro2(X), W, C, D) == pytest.approx(direct, rel=1e-12)


# ------------------------------------------------------- HALS closed form

def _objective(X, W, H):
    return float(np.sum((X - W @ H) ** 2))


def _argmin_1d(f, hi):
    """Minimise a convex scalar f on [0, hi] by grid + golden section."""
    ts = np.linspace(0.0, hi, 2001)
    vals = np.array([f(t) for t in ts])
    i = int(np.argmin(vals))
    a, b = ts[max(i - 1, 0)], ts[min(i + 1, len(ts) - 1)]
    phi = (np.sqrt(5) - 1) / 2
    for _ in range(200):
        c, d = b - phi * (b - a), a + phi * (b - a)
        if f(c) <= f(d):
            b = d
        else:
            a = c
    return 0.5 * (a + b)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_row_update_is_exact_1d_minimiser(k):
    """Sec. 1: the closed form is argmin over H(k,:) >= 0 of ||X - WH||^2."""
    m, n, r = 9, 6, 3
    X = _rand((m, n), 7) * 2 - 0.5
    W = _rand((m, r), 8)
    H = _rand((r, n), 9)
    Hn = O.hals_row_h(W.T @ X, W.T @ W, H, k)
    assert np.all(Hn[k] >= 0)
    others = [i for i in range(r) if i != k]
    np.testing.assert_array_equal(Hn[others], H[others])
    for j in range(n):
        def f(t, j=j):
            h = H[:, j].copy()
            h[k] = t
            return float(np.sum((X[:, j] - W @ h) ** 2))
        t_star = _argmin_1d(f, 10.0)
        assert Hn[k, j] == pytest.approx(t_star, abs=1e-7)
    assert _objective(X, W, Hn) <= _objective(X, W, H) + 1e-12


@pytest.mark.parametrize("k", [0, 2])
def test_col_update_is_exact_1d_minimiser(k):
    m, n, r = 7, 10, 3
    X = _rand((m, n), 11) * 2 - 0.5
    W = _rand((m, r), 12)
    H = _rand((r, n), 13)
    Wn = O.hals_col_w(X @ H.T, H @ H.T, W, k)
    assert np.all(Wn[:, k] >= 0)
    for i in range(m):
        def f(t, i=i):
            w = W[i].copy()
            w[k] = t
            return float(np.sum((X[i] - w @ H) ** 2))
        assert Wn[i, k] == pytest.approx(_argmin_1d(f, 10.0), abs=1e-7)


def test_zero_denominator_leaves_row_unchanged():
    m, n, r = 6, 5, 3
    X = _rand((m, n), 14)
    W = _rand((m, r), 15)
    W[:, 1] = 0.0
    H = _rand((r, n), 16)
    Hn = O.hals_row_h(W.T @ X, W.T @ W, H, 1)
    np.testing.assert_array_equal(Hn, H)


def _nnls_bruteforce(W, x):
    """Exact min_{h>=0} ||x - W h|| by enumerating every passive set."""
    r = W.shape[1]
    best, best_h = np.inf, None
    for mask in itertools.product([0, 1], repeat=r):
        S = [i for i in range(r) if mask[i]]
        h = np.zeros(r)
        if S:
            sol, *_ = np.linalg.lstsq(W[:, S], x, rcond=None)
            if np.any(sol < 0):
                continue
            h[S] = sol
        v = float(np.sum((x - W @ h) ** 2))
        if v < best:
            best, best_h = v, h
    return best_h


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_sweeps_converge_to_bruteforce_nnls(r):
    m, n = 12, 8
    X = _rand((m, n), 20 + r) * 2 - 0.6
    W = _rand((m, r), 30 + r) + 0.05
    H0 = _rand((r, n), 40 + r)
    H = O.hals_sweeps_h(W.T @ X, W.T @ W, H0, 3000)
    for j in range(n):
        np.testing.assert_allclose(H[:, j], _nnls_bruteforce(W, X[:, j]), atol=1e-9)
    # and the W side through the transposed problem
    Ht = _rand((r, m), 50 + r) + 0.05
    W0 = _rand((n, r), 60 + r)
    Wn = O.hals_sweeps_w(X.T @ Ht.T, Ht @ Ht.T, W0, 3000)
    for i in range(n):
        np.testing.assert_allclose(Wn[i], _nnls_bruteforce(Ht.T, X[:, i]), atol=1e-9)


def test_every_row_update_decreases_objective():
    """HALS is an exact block coordinate descent: no single update can
    increase ||X - WH||^2 (Sec. 1)."""
    m, n, r = 20, 15, 5
    X = _rand((m, n), 70)
    W = _rand((m, r), 71)
    H = _rand((r, n), 72)
    f = _objective(X, W, H)
    for sweep in range(4):
        A, G = W.T @ X, W.T @ W
        for k in range(r):
            H = O.hals_row_h(A, G, H, k)
            f2 = _objective(X, W, H)
            assert f2 <= f * (1 + 1e-14)
            f = f2
        C, D = X @ H.T, H @ H.T
        for k in range(r):
            W = O.hals_col_w(C, D, W, k)
            f2 = _objective(X, W, H)
            assert f2 <= f * (1 + 1e-14)
            f = f2


# -------------------------------------------------------- sweep budget

def test_sweep_counts_hand_evaluated():
    # rho_W = 1 + (K + n r)/(m (r+1)), L = floor(1 + 0.5 rho)
    # 200x150 r=10: rho_W = 1 + 31500/2200 = 15.32 -> 8; rho_H = 1 + 32000/1650 = 20.39 -> 11
    assert O.sweep_counts(200, 150, 200 * 150, 10) == (8, 11)
    # 10000x4000 r=50: rho_W = 79.82 -> 40; rho_H = 199.5 -> 100
    assert O.sweep_counts(10000, 4000, 10000 * 4000, 50) == (40, 100)
    # 10304x4000 r=64: rho_W = 1 + 41472000/669760 = 62.9 -> 32; rho_H = 1 + 41875456/260000 = 162.06 -> 82
    assert O.sweep_counts(10304, 4000, 10304 * 4000, 64) == (32, 82)
    # 50000x20000 r=30, K=3e6: rho_W = 3.32 -> 2; rho_H = 8.26 -> 5
    assert O.sweep_counts(50000, 20000, 3_000_000, 30) == (2, 5)


# -------------------------------------------------------- Algorithm 3

def test_beta_update_hand_derived():
    with open(os.path.join(GOLDEN, "beta_update_alg3.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        pr = case["params"]
        p = O.Params(beta0=pr["beta0"], gamma=pr["gamma"], gamma_bar=pr["gamma_bar"], eta=pr["eta"])
        s = O.Scalars(beta=pr["beta0"], beta_bar=1.0, beta_prev=pr["beta0"])
        for t, d in enumerate(case["decisions"]):
            s = O.beta_update(p, s, bool(d))
            assert s.beta == pytest.approx(case["beta"][t], rel=1e-15)
            assert s.beta_bar == pytest.approx(case["beta_bar"][t], rel=1e-15)
            assert s.beta_prev == pytest.approx(case["beta_prev"][t], rel=1e-15)


def test_beta_zero_stays_zero():
    """beta_k = 0 for all k gives back the original algorithm (Sec. 2)."""
    p = O.Params(beta0=0.0)
    s = O.Scalars(beta=0.0, beta_bar=1.0, beta_prev=0.0)
    for d in [1, 0, 1, 1, 0]:
        s = O.beta_update(p, s, bool(d))
        assert s.beta == 0.0


# -------------------------------------------------------- Algorithm 2

def test_worked_example_2x2_rank1():
    with open(os.path.join(GOLDEN, "worked_example_2x2_r1.json")) as f:
        g = json.load(f)
    pr = g["problem"]
    X = np.array(pr["X"])
    p = O.Params(hp=pr["hp"], beta0=pr["beta0"], eta=pr["eta"], gamma=pr["gamma"],
                 gamma_bar=pr["gamma_bar"], lw=pr["lw"], lh=pr["lh"])
    st = O.eahals_init(X, np.array(pr["W0"]), np.array(pr["H0"]), p)
    assert st.s.e_last == pytest.approx(g["e0"], rel=1e-14)
    te, tb, ta = O.eahals_run(X, st, p, 2)
    np.testing.assert_allclose(te, g["e"], rtol=1e-12)
    np.testing.assert_allclose(tb, g["beta_used"], rtol=1e-15)
    np.testing.assert_array_equal(ta, np.array(g["accepted"], dtype=bool))
    fin = g["final"]
    for name in ("W", "H", "Wy", "Hy"):
        np.testing.assert_allclose(getattr(st, name), np.array(fin[name]), rtol=1e-12, atol=1e-14)
    assert st.s.beta == pytest.approx(fin["beta"], rel=1e-15)
    assert st.s.beta_bar == pytest.approx(fin["beta_bar"], rel=1e-15)
    assert st.s.beta_prev == pytest.approx(fin["beta_prev"], rel=1e-15)


@pytest.mark.parametrize("name", ["worked_example_restart_2x2_r1", "worked_example_hp1_2x2_r1",
                                  "worked_example_hp2_2x2_r1"])
def test_worked_examples_step_by_step(name):
    """Hand-worked 2x2 rank-1 runs in exact fractions (tests/golden/), checked
    after every iteration: e(k), the beta it used, the decision, W, H, W_y,
    H_y and the Algorithm 3 scalars.  The restart example pins steps 16-17
    (W_y = W and H_y = H after the restart; beta/eta and beta_bar = beta_{k-1}
    from Algorithm 3) and step 16 as written: its third iteration is accepted
    because e(3) <= e(2), although e(3) exceeds the last accepted error e(1).
    The hp = 2 example keeps a negative H_y (no projection); the hp = 1
    example feeds H_n to the W-update and extrapolates H after it."""
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    pr = g["problem"]
    X = np.array(pr["X"])
    p = O.Params(hp=pr["hp"], beta0=pr["beta0"], eta=pr["eta"], gamma=pr["gamma"],
                 gamma_bar=pr["gamma_bar"], lw=pr["lw"], lh=pr["lh"],
                 compare_prev=pr["compare_prev"])
    st = O.eahals_init(X, np.array(pr["W0"]), np.array(pr["H0"]), p)
    assert st.s.e_last == pytest.approx(g["e0"], rel=1e-14)
    for it in g["iterations"]:
        e, b, acc = O.eahals_step(X, st, p)
        num, den = (int(v) for v in it["e2_exact"].split("/"))
        assert e * e == pytest.approx(num / den, rel=1e-12)
        assert b == pytest.approx(it["beta_used"], rel=1e-15)
        assert acc == bool(it["accepted"])
        aft = it["after"]
        for nm in ("W", "H", "Wy", "Hy"):
            np.testing.assert_allclose(getattr(st, nm), np.array(aft[nm]), rtol=1e-12, atol=1e-14,
                                       err_msg=f"{name} k={it['k']} {nm}")
        assert st.s.beta == pytest.approx(aft["beta"], rel=1e-14)
        assert st.s.beta_bar == pytest.approx(aft["beta_bar"], rel=1e-14)
        assert st.s.beta_prev == pytest.approx(aft["beta_prev"], rel=1e-14)


def test_restart_example_under_the_accepted_error_option():
    """The option compare_prev = 0 (compare with the last accepted error)
    restarts the restart example's third iteration, where step 16 as
    written accepts: the two readings really differ on it."""
    with open(os.path.join(GOLDEN, "worked_example_restart_2x2_r1.json")) as f:
        g = json.load(f)
    pr = g["problem"]
    X = np.array(pr["X"])
    p = O.Params(hp=3, beta0=pr["beta0"], lw=1, lh=1, compare_prev=0)
    st = O.eahals_init(X, np.array(pr["W0"]), np.array(pr["H0"]), p)
    _, _, ta = O.eahals_run(X, st, p, 3)
    np.testing.assert_array_equal(ta, [True, False, False])


@pytest.mark.parametrize("hp", [1, 2, 3])
def test_beta0_zero_is_ahals(hp):
    P = wl.low_rank(40, 30, 5, seed=3, noise=0.05, dtype=np.float64)
    p = O.Params(hp=hp, beta0=0.0, lw=3, lh=4)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    te, tb, ta = O.eahals_run(P.X, st, p, 40)
    assert ta.all()
    W, H, tea = O.ahals_run(P.X, P.W0, P.H0, 3, 4, 40)
    np.testing.assert_array_equal(st.W, W)
    np.testing.assert_array_equal(st.H, H)
    np.testing.assert_array_equal(te, tea)


@pytest.mark.parametrize("hp,compare_prev", [(1, 1), (2, 1), (3, 1), (3, 0)])
def test_restart_logic_and_accepted_errors(hp, compare_prev):
    P = wl.low_rank(60, 45, 6, seed=5, noise=0.02, dtype=np.float64)
    p = O.Params(hp=hp, beta0=0.75, eta=1.5, gamma=1.1, gamma_bar=1.05, lw=2, lh=3,
                 compare_prev=compare_prev)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    e0 = st.s.e_last
    te, tb, ta = O.eahals_run(P.X, st, p, 120)
    assert (~ta).any(), "aggressive parameters should trigger at least one restart"
    ref, prev = e0, e0
    for e, a in zip(te, ta):
        cmp = prev if compare_prev else ref
        assert a == (not e > cmp)
        if a:
            ref = e
        prev = e
    if not compare_prev:
        acc = np.concatenate([[e0], te[ta]])
        assert np.all(np.diff(acc) <= 0.0)


def test_hp3_keeps_extrapolated_h_feasible_and_error_is_of_feasible_pair():
    """hp = 3 projects H_y, so (W_n, H_y) is feasible (Sec. 2)."""
    P = wl.low_rank(50, 40, 5, seed=8, noise=0.0, dtype=np.float64)
    p = O.Params(hp=3, lw=3, lh=3)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    for _ in range(30):
        O.eahals_step(P.X, st, p)
        assert np.all(st.Hy >= 0)
        assert np.all(st.H >= 0) and np.all(st.W >= 0)


def test_hp1_error_is_of_wn_hn():
    """For hp = 1 the W-update and e(k) use H_n (H is extrapolated after)."""
    P = wl.low_rank(30, 25, 4, seed=9, noise=0.05, dtype=np.float64)
    p = O.Params(hp=1, lw=2, lh=2)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    for _ in range(10):
        e, _, acc = O.eahals_step(P.X, st, p)
        if acc:
            assert e == pytest.approx(np.linalg.norm(P.X - st.W @ st.H), rel=1e-9)


def test_power_of_two_scaling_equivariance_is_exact():
    """W -> W L, H -> L^-1 H leaves WH unchanged; every step of Algorithm 2 is
    equivariant, and power-of-two scalings make it exact in floating point."""
    P = wl.low_rank(40, 35, 4, seed=10, noise=0.05, dtype=np.float64)
    lam = np.array([2.0, 0.25, 8.0, 0.5])
    p = O.Params(hp=3, lw=3, lh=4)
    st1 = O.eahals_init(P.X, P.W0, P.H0, p)
    st2 = O.eahals_init(P.X, P.W0 * lam, P.H0 / lam[:, None], p)
    te1, _, ta1 = O.eahals_run(P.X, st1, p, 25)
    te2, _, ta2 = O.eahals_run(P.X, st2, p, 25)
    np.testing.assert_array_equal(ta1, ta2)
    np.testing.assert_allclose(te1, te2, rtol=1e-13)
    np.testing.assert_allclose(st2.W, st1.W * lam, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(st2.H, st1.H / lam[:, None], rtol=1e-12, atol=1e-300)


def test_csr_and_dense_give_the_same_iterates():
    X = _sparse_dense(40, 30, 0.3, 11)
    W0, H0 = wl.init_factors(40, 30, 4, 12, np.float64)
    p = O.Params(hp=3, lw=2, lh=3)
    st1 = O.eahals_init(X, W0, H0, p)
    st2 = O.eahals_init(_csr(X), W0, H0, p)
    te1, _, ta1 = O.eahals_run(X, st1, p, 15)
    te2, _, ta2 = O.eahals_run(_csr(X), st2, p, 15)
    np.testing.assert_array_equal(ta1, ta2)
    np.testing.assert_allclose(te1, te2, rtol=1e-10)
    np.testing.assert_allclose(st1.W, st2.W, rtol=1e-9, atol=1e-12)


def test_extrapolation_accelerates_ahals_on_low_rank():
    """Table 3 / Fig. 3: on exactly low-rank synthetic data E-A-HALS (hp=3,
    beta0=.5, eta=1.5, gamma=1.01, gamma_bar=1.005) ends far below A-HALS
    after the same number of outer iterations."""
    wins = 0
    for seed in range(3):
        P = wl.low_rank(100, 80, 8, seed=100 + seed, dtype=np.float64)
        lw, lh = O.sweep_counts(P.m, P.n, P.nnz, P.r)
        nrm = np.sqrt(O.fro2(P.X))
        p = O.Params(hp=3, lw=lw, lh=lh)
        st = O.eahals_init(P.X, P.W0, P.H0, p)
        O.eahals_run(P.X, st, p, 150)
        e_ext = np.linalg.norm(P.X - st.W @ st.H) / nrm
        W, H, _ = O.ahals_run(P.X, P.W0, P.H0, lw, lh, 150)
        e_plain = np.linalg.norm(P.X - W @ H) / nrm
        wins += e_ext < 0.5 * e_plain
    assert wins == 3


@pytest.mark.slow
def test_low_rank_recovery_and_kkt():
    """X = W0 H0 admits zero error (e_min = 0, Sec. 4.2); E-A-HALS drives the
    relative error and the KKT residuals of (1) towards zero."""
    P = wl.oracle_scale(0)
    lw, lh = O.sweep_counts(P.m, P.n, P.nnz, P.r)
    p = O.Params(hp=3, lw=lw, lh=lh)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    X = P.X

    def kkt(W, H):
        gW = 2 * (W @ (H @ H.T) - X @ H.T)      # gradient, Remark 1
        gH = 2 * ((W.T @ W) @ H - W.T @ X)
        return np.linalg.norm(np.minimum(W, gW)) + np.linalg.norm(np.minimum(H, gH))

    k0 = kkt(st.W, st.H)
    O.eahals_run(X, st, p, 3000)
    rel = np.linalg.norm(X - st.W @ st.H) / np.linalg.norm(X)
    assert rel < 1e-6
    assert kkt(st.W, st.H) < 1e-6 * k0


def test_tie_is_accepted():
    """Algorithm 2 restarts only when e(k) > e(k-1): an exact fixed point
    (X = [1], W = H = [1], every quantity exact in binary) ties at e = 0 and
    must keep accepting, so beta grows as on a decrease (Algorithm 3)."""
    X = np.array([[1.0]])
    p = O.Params(hp=3, lw=1, lh=1)
    st = O.eahals_init(X, np.array([[1.0]]), np.array([[1.0]]), p)
    assert st.s.e_last == 0.0
    te, tb, ta = O.eahals_run(X, st, p, 3)
    np.testing.assert_array_equal(te, [0.0, 0.0, 0.0])
    assert ta.all()
    np.testing.assert_allclose(tb, [0.5, 0.505, 0.51005], rtol=1e-15)


# ------------------------------------------------- line-search step (Sec. 3)

def _f_direct(X, W, H):
    return O.err2_direct(X, W, H)


@pytest.mark.parametrize("csr", [False, True])
def test_line_search_beta_is_the_parabola_vertex(csr):
    """f(beta) = ||X - (W_n + beta (W_n - W)) H_y||^2 is a quadratic; its
    vertex from f(-1), f(0), f(1) (direct errors, no shared formula) is
    beta*, and nearby betas do no better."""
    m, n, r = 23, 17, 4
    Xd = _sparse_dense(m, n, 0.4, 41) if csr else _rand((m, n), 41)
    X = _csr(Xd) if csr else Xd
    W, Wn, Hy = _rand((m, r), 42), _rand((m, r), 43), _rand((r, n), 44)
    D = Wn - W
    f = {b: _f_direct(X, Wn + b * D, Hy) for b in (-1.0, 0.0, 1.0)}
    vertex = (f[-1.0] - f[1.0]) / (2.0 * (f[-1.0] - 2.0 * f[0.0] + f[1.0]))
    bs = O.line_search_beta(X, W, Wn, Hy)
    assert bs == pytest.approx(vertex, rel=1e-9, abs=1e-12)
    fb = _f_direct(X, Wn + bs * D, Hy)
    for eps in (1e-2, -1e-2):
        assert fb <= _f_direct(X, Wn + (bs + eps) * D, Hy)


def test_line_search_beta_zero_cases():
    """No direction (W_n = W) gives 0; an exact fit X = W_n H_y gives 0
    whatever W (the residual is zero)."""
    m, n, r = 12, 9, 3
    W, Wn, Hy = _rand((m, r), 51), _rand((m, r), 52), _rand((r, n), 53)
    X = Wn @ Hy
    assert O.line_search_beta(X, W, Wn, Hy) == pytest.approx(0.0, abs=1e-12)
    assert O.line_search_beta(_rand((m, n), 54), Wn, Wn, Hy) == 0.0


def test_step_line_search_uses_the_iterations_w_wn_hy():
    """hp = 1: the W-update uses H_n, and an accepted step returns W_n, H_n
    as the new W, H; the step's beta* must equal the formula on (the W
    before the step, W_n, H_n)."""
    P = wl.low_rank(30, 25, 4, seed=19, noise=0.05, dtype=np.float64)
    p = O.Params(hp=1, lw=2, lh=2)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    seen = 0
    for _ in range(8):
        W_before = st.W.copy()
        _, _, acc, bs = O.eahals_step(P.X, st, p, line_search=True)
        if acc:
            assert bs == pytest.approx(O.line_search_beta(P.X, W_before, st.W, st.H),
                                       rel=1e-12, abs=1e-15)
            seen += 1
    assert seen >= 3


# ------------------------------------- exact NNLS and E-ANLS (Sec. 1, Sec. 4)

def _nnls_problem(m, r, seed):
    g = wl.rng(seed)
    W = g.random((m, r)) - 0.2          # some negative entries: active bounds occur
    v = g.random(m) * 2.0 - 0.7
    return W, v


@pytest.mark.parametrize("r", [1, 2, 3, 5, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_nnls_matches_bruteforce(r, seed):
    """orc_nnls against enumeration of every free set (small r), from a
    zero and from a random warm start (the minimiser is unique)."""
    W, v = _nnls_problem(3 * r + 4, r, 700 + 10 * r + seed)
    G, b = W.T @ W, W.T @ v
    ref = _nnls_bruteforce(W, v)
    x0, it0 = O.nnls(G, b)
    x1, it1 = O.nnls(G, b, x0=_rand(r, 900 + seed))
    assert it0 >= 0 and it1 >= 0
    np.testing.assert_allclose(x0, ref, atol=1e-10)
    np.testing.assert_allclose(x1, ref, atol=1e-10)


@pytest.mark.parametrize("r", [12, 40])
def test_nnls_matches_scipy_and_kkt(r):
    """Larger r: scipy.optimize.nnls (Lawson-Hanson, a different algorithm)
    and the KKT conditions x >= 0, y = Gx - b >= 0, x_i y_i = 0."""
    from scipy.optimize import nnls as sp_nnls
    W, v = _nnls_problem(3 * r, r, 800 + r)
    G, b = W.T @ W, W.T @ v
    x, it = O.nnls(G, b)
    assert it >= 0
    ref, _ = sp_nnls(W, v)
    np.testing.assert_allclose(x, ref, atol=1e-9)
    y = G @ x - b
    scale = max(np.abs(b).max(), np.abs(G).max())
    assert x.min() >= 0.0
    assert y.min() >= -1e-10 * scale
    assert np.abs(x * y).max() <= 1e-10 * scale * max(1.0, x.max())
    assert 0 < np.count_nonzero(x) < r          # the bounds are active somewhere


def test_nnls_zero_column_keeps_its_value():
    """A zero column of W makes row and column i of G zero: that coordinate
    takes no part and keeps its warm-start value (as in HALS)."""
    W, v = _nnls_problem(20, 4, 31)
    W[:, 2] = 0.0
    G, b = W.T @ W, W.T @ v
    x, it = O.nnls(G, b, x0=np.array([0.3, 0.0, 0.7, 0.1]))
    assert it >= 0 and x[2] == 0.7
    keep = [0, 1, 3]
    np.testing.assert_allclose(x[keep], _nnls_bruteforce(W[:, keep], v), atol=1e-10)


def _eanls_params(P, hp, beta0=0.5):
    return O.Params(hp=hp, beta0=beta0, eta=1.5, gamma=1.1, gamma_bar=1.05, nnls_exact=1)


def test_anls_is_monotone_and_solves_each_subproblem():
    """beta0 = 0 gives ANLS: alternating exact minimisation, so the error of
    the accepted pair never increases, and every H is the exact NNLS
    solution for the W_y it was computed from (hp = 1 keeps it visible)."""
    P = wl.low_rank(40, 30, 4, seed=23, noise=0.1, dtype=np.float64)
    p = _eanls_params(P, hp=1, beta0=0.0)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    prev = np.inf
    for _ in range(15):
        Wy = st.Wy.copy()
        e, _, acc = O.eahals_step(P.X, st, p)
        assert acc
        err = np.linalg.norm(P.X - st.W @ st.H)
        assert err <= prev * (1 + 1e-12)
        prev = err
        for j in range(P.n):
            np.testing.assert_allclose(st.H[:, j], _nnls_bruteforce(Wy, P.X[:, j]), atol=1e-9)


@pytest.mark.parametrize("m,n,r,seed,floor", [(50, 40, 5, 29, 1e-10), (80, 60, 8, 37, 1e-4)])
def test_eanls_accelerates_anls_on_low_rank(m, n, r, seed, floor):
    """Sec. 4.3: with extrapolation (hp = 1, beta0 = 0.5, eta = 1.5,
    (gamma, gamma_bar) = (1.1, 1.05)) ANLS finds near-exact factorisations
    of exactly low-rank data that plain ANLS does not reach in the same
    number of iterations (measured at 150: 1.2e-15 / 9.5e-6 against
    1.9e-3 / 2.4e-3)."""
    P = wl.low_rank(m, n, r, seed=seed, dtype=np.float64)
    K = 150
    errs = {}
    for name, beta0 in (("anls", 0.0), ("eanls", 0.5)):
        p = _eanls_params(P, hp=1, beta0=beta0)
        st = O.eahals_init(P.X, P.W0, P.H0, p)
        O.eahals_run(P.X, st, p, K)
        errs[name] = np.linalg.norm(P.X - st.W @ st.H) / np.linalg.norm(P.X)
    assert errs["eanls"] < floor and errs["anls"] > 1e-3, errs


def test_eanls_csr_and_dense_agree_and_hp3_stays_feasible():
    """E-ANLS on a sparse X: the CSR and dense oracles take the same
    decisions and reach the same iterates; with hp = 3 every accepted pair
    and the projected H_y stay nonnegative."""
    X = _sparse_dense(40, 30, 0.3, 13)
    W0, H0 = wl.init_factors(40, 30, 4, 14, np.float64)
    p = O.Params(hp=3, beta0=0.5, eta=1.5, gamma=1.1, gamma_bar=1.05, nnls_exact=1)
    st1 = O.eahals_init(X, W0, H0, p)
    st2 = O.eahals_init(_csr(X), W0, H0, p)
    te1, _, ta1 = O.eahals_run(X, st1, p, 12)
    te2, _, ta2 = O.eahals_run(_csr(X), st2, p, 12)
    np.testing.assert_array_equal(ta1, ta2)
    np.testing.assert_allclose(te1, te2, rtol=1e-10)
    np.testing.assert_allclose(st1.W, st2.W, rtol=1e-9, atol=1e-12)
    assert np.all(st1.W >= 0) and np.all(st1.H >= 0) and np.all(st1.Hy >= 0)


@pytest.mark.parametrize("side", ["rows", "cols"])
def test_permutation_equivariance(side):
    """Permuting the rows of X and W (or the columns of X and H) permutes
    the iterates: the closed-form updates act per row of W / column of H and
    the products only sum in another order (agreement to round-off, same
    decisions)."""
    P = wl.low_rank(36, 28, 4, seed=17, noise=0.05, dtype=np.float64)
    perm = wl.rng(18).permutation(P.m if side == "rows" else P.n)
    X, W0, H0 = P.X, P.W0, P.H0
    if side == "rows":
        Xp, W0p, H0p = X[perm], W0[perm], H0
    else:
        Xp, W0p, H0p = X[:, perm], W0, H0[:, perm]
    p = O.Params(hp=3, lw=3, lh=3)
    st = O.eahals_init(X, W0, H0, p)
    stp = O.eahals_init(Xp, W0p, H0p, p)
    te, _, ta = O.eahals_run(X, st, p, 20)
    tep, _, tap = O.eahals_run(Xp, stp, p, 20)
    np.testing.assert_array_equal(ta, tap)
    np.testing.assert_allclose(te, tep, rtol=1e-10)
    if side == "rows":
        np.testing.assert_allclose(st.W[perm], stp.W, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(st.H, stp.H, rtol=1e-8, atol=1e-12)
    else:
        np.testing.assert_allclose(st.W, stp.W, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(st.H[:, perm], stp.H, rtol=1e-8, atol=1e-12)


def test_thread_count_does_not_change_results():
    """The oracle's parallel loops only split independent outputs, each
    summed in the sequential order: 1 and several threads agree bit for bit."""
    P = wl.low_rank(130, 90, 7, seed=21, noise=0.03, dtype=np.float64)
    out = []
    for nt in (1, 3):
        O.set_threads(nt)
        p = O.Params(hp=3, lw=3, lh=4)
        st = O.eahals_init(P.X, P.W0, P.H0, p)
        te, _, _ = O.eahals_run(P.X, st, p, 12)
        e2 = O.err2_direct(P.X, st.W, st.H)
        Hn, _ = O.nnls_h(O.wtx(P.X, st.W), O.gram_w(st.W), st.H)
        out.append((te, st.W, st.H, e2, Hn))
    O.set_threads(0)
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


# ------------------------------------------- A-HALS inner stopping rule

@pytest.mark.parametrize("delta", [1e-12, 0.5, 0.1, 0.01])
def test_delta_rule_stops_where_the_definition_says(delta):
    """orc_hals_sweeps_h_delta against the rule of Gillis & Glineur (2012)
    evaluated with numpy on single sweeps: stop after the first sweep l >= 2
    with ||H^(l) - H^(l-1)||_F <= delta ||H^(1) - H^(0)||_F (cap 30), and
    the result equals that many plain sweeps bit for bit."""
    P = wl.low_rank(60, 40, 6, seed=30, noise=0.05, dtype=np.float64)
    W = _rand((60, 6), 31)
    A, G = O.wtx(P.X, W), O.gram_w(W)
    H0 = _rand((6, 40), 32)
    Hd, used = O.hals_sweeps_h_delta(A, G, H0, 30, delta)
    H = H0.copy()
    first, want = None, 30
    for l in range(1, 31):
        Hn = O.hals_sweeps_h(A, G, H, 1)
        d = np.linalg.norm(Hn - H)
        H = Hn
        if l == 1:
            first = d
        elif d <= delta * first:
            want = l
            break
    assert used == want
    np.testing.assert_array_equal(Hd, O.hals_sweeps_h(A, G, H0, used))
    if delta >= 0.5:
        assert used < 30
    if delta == 1e-12:
        assert used == 30


@pytest.mark.parametrize("delta", [1e-12, 0.5, 0.1])
def test_delta_rule_w_side_stops_where_the_definition_says(delta):
    """orc_hals_sweeps_w_delta against the same rule evaluated with numpy
    over single sweeps of the rows of W: stop after the first sweep l >= 2
    with ||W^(l) - W^(l-1)||_F <= delta ||W^(1) - W^(0)||_F (cap 25), and
    the result equals that many plain sweeps bit for bit."""
    P = wl.low_rank(50, 45, 5, seed=34, noise=0.05, dtype=np.float64)
    H = _rand((5, 45), 35)
    C, D = O.xht(P.X, H), O.gram_h(H)
    W0 = _rand((50, 5), 36)
    Wd, used = O.hals_sweeps_w_delta(C, D, W0, 25, delta)
    W = W0.copy()
    first, want = None, 25
    for l in range(1, 26):
        Wn = O.hals_sweeps_w(C, D, W, 1)
        d = np.linalg.norm(Wn - W)
        W = Wn
        if l == 1:
            first = d
        elif d <= delta * first:
            want = l
            break
    assert used == want
    np.testing.assert_array_equal(Wd, O.hals_sweeps_w(C, D, W0, used))
    if delta >= 0.5:
        assert used < 25
    if delta == 1e-12:
        assert used == 25


def test_delta_rule_in_the_step_reports_its_sweeps():
    P = wl.low_rank(50, 40, 5, seed=33, noise=0.05, dtype=np.float64)
    p = O.Params(hp=3, lw=20, lh=25, delta=0.1)
    st = O.eahals_init(P.X, P.W0, P.H0, p)
    O.eahals_step(P.X, st, p)
    assert 2 <= st.s.lh_used <= 25 and 2 <= st.s.lw_used <= 20
    # the same step with fixed counts equal to those sweeps is identical
    q = O.Params(hp=3, lw=st.s.lw_used, lh=st.s.lh_used)
    s2 = O.eahals_init(P.X, P.W0, P.H0, q)
    O.eahals_step(P.X, s2, q)
    np.testing.assert_array_equal(st.W, s2.W)
    np.testing.assert_array_equal(st.H, s2.H)
