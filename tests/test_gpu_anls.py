"""E-ANLS on the GPU (nmf_params.exact_nnls = 1): Algorithm 2 with both NNLS
subproblems solved exactly by block principal pivoting (Sec. 1: ANLS solves
them exactly with the active-set-like method of Kim & Park), against the
FP64 oracle's orc_nnls / nnls_exact path.

Tolerances: a single step from an identical state within the FP32 step gate
of the HALS path, max(1e-5, 4 kappa 2^-24) normwise (the exact solution of
an FP32-rounded subproblem moves by up to ~kappa u); on tiny r the zero
pattern of every column of H and row of W -- the final free sets -- equals
the oracle's; after K iterations the relative error of the returned pair
within 1e-4 relative of the oracle's (with decision replay where an FP32
near-tie flipped a restart decision, as for the HALS path)."""
import numpy as np
import pytest

import oracle as O
from paper_1805_06604_gb300 import nmf
from paper_1805_06604_gb300 import workloads as wl

from gpu_helpers import normwise, oracle_params, single_step
from test_gpu_parity import _check_step, k_iteration_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_06604_gb300 import build
    build.build()
    O.build()
    nmf.load()


@pytest.mark.parametrize("m,n,r,hp,warm", [
    (200, 150, 6, 3, 0),
    (300, 220, 12, 3, 2),
    (257, 193, 33, 3, 2),      # ragged shapes, r > 32 (two slots per lane)
    (200, 150, 10, 1, 2),      # hp = 1
    (600, 500, 80, 3, 0),      # r > 64 (three slots per lane)
])
def test_exact_single_step_matches_oracle(m, n, r, hp, warm):
    """One E-ANLS step from an identical state, each exact subproblem checked
    on its own inputs: H_n against the oracle's (same W_y, H_y); W_n against
    the oracle's exact solve of the W-subproblem built from the H_y the GPU's
    W-update used (an exact solve carries the H side's round-off into W
    amplified by the conditioning of H_y H_y^T, so comparing W_n with the
    oracle's own full step measures that amplification, not the solver).
    Gates: max(1e-5, 4 kappa 2^-24) with kappa of the subproblem's Gram."""
    from gpu_helpers import gram_kappa, state_to_f32, oracle_X, make_solver, load_state, f32
    P = wl.low_rank(m, n, r, seed=m + r, noise=0.02)
    p = oracle_params(P, hp=hp, nnls_exact=1)
    Xo = oracle_X(P)
    st = O.eahals_init(Xo, P.W0.astype(np.float32), P.H0.astype(np.float32), p)
    if warm:
        O.eahals_run(Xo, st, p, warm)
    st = state_to_f32(st)
    start = st.copy()
    with make_solver(P, p) as s:
        load_state(s, st)
        s.step(1)
        sc, W, H, Wy, Hy = s.get_state()
        te, _, ta = s.trace()
        assert s.info().exact_failed == 0
    e_o, _, acc_o = O.eahals_step(Xo, st, p)
    assert bool(ta[-1]) == acc_o

    def tol(G):
        keep = np.diag(G) > 0
        ev = np.linalg.eigvalsh(G[np.ix_(keep, keep)])
        return max(1e-5, 4.0 * ev[-1] / ev[0] * 2.0 ** -24)

    # H side: same inputs as the oracle's step.
    G = start.Wy.T @ start.Wy
    Hn = H if acc_o else None
    if acc_o:
        errH = normwise(H, st.H)
        assert errH <= tol(G), (errH, tol(G))
    # W side from the GPU's own H_y (hp >= 2: the extrapolated H_y; hp = 1: H_n).
    Hw = np.asarray(Hy if hp >= 2 else H, np.float64) if acc_o else None
    if acc_o:
        C = O.xht(Xo, Hw)
        D = O.gram_h(Hw)
        Wref, worst = O.nnls_w(C, D, start.Wy)
        assert worst >= 0
        errW = normwise(W, Wref)
        print(f"\n{m}x{n} r={r} hp={hp}: H {errH:.2e} (gate {tol(G):.1e}), W {errW:.2e} "
              f"(gate {tol(D):.1e}), e(k)^2 diff {abs(te[-1] ** 2 - e_o ** 2) / O.fro2(Xo):.1e}")
        assert errW <= tol(D), (errW, tol(D))


@pytest.mark.parametrize("r", [2, 3, 4, 6])
def test_exact_free_sets_tiny_r(r):
    """The zero pattern of every column of H_n and row of W_n (the final
    free sets of the block principal pivoting) equals the oracle's."""
    P = wl.low_rank(120, 90, r, seed=40 + r, noise=0.3)
    p = oracle_params(P, nnls_exact=1)
    res = single_step(P, p, 1)
    g, o = res["gpu"], res["orc"]
    for name in ("W", "H"):
        zg, zo = np.asarray(g[name]) > 0, np.asarray(o[name]) > 0
        assert (zg == zo).all(), f"{name}: {(zg != zo).sum()} free-set differences"
        assert 0 < zo.sum() < zo.size
    _check_step(res)


def test_exact_k_iterations_relative_error():
    k_iteration_parity(300, 200, 8, 100, 3, 0.05, nnls_exact=1)


def test_anls_is_monotone_and_settles():
    """beta0 = 0 gives plain ANLS: every block update solves its subproblem
    exactly, so the error never increases and no restart happens; every
    subproblem settles (exact_failed = 0)."""
    P = wl.low_rank(400, 300, 16, seed=3, noise=0.01)
    from gpu_helpers import make_solver
    p = oracle_params(P, beta0=0.0, nnls_exact=1)
    with make_solver(P, p) as s:
        e0 = s.info().e_last
        s.step(20)
        info = s.info()
        te, _, ta = s.trace()
    assert info.exact_failed == 0 and info.device_status == 0
    assert ta.all()
    e = np.concatenate([[e0], te])
    assert np.all(np.diff(e) <= 1e-6 * e[:-1])
