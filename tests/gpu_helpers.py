"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64
oracle from identical (float32-representable) states and compare."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1805_06604_gb300 import nmf

# FP32 single-step gate of the solver, on the normwise max error of every
# factor (max |gpu - oracle| / max |oracle|): 1e-5, raised to 4 kappa u when
# the subproblems are too ill-conditioned for FP32 to reach it.  kappa is the
# larger condition number of the two Grams W_y^T W_y and H_y H_y^T and
# u = 2^-24: merely rounding the inputs of an NNLS subproblem (A, G or C, D)
# to FP32 perturbs its solution by up to ~kappa u, and the FP32 sweeps add an
# error of the same order (checked in FP64 emulation: exactly rounded FP32
# inputs with FP64 sweeps already give 1.3e-5 at kappa = 195).
STEP_TOL = 1e-5
U32 = 2.0 ** -24


def step_tol(kappa: float) -> float:
    return max(STEP_TOL, 4.0 * kappa * U32)


def gram_kappa(st) -> float:
    """Condition number of the Grams the two NNLS subproblems see.  A
    coordinate whose Gram diagonal is zero (a zero column of W_y or row of
    H_y) is skipped by the HALS update and takes no part in the subproblem,
    so the condition number is that of the Gram restricted to the others."""
    def cond(M):
        keep = np.diag(M) > 0.0
        M = M[np.ix_(keep, keep)]
        if M.size == 0:
            return 1.0
        ev = np.linalg.eigvalsh(M)
        return float(ev[-1] / max(ev[0], ev[-1] * 1e-16))
    return max(cond(st.Wy.T @ st.Wy), cond(st.Hy @ st.Hy.T))


def f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def normwise(a, b) -> float:
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(np.asarray(a, np.float64) - b).max() / (den if den > 0 else 1.0))


def oracle_params(P, hp=3, beta0=0.5, eta=1.5, gamma=1.01, gamma_bar=1.005, project_w=0,
                  compare_prev=1, lw=None, lh=None, nnls_exact=0, delta=0.0):
    if lw is None or lh is None:
        aw, ah = O.sweep_counts(P.m, P.n, P.nnz, P.r)
        lw = aw if lw is None else lw
        lh = ah if lh is None else lh
    return O.Params(hp=hp, beta0=beta0, eta=eta, gamma=gamma, gamma_bar=gamma_bar, lw=lw, lh=lh,
                    project_w=project_w, compare_prev=compare_prev, nnls_exact=nnls_exact,
                    delta=delta)


def gpu_kwargs(p: O.Params) -> dict:
    return dict(hp=p.hp, beta0=p.beta0, eta=p.eta, gamma=p.gamma, gamma_bar=p.gamma_bar,
                lw=p.lw, lh=p.lh, project_w=p.project_w, compare_prev=p.compare_prev,
                exact_nnls=p.nnls_exact, delta=p.delta)


def oracle_X(P):
    """The oracle's view of X: the float32 values the GPU sees, widened."""
    if P.is_csr:
        return O.Matrix(m=P.m, n=P.n, rowptr=P.rowptr, colidx=P.colidx,
                        val=P.val.astype(np.float32).astype(np.float64))
    return P.X.astype(np.float32).astype(np.float64)


def make_solver(P, p: O.Params, **extra):
    if P.is_csr:
        return nmf.Solver(None, P.r, f32(P.W0), f32(P.H0), csr=(P.rowptr, P.colidx, f32(P.val)),
                          m=P.m, n=P.n, **gpu_kwargs(p), **extra)
    return nmf.Solver(f32(P.X), P.r, f32(P.W0), f32(P.H0), **gpu_kwargs(p), **extra)


def state_to_f32(st: O.State) -> O.State:
    """Round an oracle state to float32 (so both sides start identically)."""
    return O.State(f32(st.W).astype(np.float64), f32(st.H).astype(np.float64),
                   f32(st.Wy).astype(np.float64), f32(st.Hy).astype(np.float64),
                   O.Scalars(**vars(st.s)))


def load_state(solver, st: O.State):
    s = nmf.nmf_scalars(st.s.beta, st.s.beta_bar, st.s.beta_prev, st.s.e_last, st.s.e_prev,
                        st.s.k)
    solver.set_state(s, f32(st.W), f32(st.H), f32(st.Wy), f32(st.Hy))


def single_step(P, p: O.Params, warm: int):
    """Oracle runs `warm` iterations; both sides then take one step from the
    float32-rounded state.  Returns a dict of gpu / oracle results."""
    Xo = oracle_X(P)
    st = O.eahals_init(Xo, P.W0.astype(np.float32), P.H0.astype(np.float32), p)
    if warm:
        O.eahals_run(Xo, st, p, warm)
    st = state_to_f32(st)
    kappa = gram_kappa(st)
    with make_solver(P, p) as s:
        load_state(s, st)
        s.step(1)
        sc, W, H, Wy, Hy = s.get_state()
        te, tb, ta = s.trace()
    e_o, b_o, acc_o = O.eahals_step(Xo, st, p)
    return dict(gpu=dict(W=W, H=H, Wy=Wy, Hy=Hy, e=te[-1], beta=tb[-1], acc=bool(ta[-1]),
                         scalars=sc),
                orc=dict(W=st.W, H=st.H, Wy=st.Wy, Hy=st.Hy, e=e_o, beta=b_o, acc=acc_o,
                         scalars=st.s),
                fro2=O.fro2(Xo), kappa=kappa, tol=step_tol(kappa))


def direct_relerr_gpu(P, W, H) -> float:
    """||X - W H||_F / ||X||_F of host factors, evaluated in FP64 with torch
    on the GPU (row blocks for dense X; for CSR X as ||X||^2 - 2<X, WH> +
    <W^T W, H H^T>, <X, WH> entry by entry over the stored entries)."""
    import torch
    W = torch.as_tensor(np.asarray(W, np.float64), device="cuda")
    H = torch.as_tensor(np.asarray(H, np.float64), device="cuda")
    if P.is_csr:
        rp = torch.as_tensor(P.rowptr, device="cuda")
        rows = torch.repeat_interleave(torch.arange(P.m, device="cuda"), rp[1:] - rp[:-1])
        cols = torch.as_tensor(P.colidx.astype(np.int64), device="cuda")
        val = torch.as_tensor(P.val.astype(np.float32).astype(np.float64), device="cuda")
        fro2 = float((val * val).sum())
        cross = 0.0
        for s0 in range(0, val.numel(), 1 << 20):
            sl = slice(s0, s0 + (1 << 20))
            cross += float((val[sl] * (W[rows[sl]] * H[:, cols[sl]].T).sum(1)).sum())
        quad = float(((W.T @ W) * (H @ H.T)).sum())
        return max(fro2 - 2.0 * cross + quad, 0.0) ** 0.5 / fro2 ** 0.5
    X = torch.as_tensor(P.X.astype(np.float32), device="cuda")
    num = den = 0.0
    for i in range(0, P.m, 2048):
        Xb = X[i:i + 2048].double()
        num += float(((Xb - W[i:i + 2048] @ H) ** 2).sum())
        den += float((Xb ** 2).sum())
    return (num / den) ** 0.5
