"""Tensor-core precision modes (tcgen05): the product kernel in isolation and
the solver in TF32 and split-BF16 modes against the FP64 oracle.

Tolerances come from the operand precision: TF32 keeps 10 explicit mantissa
bits and the operands are rounded to nearest, so each product term is off by
up to ~2^-10 relative and the normwise error of P Q^T is bounded by ~2^-10;
split BF16 keeps ~16 bits of each operand and drops lo.lo, so the terms are
off by ~2^-16 and sums by ~1e-5 relative.  Accumulation over K adds little:
each 64-deep K stage is summed by the tensor core and the stages are added
with compensation.  After K iterations to convergence the solver in both
modes must match the oracle's final relative error within 1e-4 relative,
the same gate as the FP32 path.
"""
import numpy as np
import pytest

import oracle as O
from paper_1805_06604_gb300 import nmf
from paper_1805_06604_gb300 import workloads as wl

from gpu_helpers import f32, gpu_kwargs, normwise, oracle_X, oracle_params

pytestmark = pytest.mark.gpu

TOL = {nmf.NMF_PREC_TF32: 2.0 ** -10, nmf.NMF_PREC_BF16X3: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_06604_gb300 import build
    build.build()
    O.build()
    nmf.load()


@pytest.mark.parametrize("prec", [nmf.NMF_PREC_TF32, nmf.NMF_PREC_BF16X3])
@pytest.mark.parametrize("M,K,q", [(300, 1000, 50), (128, 64, 16), (1000, 4000, 64),
                                   (257, 333, 1), (512, 2048, 128), (129, 96, 33)])
def test_matmul_nt_matches_fp64(prec, M, K, q):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + K + q)
    ldp = (K + 7) // 8 * 8
    Pb = torch.rand((M, ldp), device="cuda", generator=g)
    Qb = torch.rand((q, ldp), device="cuda", generator=g) * 2.0 - 0.5
    P, Q = Pb[:, :K], Qb[:, :K]
    out = torch.full((M, q), float("nan"), device="cuda")
    nmf.nmf_matmul_nt(P, Q, out, prec)
    ref = (P.double() @ Q.double().T).cpu().numpy()
    err = normwise(out.cpu().numpy(), ref)
    assert np.isfinite(out.cpu().numpy()).all()
    assert err <= TOL[prec], err


def test_matmul_nt_rejects_fp32_and_bad_shapes():
    import torch
    P = torch.rand((64, 64), device="cuda")
    out = torch.empty((64, 8), device="cuda")
    with pytest.raises(nmf.NmfError) as ei:
        nmf.nmf_matmul_nt(P, P[:8], out, nmf.NMF_PREC_FP32)
    assert ei.value.status == nmf.NMF_ENOTSUP
    with pytest.raises(nmf.NmfError) as ei:
        nmf.nmf_matmul_nt(P[:, :60], P[:8, :60], out, 7)
    assert ei.value.status in (nmf.NMF_ENOTSUP, nmf.NMF_EINVAL)


@pytest.mark.parametrize("prec", [nmf.NMF_PREC_TF32, nmf.NMF_PREC_BF16X3])
def test_solver_single_step_precision_modes(prec):
    """One step from an identical state in a tensor-core mode: the factors
    differ from the FP64 oracle by the operand precision times the
    subproblem conditioning."""
    from gpu_helpers import gram_kappa, load_state, state_to_f32
    P = wl.low_rank(700, 520, 24, seed=21, noise=0.02)
    p = oracle_params(P)
    Xo = oracle_X(P)
    st = O.eahals_init(Xo, P.W0, P.H0, p)
    O.eahals_run(Xo, st, p, 3)
    st = state_to_f32(st)
    kappa = gram_kappa(st)
    s = nmf.Solver(f32(P.X), P.r, f32(P.W0), f32(P.H0), precision=prec, **gpu_kwargs(p))
    load_state(s, st)
    s.step(1)
    _, W, H, Wy, Hy = s.get_state()
    info = s.info()
    s.close()
    assert info.device_status == 0
    O.eahals_step(Xo, st, p)
    for a, b in ((W, st.W), (H, st.H)):
        assert normwise(a, b) <= 4.0 * kappa * TOL[prec]


def test_precision_study_image_like_small():
    """The precision study on a reduced image-like matrix: FP32 CUDA cores,
    TF32 and split BF16 against the FP64 oracle after K iterations.  Prints
    the errors; both tensor-core modes must stay within 1e-3 relative of
    the oracle's final error (measured: TF32 8.8e-5, BF16X3 1.2e-4 after 60
    unconverged iterations; TF32 factors X rounded to 10 mantissa bits, about
    2e-4 relative RMS from X, which bounds how close it can come).  The
    full-size image-like run (tests/test_gpu_fullsize_k.py) holds both at 1e-4."""
    P = wl.image_like(seed=3, grid=(32, 28), n=600, r=16, blobs=16)
    p = oracle_params(P)
    Xo = oracle_X(P)
    K = 60
    st = O.eahals_init(Xo, P.W0, P.H0, p)
    O.eahals_run(Xo, st, p, K)
    rel_o = np.linalg.norm(Xo - st.W @ st.H) / np.linalg.norm(Xo)
    report = {}
    for name, prec in (("fp32", nmf.NMF_PREC_FP32), ("tf32", nmf.NMF_PREC_TF32),
                       ("bf16x3", nmf.NMF_PREC_BF16X3)):
        with nmf.Solver(f32(P.X), P.r, f32(P.W0), f32(P.H0), precision=prec,
                        **gpu_kwargs(p)) as s:
            s.step(K)
            W, H = s.factors()
            assert s.info().device_status == 0
        rel = np.linalg.norm(Xo - W.astype(np.float64) @ H) / np.linalg.norm(Xo)
        report[name] = (rel, abs(rel - rel_o) / rel_o, normwise(W, st.W), normwise(H, st.H))
    print("\nprecision study (final relerr, |d relerr|/relerr, W err, H err); oracle", rel_o)
    for k, v in report.items():
        print(f"  {k:7s} {v[0]:.6e} {v[1]:.2e} {v[2]:.2e} {v[3]:.2e}")
    assert report["fp32"][1] <= 1e-4
    assert report["bf16x3"][1] <= 1e-3
    assert report["tf32"][1] <= 1e-3


@pytest.mark.parametrize("prec", [nmf.NMF_PREC_TF32, nmf.NMF_PREC_BF16X3])
@pytest.mark.parametrize("m,n,r,K,hp", [(300, 200, 8, 800, 3), (400, 300, 10, 800, 1)])
def test_k_iterations_precision_modes(prec, m, n, r, K, hp):
    """K iterations on noisy low-rank X to the oracle's floor (restart test
    against e(k-1), as in the FP32 gate): the tensor-core modes reach the
    oracle's relative error within 1e-4 relative.  This needs the products
    and the Grams to see one and the same rounded factor, else the Remark 1
    error that decides every restart carries per-iteration noise far above
    the differences it has to resolve."""
    P = wl.low_rank(m, n, r, seed=11, noise=0.05)
    p = oracle_params(P, hp=hp, compare_prev=1)
    Xo = oracle_X(P)
    st = O.eahals_init(Xo, P.W0, P.H0, p)
    O.eahals_run(Xo, st, p, K)
    rel_o = np.linalg.norm(Xo - st.W @ st.H) / np.linalg.norm(Xo)
    with nmf.Solver(f32(P.X), P.r, f32(P.W0), f32(P.H0), precision=prec, **gpu_kwargs(p)) as s:
        s.step(K)
        W, H = s.factors()
        assert s.info().device_status == 0
    rel_g = np.linalg.norm(Xo - W.astype(np.float64) @ H) / np.linalg.norm(Xo)
    assert abs(rel_g - rel_o) <= 1e-4 * rel_o, (rel_g, rel_o)
