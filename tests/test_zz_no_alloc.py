"""nmf_fro2_noalloc, the entry point for callers that cannot allocate device
memory where they need ||X||_F^2 (their device memory belongs to another
allocator, or an allocation could stall a latency-critical loop).  It must
agree with the value nmf_create computes with allocated scratch -- the
||X||^2 that nmf_get_info reports -- on two calls in a row, since every call
reuses the same fixed scratch array.  Kept in a file that is collected last.
"""
import numpy as np
import pytest

from paper_1805_06604_gb300 import nmf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_06604_gb300 import build
    build.build()
    nmf.load()


def _reference_fro2(X, r=4):
    """||X||^2 as nmf_create computes it (allocated scratch)."""
    import torch
    m, n = X.shape
    g = np.random.default_rng(0)
    W0 = torch.from_numpy(g.random((m, r), dtype=np.float32)).cuda()
    H0 = torch.from_numpy(g.random((r, n), dtype=np.float32)).cuda()
    with nmf.Solver(X.contiguous(), r, W0, H0, stream=torch.cuda.current_stream()) as s:
        return s.info().fro2


def test_noalloc_matches_allocating_path_twice():
    import torch
    g = torch.Generator(device="cuda").manual_seed(3)
    cases = [torch.rand((1500, 997), device="cuda", generator=g),
             torch.rand((333, 4096), device="cuda", generator=g) * 3.0 - 1.0]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for X in cases:
        ref = _reference_fro2(X)
        for call in range(2):
            out.zero_()
            nmf.nmf_fro2_noalloc(X, out[call:call + 1], stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            got = float(out[call].item())
            assert got == pytest.approx(ref, rel=1e-12), (call, got, ref)


def test_noalloc_strided_rows():
    import torch
    base = torch.rand((700, 640), device="cuda")
    X = base[:, :513]                         # row stride 640 > n
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    nmf.nmf_fro2_noalloc(X, out)
    torch.cuda.synchronize()
    assert float(out.item()) == pytest.approx(_reference_fro2(X), rel=1e-12)


def test_noalloc_rejects_oversized_input():
    import torch
    X = torch.empty((1, 1), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = nmf.load()
    st = lib.nmf_fro2_noalloc(X.data_ptr(), 1 << 15, 1 << 14, 1 << 14, out.data_ptr(), None)
    assert st == nmf.NMF_ENOTSUP
    assert "2^28" in nmf.nmf_last_error()
    # m * n wraps to 1 in 64-bit arithmetic: still rejected, nothing launched
    st = lib.nmf_fro2_noalloc(X.data_ptr(), 274177, 67280421310721, 67280421310721,
                              out.data_ptr(), None)
    assert st == nmf.NMF_ENOTSUP
