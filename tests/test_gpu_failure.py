"""Failure detection without a GPU fault.  The tensor-core product's waits
are bounded; nmf_debug_set_fixup_stall makes one of them -- the last CTA's
wait for the other CTAs' partials of a shared tile, in its final segment,
when none of its copies or MMAs is in flight -- wait for partials that never
come.  The wait runs out (about 0.1 s), the kernel records it and returns,
the call reports NMF_ETIMEOUT, and the context stays usable: the next calls,
and a fresh solver, run normally."""
import numpy as np
import pytest

from paper_1805_06604_gb300 import nmf
from paper_1805_06604_gb300 import workloads as wl

from gpu_helpers import f32, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1805_06604_gb300 import build
    build.build()
    nmf.load()


def test_bounded_wait_times_out_and_context_stays_usable():
    import torch
    # One 128-row tile over a long K: stream-K gives every CTA exactly one
    # segment of it, so the CTA that sums the partials is in its final
    # segment whichever arrives last.
    g = torch.Generator(device="cuda").manual_seed(5)
    P = torch.rand((128, 8192), device="cuda", generator=g)
    Q = torch.rand((16, 8192), device="cuda", generator=g)
    out = torch.zeros((128, 16), device="cuda")
    ref = (P.double() @ Q.double().T).cpu().numpy()
    nmf.nmf_debug_set_fixup_stall(1)
    try:
        with pytest.raises(nmf.NmfError) as ei:
            nmf.nmf_matmul_nt(P, Q, out, nmf.NMF_PREC_TF32)
        assert ei.value.status == nmf.NMF_ETIMEOUT
    finally:
        nmf.nmf_debug_set_fixup_stall(0)
    torch.cuda.synchronize()
    out.zero_()
    nmf.nmf_matmul_nt(P, Q, out, nmf.NMF_PREC_TF32)
    assert normwise(out.cpu().numpy(), ref) <= 2.0 ** -10
    # A fresh solver in the same context runs normally.
    Pb = wl.low_rank(300, 260, 12, seed=9, noise=0.01)
    with nmf.Solver(f32(Pb.X), Pb.r, f32(Pb.W0), f32(Pb.H0), precision=nmf.NMF_PREC_TF32) as s:
        s.step(10)
        info = s.info()
        assert info.device_status == 0 and info.k == 10 and np.isfinite(info.e_last)


def test_fixup_stall_rejects_negative():
    with pytest.raises(nmf.NmfError) as ei:
        nmf.nmf_debug_set_fixup_stall(-1)
    assert ei.value.status == nmf.NMF_EINVAL
