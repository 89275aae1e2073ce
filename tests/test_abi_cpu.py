"""CPU-side checks of the boundary: the library builds for sm_103a, loads
without a GPU, exports every function that include/*.h declares, and its
pure-host entry points (defaults, sweep budget) agree with the oracle.  No
device work is attempted here."""
import ctypes as ct
import os
import re

import pytest

import oracle as O
from paper_1805_06604_gb300 import build, nmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", fn)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        for m in re.finditer(r"\b(nmf_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ct.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert "nmf_create" in declared and "nmf_step" in declared and "nmf_solve" in declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(nmf.EXPORTED) <= declared


def test_defaults_are_the_papers_final_settings():
    p = nmf.nmf_params_default()
    assert (p.hp, p.beta0, p.eta, p.gamma, p.gamma_bar) == (3, 0.5, 1.5, 1.01, 1.005)
    assert p.lw == 0 and p.lh == 0 and p.alpha == 0.5 and p.project_w == 0


@pytest.mark.parametrize("m,n,K,r", [(200, 150, 30000, 10), (10000, 4000, 40_000_000, 50),
                                     (10304, 4000, 41_216_000, 64), (50000, 20000, 3_000_000, 30),
                                     (7, 3, 5, 1), (64, 2048, 100, 32)])
def test_sweep_counts_bit_exact_with_oracle(m, n, K, r):
    assert nmf.nmf_sweep_counts(m, n, K, r) == O.sweep_counts(m, n, K, r)


def test_version_and_error_string():
    assert "sm_103a" in nmf.nmf_version()
    with pytest.raises(nmf.NmfError) as ei:
        nmf.nmf_sweep_counts(0, 1, 1, 1)
    assert ei.value.status == nmf.NMF_EINVAL
    assert "nmf_sweep_counts" in nmf.nmf_last_error()


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    X = np.ones((4, 3), np.float32)
    with pytest.raises(nmf.NmfError) as ei:
        nmf.Solver(X, 2, np.ones((4, 2), np.float32), np.ones((2, 3), np.float32))
    assert ei.value.status == nmf.NMF_ECUDA


def test_optional_diagnostics_are_off_by_default(lib):
    p = nmf.nmf_params_default()
    assert p.line_search_trace == 0 and p.trace_capacity == 4096
    assert nmf.nmf_params_default(line_search_trace=1).line_search_trace == 1


def test_batch_per_instance_length_is_checked_before_any_device_call(lib):
    import numpy as np
    X = np.ones((8, 6), np.float32)
    W0, H0 = np.ones((8, 2), np.float32), np.ones((2, 6), np.float32)
    with pytest.raises(ValueError):
        nmf.Batch([(X, 2, W0, H0)] * 2, per_instance=[{}])
