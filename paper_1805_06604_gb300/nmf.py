"""ctypes binding of libnmf_gb300 (include/nmf.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch tensors into pointers and sizes and raises ``NmfError`` on a
non-OK status.  If the shared library has not been built the first call
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

NMF_OK, NMF_EINVAL, NMF_ENOMEM, NMF_ECUDA, NMF_ENONFINITE, NMF_ETIMEOUT, NMF_ENOTSUP = range(7)
NMF_DENSE, NMF_CSR = 0, 1
NMF_PREC_FP32, NMF_PREC_TF32, NMF_PREC_BF16X3 = 0, 1, 2
STATUS_NAMES = ["NMF_OK", "NMF_EINVAL", "NMF_ENOMEM", "NMF_ECUDA", "NMF_ENONFINITE",
                "NMF_ETIMEOUT", "NMF_ENOTSUP"]


class NmfError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


class nmf_matrix(ct.Structure):
    _fields_ = [("format", ct.c_int32), ("on_device", ct.c_int32), ("m", ct.c_int64),
                ("n", ct.c_int64), ("ld", ct.c_int64), ("nnz", ct.c_int64),
                ("values", ct.c_void_p), ("rowptr", ct.c_void_p), ("colidx", ct.c_void_p)]


class nmf_params(ct.Structure):
    _fields_ = [("hp", ct.c_int32), ("beta0", ct.c_double), ("eta", ct.c_double),
                ("gamma", ct.c_double), ("gamma_bar", ct.c_double), ("lw", ct.c_int32),
                ("lh", ct.c_int32), ("alpha", ct.c_double), ("project_w", ct.c_int32),
                ("compare_prev", ct.c_int32), ("precision", ct.c_int32),
                ("trace_capacity", ct.c_int64), ("line_search_trace", ct.c_int32),
                ("delta", ct.c_double), ("exact_nnls", ct.c_int32)]


class nmf_info(ct.Structure):
    _fields_ = [("k", ct.c_int64), ("e_last", ct.c_double), ("e_k", ct.c_double),
                ("fro2", ct.c_double), ("relerr", ct.c_double), ("beta", ct.c_double),
                ("beta_bar", ct.c_double), ("beta_prev", ct.c_double), ("accepted", ct.c_int32),
                ("lw", ct.c_int32), ("lh", ct.c_int32), ("device_status", ct.c_int32),
                ("launches_per_iter", ct.c_int32), ("lh_used", ct.c_int32),
                ("lw_used", ct.c_int32), ("exact_failed", ct.c_int32)]


class nmf_result(ct.Structure):
    _fields_ = [("iters", ct.c_int64), ("relerr", ct.c_double), ("relerr_last", ct.c_double),
                ("seconds", ct.c_double), ("reached", ct.c_int32), ("timed_out", ct.c_int32)]


class nmf_scalars(ct.Structure):
    _fields_ = [("beta", ct.c_double), ("beta_bar", ct.c_double), ("beta_prev", ct.c_double),
                ("e_last", ct.c_double), ("e_prev", ct.c_double), ("k", ct.c_int64)]


class nmf_batch_plan(ct.Structure):
    _fields_ = [("grouped", ct.c_int32), ("branches", ct.c_int32),
                ("h_cols_per_cta", ct.c_int32), ("launches_per_iter", ct.c_int32),
                ("ms_per_iter", ct.c_double)]


_lib = None
_SIGS = {
    "nmf_params_default": [ct.POINTER(nmf_params)],
    "nmf_sweep_counts": [ct.c_int64, ct.c_int64, ct.c_int64, ct.c_int32, ct.c_double,
                         ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)],
    "nmf_create": [ct.POINTER(ct.c_void_p), ct.POINTER(nmf_matrix), ct.c_int32, ct.c_void_p,
                   ct.c_void_p, ct.c_int32, ct.POINTER(nmf_params), ct.c_void_p],
    "nmf_step": [ct.c_void_p, ct.c_int32, ct.c_void_p],
    "nmf_solve": [ct.c_void_p, ct.c_int64, ct.c_double, ct.c_double, ct.c_int32,
                  ct.POINTER(nmf_result)],
    "nmf_eval_error": [ct.c_void_p, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)],
    "nmf_set_forced_decisions": [ct.c_void_p, ct.c_void_p, ct.c_int64],
    "nmf_get_info": [ct.c_void_p, ct.POINTER(nmf_info)],
    "nmf_get_factors": [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int32],
    "nmf_get_extrapolated": [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int32],
    "nmf_get_trace": [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64,
                      ct.POINTER(ct.c_int64)],
    "nmf_get_state": [ct.c_void_p, ct.POINTER(nmf_scalars), ct.c_void_p, ct.c_void_p,
                      ct.c_void_p, ct.c_void_p, ct.c_int32],
    "nmf_set_state": [ct.c_void_p, ct.POINTER(nmf_scalars), ct.c_void_p, ct.c_void_p,
                      ct.c_void_p, ct.c_void_p, ct.c_int32],
    "nmf_profile_phases": [ct.c_void_p, ct.c_int32, ct.c_void_p],
    "nmf_matmul_nt": [ct.c_void_p, ct.c_int64, ct.c_int64, ct.c_int64, ct.c_void_p, ct.c_int32,
                      ct.c_int64, ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_void_p],
    "nmf_fro2_noalloc": [ct.c_void_p, ct.c_int64, ct.c_int64, ct.c_int64, ct.c_void_p,
                         ct.c_void_p],
    "nmf_destroy": [ct.c_void_p],
    "nmf_debug_set_fixup_stall": [ct.c_int32],
    "nmf_batch_create": [ct.POINTER(ct.c_void_p), ct.c_int32, ct.c_void_p, ct.c_void_p,
                         ct.c_void_p, ct.c_void_p, ct.c_int32, ct.POINTER(nmf_params),
                         ct.c_void_p],
    "nmf_get_line_search_trace": [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.POINTER(ct.c_int64)],
    "nmf_batch_create_params": [ct.POINTER(ct.c_void_p), ct.c_int32, ct.c_void_p, ct.c_void_p,
                                ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p,
                                ct.c_void_p],
    "nmf_batch_step": [ct.c_void_p, ct.c_int32],
    "nmf_batch_step_loop": [ct.c_void_p, ct.c_int32],
    "nmf_batch_get_info": [ct.c_void_p, ct.c_int32, ct.POINTER(nmf_info)],
    "nmf_batch_get_factors": [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_int32],
    "nmf_batch_schedule": [ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_double)],
    "nmf_batch_get_plan": [ct.c_void_p, ct.POINTER(nmf_batch_plan)],
    "nmf_batch_set_plan": [ct.c_void_p, ct.POINTER(nmf_batch_plan)],
    "nmf_batch_destroy": [ct.c_void_p],
}
PHASES = ["gram_w", "wtx", "hals_h", "gram_h", "xht", "hals_w", "finalize"]
EXPORTED = sorted(list(_SIGS) + ["nmf_last_error", "nmf_version"])


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None) -> ct.CDLL:
    """Loads the built library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1805_06604_gb300.build` (no CPU fallback exists)")
    lib = ct.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ct.c_int
    lib.nmf_last_error.restype = ct.c_char_p
    lib.nmf_last_error.argtypes = []
    lib.nmf_version.restype = ct.c_char_p
    lib.nmf_version.argtypes = []
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != NMF_OK:
        raise NmfError(status, where, load().nmf_last_error().decode())


def nmf_last_error() -> str:
    return load().nmf_last_error().decode()


def nmf_version() -> str:
    return load().nmf_version().decode()


def nmf_params_default(**overrides) -> nmf_params:
    p = nmf_params()
    _check(load().nmf_params_default(ct.byref(p)), "nmf_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def nmf_sweep_counts(m: int, n: int, K: int, r: int, alpha: float = 0.5):
    lw, lh = ct.c_int32(), ct.c_int32()
    _check(load().nmf_sweep_counts(m, n, K, r, alpha, ct.byref(lw), ct.byref(lh)),
           "nmf_sweep_counts")
    return lw.value, lh.value


# ------------------------------------------------------------------ helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr_and_dev(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if _is_torch(x):
        import torch
        want = {np.float32: torch.float32, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return x.data_ptr(), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class _Keep:
    items: list


def make_matrix(X=None, *, csr=None, m=None, n=None):
    """nmf_matrix for a dense X (m x n) or csr=(rowptr, colidx, values)."""
    keep = []
    mat = nmf_matrix()
    if csr is not None:
        rowptr, colidx, vals = csr
        pr, dr, k1 = _ptr_and_dev(rowptr, np.int64)
        pc, dc, k2 = _ptr_and_dev(colidx, np.int32)
        pv, dv, k3 = _ptr_and_dev(vals, np.float32)
        if not (dr == dc == dv):
            raise ValueError("CSR arrays must all be on the host or all on the device")
        keep += [k1, k2, k3]
        mat.format, mat.on_device = NMF_CSR, dv
        mat.m, mat.n, mat.ld = int(m), int(n), 0
        mat.nnz = int(len(vals)) if not _is_torch(vals) else int(vals.numel())
        mat.values, mat.rowptr, mat.colidx = pv, pr, pc
    else:
        pv, dv, k = _ptr_and_dev(X, np.float32)
        keep.append(k)
        mat.format, mat.on_device = NMF_DENSE, dv
        mat.m, mat.n = int(X.shape[0]), int(X.shape[1])
        mat.ld, mat.nnz = int(X.shape[1]), int(X.shape[0]) * int(X.shape[1])
        mat.values = pv
    return mat, _Keep(keep)


def nmf_create(X=None, r: int = 1, W0=None, H0=None, params: nmf_params | None = None,
               stream=None, *, csr=None, m=None, n=None):
    """Returns a handle (c_void_p).  X: dense numpy/torch (m x n) or csr=(...)."""
    mat, keep = make_matrix(X, csr=csr, m=m, n=n)
    pw, dw, kw = _ptr_and_dev(W0, np.float32)
    ph, dh, kh = _ptr_and_dev(H0, np.float32)
    if dw != dh:
        raise ValueError("W0 and H0 must both be on the host or both on the device")
    h = ct.c_void_p()
    p = params if params is not None else nmf_params_default()
    _check(load().nmf_create(ct.byref(h), ct.byref(mat), int(r), pw, ph, dw, ct.byref(p),
                             _stream_ptr(stream)), "nmf_create")
    del keep, kw, kh
    return h


def nmf_step(h, iters: int = 1, last: bool = False):
    """Enqueues `iters` iterations; with last=True also synchronises and
    returns the nmf_info of the last one."""
    info = nmf_info() if last else None
    _check(load().nmf_step(h, int(iters), ct.byref(info) if last else None), "nmf_step")
    return info


def nmf_solve(h, max_iters: int, target_relerr: float = 0.0, max_seconds: float = 0.0,
              check_every: int = 10) -> nmf_result:
    res = nmf_result()
    _check(load().nmf_solve(h, int(max_iters), float(target_relerr), float(max_seconds),
                            int(check_every), ct.byref(res)), "nmf_solve")
    return res


def nmf_eval_error(h):
    """(||X - WH||_F, relative error) of the pair (W, H) the handle returns."""
    e, rel = ct.c_double(), ct.c_double()
    _check(load().nmf_eval_error(h, ct.byref(e), ct.byref(rel)), "nmf_eval_error")
    return e.value, rel.value


def nmf_set_forced_decisions(h, accepted):
    """Decision replay: iteration k takes accepted[k] (bool) instead of the
    restart test; an empty sequence clears it."""
    a = np.ascontiguousarray(np.asarray(accepted, dtype=np.uint8))
    _check(load().nmf_set_forced_decisions(h, a.ctypes.data if a.size else None, int(a.size)),
           "nmf_set_forced_decisions")


def nmf_get_info(h) -> nmf_info:
    info = nmf_info()
    _check(load().nmf_get_info(h, ct.byref(info)), "nmf_get_info")
    return info


def _out_pair(W, H):
    pw, dw, _ = _ptr_and_dev(W, np.float32) if W is not None else (None, 0, None)
    ph, dh, _ = _ptr_and_dev(H, np.float32) if H is not None else (None, 0, None)
    if W is not None and H is not None and dw != dh:
        raise ValueError("outputs must both be host or both device")
    return pw, ph, (dw if W is not None else dh)


def nmf_get_factors(h, W, H):
    """Copies the accepted (W, H) into W (m x r) and H (r x n) (numpy or torch)."""
    pw, ph, dev = _out_pair(W, H)
    _check(load().nmf_get_factors(h, pw, ph, dev), "nmf_get_factors")


def nmf_get_extrapolated(h, Wy, Hy):
    pw, ph, dev = _out_pair(Wy, Hy)
    _check(load().nmf_get_extrapolated(h, pw, ph, dev), "nmf_get_extrapolated")


def nmf_get_trace(h, cap: int):
    e = np.zeros(cap)
    b = np.zeros(cap)
    a = np.zeros(cap, dtype=np.uint8)
    ln = ct.c_int64()
    _check(load().nmf_get_trace(h, e.ctypes.data, b.ctypes.data, a.ctypes.data, cap,
                                ct.byref(ln)), "nmf_get_trace")
    n = ln.value
    return e[:n], b[:n], a[:n].astype(bool)


def nmf_get_state(h, W, H, Wy, Hy) -> nmf_scalars:
    s = nmf_scalars()
    ptrs = [_ptr_and_dev(x, np.float32) for x in (W, H, Wy, Hy)]
    dev = ptrs[0][1]
    _check(load().nmf_get_state(h, ct.byref(s), *[p[0] for p in ptrs], dev), "nmf_get_state")
    return s


def nmf_set_state(h, s: nmf_scalars, W, H, Wy, Hy):
    ptrs = [_ptr_and_dev(x, np.float32) for x in (W, H, Wy, Hy)]
    devs = {p[1] for p in ptrs}
    if len(devs) != 1:
        raise ValueError("all four factors must be host or all device")
    _check(load().nmf_set_state(h, ct.byref(s), *[p[0] for p in ptrs], devs.pop()),
           "nmf_set_state")
    del ptrs


def nmf_profile_phases(h, iters: int) -> dict:
    """Mean device milliseconds per phase over `iters` real (ungraphed) iterations."""
    ms = np.zeros(len(PHASES))
    _check(load().nmf_profile_phases(h, int(iters), ms.ctypes.data), "nmf_profile_phases")
    return dict(zip(PHASES, ms.tolist()))


def nmf_matmul_nt(P, Q, out, precision, stream=None):
    """out = P Q^T on the tensor cores for CUDA float32 tensors P (M x K),
    Q (q x K) and out (M x q); row strides must be multiples of 8."""
    for t in (P, Q, out):
        if not (_is_torch(t) and t.is_cuda and t.stride(1) == 1):
            raise TypeError("P, Q, out must be CUDA tensors with unit column stride")
    _check(load().nmf_matmul_nt(P.data_ptr(), P.shape[0], P.shape[1], P.stride(0), Q.data_ptr(),
                                Q.shape[0], Q.stride(0), out.data_ptr(), out.stride(0),
                                int(precision), _stream_ptr(stream)), "nmf_matmul_nt")


def nmf_fro2_noalloc(X, out, stream=None):
    """||X||_F^2 of a CUDA float32 tensor X (m x n, rows may be strided) into
    the CUDA float64 tensor `out` (one element), with no device allocation."""
    if not (_is_torch(X) and X.is_cuda and _is_torch(out) and out.is_cuda):
        raise TypeError("X and out must be CUDA tensors")
    import torch
    if X.dtype != torch.float32 or X.dim() != 2 or X.stride(1) != 1:
        raise TypeError("X must be a 2-D float32 tensor with unit column stride")
    if out.dtype != torch.float64 or out.numel() < 1:
        raise TypeError("out must hold at least one float64")
    _check(load().nmf_fro2_noalloc(X.data_ptr(), X.shape[0], X.shape[1], X.stride(0),
                                   out.data_ptr(), _stream_ptr(stream)), "nmf_fro2_noalloc")


def nmf_debug_set_fixup_stall(extra: int):
    """Failure-detection hook: make the tensor-core product's bounded fix-up
    wait run out (extra > 0) or restore normal operation (0)."""
    _check(load().nmf_debug_set_fixup_stall(int(extra)), "nmf_debug_set_fixup_stall")


def nmf_destroy(h):
    if h is not None and h.value:
        _check(load().nmf_destroy(h), "nmf_destroy")
        h.value = None


class Batch:
    """Many independent instances (host numpy inputs): one graph per iteration."""

    def __init__(self, problems, stream=None, per_instance=None, **params):
        """problems: list of (X m x n float32, r, W0 m x r, H0 r x n).
        per_instance: optional list (one dict per problem) of parameter
        overrides applied on top of **params (nmf_batch_create_params)."""
        self.params = nmf_params_default(**params)
        n = len(problems)
        plist = None
        if per_instance is not None:
            if len(per_instance) != n:
                raise ValueError("per_instance needs one entry per problem")
            plist = (nmf_params * n)()
            for i, over in enumerate(per_instance):
                plist[i] = nmf_params_default(**{**params, **over})
        mats = (nmf_matrix * n)()
        self._keep = []
        ranks = (ct.c_int32 * n)()
        w0 = (ct.c_void_p * n)()
        h0 = (ct.c_void_p * n)()
        self.shapes = []
        for i, (X, r, W0, H0) in enumerate(problems):
            m, k = make_matrix(X)
            mats[i] = m
            self._keep.append(k)
            pw, _, kw = _ptr_and_dev(W0, np.float32)
            ph, _, kh = _ptr_and_dev(H0, np.float32)
            self._keep += [kw, kh]
            w0[i], h0[i] = pw, ph
            ranks[i] = int(r)
            self.shapes.append((int(X.shape[0]), int(X.shape[1]), int(r)))
        self.h = ct.c_void_p()
        if plist is None:
            _check(load().nmf_batch_create(ct.byref(self.h), n, mats, ranks, w0, h0, 0,
                                           ct.byref(self.params), _stream_ptr(stream)),
                   "nmf_batch_create")
        else:
            _check(load().nmf_batch_create_params(ct.byref(self.h), n, mats, ranks, w0, h0, 0,
                                                  ct.cast(plist, ct.c_void_p),
                                                  _stream_ptr(stream)),
                   "nmf_batch_create_params")
        self._keep = None

    def step(self, iters=1):
        _check(load().nmf_batch_step(self.h, int(iters)), "nmf_batch_step")

    def step_loop(self, iters=1):
        _check(load().nmf_batch_step_loop(self.h, int(iters)), "nmf_batch_step_loop")

    def info(self, i) -> nmf_info:
        out = nmf_info()
        _check(load().nmf_batch_get_info(self.h, int(i), ct.byref(out)), "nmf_batch_get_info")
        return out

    def factors(self, i):
        m, n, r = self.shapes[i]
        W = np.zeros((m, r), np.float32)
        H = np.zeros((r, n), np.float32)
        _check(load().nmf_batch_get_factors(self.h, int(i), W.ctypes.data, H.ctypes.data, 0),
               "nmf_batch_get_factors")
        return W, H

    def schedule(self):
        b, ms = ct.c_int32(), ct.c_double()
        _check(load().nmf_batch_schedule(self.h, ct.byref(b), ct.byref(ms)), "nmf_batch_schedule")
        return b.value, ms.value

    def plan(self) -> nmf_batch_plan:
        out = nmf_batch_plan()
        _check(load().nmf_batch_get_plan(self.h, ct.byref(out)), "nmf_batch_get_plan")
        return out

    def set_plan(self, grouped, branches, h_cols_per_cta=0):
        pl = nmf_batch_plan(int(grouped), int(branches), int(h_cols_per_cta), 0, 0.0)
        _check(load().nmf_batch_set_plan(self.h, ct.byref(pl)), "nmf_batch_set_plan")

    def close(self):
        if self.h is not None and self.h.value:
            _check(load().nmf_batch_destroy(self.h), "nmf_batch_destroy")
            self.h.value = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Solver:
    """Owns one nmf_handle: numpy in, numpy out (host buffers)."""

    def __init__(self, X=None, r: int = 1, W0=None, H0=None, stream=None, *, csr=None, m=None,
                 n=None, **params):
        self.params = nmf_params_default(**params)
        if csr is not None:
            self.m, self.n = int(m), int(n)
        else:
            self.m, self.n = int(X.shape[0]), int(X.shape[1])
        self.r = int(r)
        self.h = nmf_create(X, r, W0, H0, self.params, stream, csr=csr, m=m, n=n)

    def step(self, iters: int = 1, last: bool = False):
        return nmf_step(self.h, iters, last)

    def solve(self, max_iters, target_relerr=0.0, max_seconds=0.0, check_every=10):
        return nmf_solve(self.h, max_iters, target_relerr, max_seconds, check_every)

    def eval_error(self):
        return nmf_eval_error(self.h)

    def force_decisions(self, accepted):
        nmf_set_forced_decisions(self.h, accepted)

    def info(self) -> nmf_info:
        return nmf_get_info(self.h)

    def factors(self):
        W = np.zeros((self.m, self.r), np.float32)
        H = np.zeros((self.r, self.n), np.float32)
        nmf_get_factors(self.h, W, H)
        return W, H

    def extrapolated(self):
        W = np.zeros((self.m, self.r), np.float32)
        H = np.zeros((self.r, self.n), np.float32)
        nmf_get_extrapolated(self.h, W, H)
        return W, H

    def trace(self, cap=None):
        if cap is None:
            cap = int(self.info().k)
        return nmf_get_trace(self.h, cap)

    def line_search_trace(self, cap=None):
        """beta* of Sec. 3 for every iteration's W-update (needs
        line_search_trace=1 at creation)."""
        if cap is None:
            cap = int(self.info().k)
        out = np.zeros(cap)
        ln = ct.c_int64()
        _check(load().nmf_get_line_search_trace(self.h, out.ctypes.data, cap, ct.byref(ln)),
               "nmf_get_line_search_trace")
        return out[:ln.value]

    def get_state(self):
        W = np.zeros((self.m, self.r), np.float32)
        H = np.zeros((self.r, self.n), np.float32)
        Wy = np.zeros_like(W)
        Hy = np.zeros_like(H)
        s = nmf_get_state(self.h, W, H, Wy, Hy)
        return s, W, H, Wy, Hy

    def set_state(self, s: nmf_scalars, W, H, Wy, Hy):
        nmf_set_state(self.h, s, W, H, Wy, Hy)

    def profile_phases(self, iters: int = 3) -> dict:
        return nmf_profile_phases(self.h, iters)

    def close(self):
        nmf_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
