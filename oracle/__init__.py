"""FP64 CPU oracle for E-A-HALS (Ang & Gillis, arXiv 1805.06604).

TEST INFRASTRUCTURE ONLY.  The library in ``paper_1805_06604_gb300`` never
imports this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` do.  The arithmetic lives in ``oracle.c``
(plain C, double precision); this module compiles it with gcc and marshals
numpy arrays through ctypes.

Parity status of each routine (what pins it) is listed in the test files
``tests/test_oracle_*.py``; every routine there has at least one pin.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

_DP = ct.POINTER(ct.c_double)


class _Matrix(ct.Structure):
    _fields_ = [("m", ct.c_int64), ("n", ct.c_int64), ("is_csr", ct.c_int),
                ("x", _DP), ("rowptr", ct.POINTER(ct.c_int64)),
                ("colidx", ct.POINTER(ct.c_int32)), ("val", _DP)]


class _Params(ct.Structure):
    _fields_ = [("hp", ct.c_int), ("beta0", ct.c_double), ("eta", ct.c_double),
                ("gamma", ct.c_double), ("gamma_bar", ct.c_double),
                ("lw", ct.c_int), ("lh", ct.c_int), ("project_w", ct.c_int),
                ("compare_prev", ct.c_int), ("nnls_exact", ct.c_int), ("delta", ct.c_double)]


class _Scalars(ct.Structure):
    _fields_ = [("beta", ct.c_double), ("beta_bar", ct.c_double),
                ("beta_prev", ct.c_double), ("e_last", ct.c_double),
                ("e_prev", ct.c_double), ("k", ct.c_int64), ("lh_used", ct.c_int),
                ("lw_used", ct.c_int)]


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ct.CDLL(build())
    vp = ct.c_void_p
    sig = {
        "orc_set_threads": (None, [ct.c_int]),
        "orc_get_threads": (ct.c_int, []),
        "orc_fro2": (ct.c_double, [vp]),
        "orc_wtx": (None, [vp, ct.c_int, _DP, _DP]),
        "orc_xht": (None, [vp, ct.c_int, _DP, _DP]),
        "orc_gram_w": (None, [ct.c_int64, ct.c_int, _DP, _DP]),
        "orc_gram_h": (None, [ct.c_int64, ct.c_int, _DP, _DP]),
        "orc_hals_row_h": (None, [ct.c_int64, ct.c_int, _DP, _DP, _DP, ct.c_int]),
        "orc_hals_col_w": (None, [ct.c_int64, ct.c_int, _DP, _DP, _DP, ct.c_int]),
        "orc_hals_sweeps_h": (None, [ct.c_int64, ct.c_int, _DP, _DP, _DP, ct.c_int]),
        "orc_hals_sweeps_w": (None, [ct.c_int64, ct.c_int, _DP, _DP, _DP, ct.c_int]),
        "orc_hals_sweeps_h_delta": (ct.c_int, [ct.c_int64, ct.c_int, _DP, _DP, _DP, ct.c_int,
                                               ct.c_double]),
        "orc_hals_sweeps_w_delta": (ct.c_int, [ct.c_int64, ct.c_int, _DP, _DP, _DP, ct.c_int,
                                               ct.c_double]),
        "orc_err2_expanded": (ct.c_double, [ct.c_double, ct.c_int64, ct.c_int, _DP, _DP, _DP]),
        "orc_err2_direct": (ct.c_double, [vp, ct.c_int, _DP, _DP]),
        "orc_sweep_counts": (None, [ct.c_int64, ct.c_int64, ct.c_int64, ct.c_int, ct.c_double,
                                    ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
        "orc_beta_update": (None, [vp, vp, ct.c_int]),
        "orc_eahals_init": (None, [vp, ct.c_int, _DP, _DP, _DP, _DP, vp, vp]),
        "orc_eahals_step": (None, [vp, ct.c_int, ct.c_double, _DP, _DP, _DP, _DP, vp, vp,
                                   ct.c_int, _DP, _DP, ct.POINTER(ct.c_int), _DP]),
        "orc_line_search_beta": (ct.c_double, [vp, ct.c_int, _DP, _DP, _DP]),
        "orc_nnls": (ct.c_int, [ct.c_int, _DP, _DP, _DP, ct.c_int]),
        "orc_nnls_h": (ct.c_int, [ct.c_int64, ct.c_int, _DP, _DP, _DP]),
        "orc_nnls_w": (ct.c_int, [ct.c_int64, ct.c_int, _DP, _DP, _DP]),
        "orc_eahals_run": (None, [vp, ct.c_int, _DP, _DP, _DP, _DP, vp, vp, ct.c_int,
                                  ct.POINTER(ct.c_int8), _DP, _DP, ct.POINTER(ct.c_uint8)]),
        "orc_ahals_run": (None, [vp, ct.c_int, _DP, _DP, ct.c_int, ct.c_int, ct.c_int, _DP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


class Matrix:
    """X as the oracle sees it: dense (m x n, row-major) or CSR."""

    def __init__(self, dense=None, *, m=None, n=None, rowptr=None, colidx=None, val=None):
        if dense is not None:
            self.dense = _f64(dense)
            self.m, self.n = self.dense.shape
            self.is_csr = False
            self.nnz = self.m * self.n
        else:
            self.m, self.n = int(m), int(n)
            self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
            self.val = _f64(val)
            self.is_csr = True
            self.nnz = int(self.rowptr[-1])
        s = _Matrix()
        s.m, s.n, s.is_csr = self.m, self.n, int(self.is_csr)
        if self.is_csr:
            s.rowptr = self.rowptr.ctypes.data_as(ct.POINTER(ct.c_int64))
            s.colidx = self.colidx.ctypes.data_as(ct.POINTER(ct.c_int32))
            s.val = _ptr(self.val)
        else:
            s.x = _ptr(self.dense)
        self._s = s

    @property
    def ref(self):
        return ct.byref(self._s)

    @classmethod
    def from_any(cls, X) -> "Matrix":
        if isinstance(X, Matrix):
            return X
        if hasattr(X, "indptr"):  # scipy.sparse CSR
            return cls(m=X.shape[0], n=X.shape[1], rowptr=X.indptr, colidx=X.indices, val=X.data)
        return cls(np.asarray(X))


@dataclass
class Params:
    hp: int = 3
    beta0: float = 0.5
    eta: float = 1.5
    gamma: float = 1.01
    gamma_bar: float = 1.005
    lw: int = 1
    lh: int = 1
    project_w: int = 0
    compare_prev: int = 1        # 1: restart iff e(k) > e(k-1) (Alg. 2 step 16)
    nnls_exact: int = 0          # 1: ANLS / E-ANLS (exact NNLS subproblems)
    delta: float = 0.0           # > 0: the A-HALS inner stopping rule

    def c(self) -> _Params:
        return _Params(self.hp, self.beta0, self.eta, self.gamma, self.gamma_bar,
                       self.lw, self.lh, self.project_w, self.compare_prev, self.nnls_exact,
                       self.delta)


@dataclass
class Scalars:
    beta: float = 0.0
    beta_bar: float = 1.0
    beta_prev: float = 0.0
    e_last: float = 0.0
    e_prev: float = 0.0
    k: int = 0
    lh_used: int = 0
    lw_used: int = 0

    def c(self) -> _Scalars:
        return _Scalars(self.beta, self.beta_bar, self.beta_prev, self.e_last, self.e_prev, self.k,
                        self.lh_used, self.lw_used)

    def load(self, s: _Scalars) -> "Scalars":
        self.beta, self.beta_bar, self.beta_prev = s.beta, s.beta_bar, s.beta_prev
        self.e_last, self.e_prev, self.k = s.e_last, s.e_prev, s.k
        self.lh_used, self.lw_used = s.lh_used, s.lw_used
        return self


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (results do not depend on it)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def fro2(X) -> float:
    return _load().orc_fro2(Matrix.from_any(X).ref)


def wtx(X, W) -> np.ndarray:
    X = Matrix.from_any(X)
    W = _f64(W)
    r = W.shape[1]
    A = np.zeros((r, X.n))
    _load().orc_wtx(X.ref, r, _ptr(W), _ptr(A))
    return A


def xht(X, H) -> np.ndarray:
    X = Matrix.from_any(X)
    H = _f64(H)
    r = H.shape[0]
    C = np.zeros((X.m, r))
    _load().orc_xht(X.ref, r, _ptr(H), _ptr(C))
    return C


def gram_w(W) -> np.ndarray:
    W = _f64(W)
    G = np.zeros((W.shape[1], W.shape[1]))
    _load().orc_gram_w(W.shape[0], W.shape[1], _ptr(W), _ptr(G))
    return G


def gram_h(H) -> np.ndarray:
    H = _f64(H)
    D = np.zeros((H.shape[0], H.shape[0]))
    _load().orc_gram_h(H.shape[1], H.shape[0], _ptr(H), _ptr(D))
    return D


def hals_row_h(A, G, H, k) -> np.ndarray:
    A, G, H = _f64(A), _f64(G), _f64(H).copy()
    _load().orc_hals_row_h(H.shape[1], H.shape[0], _ptr(A), _ptr(G), _ptr(H), int(k))
    return H


def hals_col_w(C, D, W, k) -> np.ndarray:
    C, D, W = _f64(C), _f64(D), _f64(W).copy()
    _load().orc_hals_col_w(W.shape[0], W.shape[1], _ptr(C), _ptr(D), _ptr(W), int(k))
    return W


def hals_sweeps_h(A, G, H, sweeps) -> np.ndarray:
    A, G, H = _f64(A), _f64(G), _f64(H).copy()
    _load().orc_hals_sweeps_h(H.shape[1], H.shape[0], _ptr(A), _ptr(G), _ptr(H), int(sweeps))
    return H


def hals_sweeps_h_delta(A, G, H, max_sweeps, delta):
    """A-HALS sweeps with the inner stopping rule; returns (H, sweeps done)."""
    A, G, H = _f64(A), _f64(G), _f64(H).copy()
    used = _load().orc_hals_sweeps_h_delta(H.shape[1], H.shape[0], _ptr(A), _ptr(G), _ptr(H),
                                           int(max_sweeps), float(delta))
    return H, used


def hals_sweeps_w_delta(C, D, W, max_sweeps, delta):
    """The W side of the inner stopping rule; returns (W, sweeps done)."""
    C, D, W = _f64(C), _f64(D), _f64(W).copy()
    used = _load().orc_hals_sweeps_w_delta(W.shape[0], W.shape[1], _ptr(C), _ptr(D), _ptr(W),
                                           int(max_sweeps), float(delta))
    return W, used


def hals_sweeps_w(C, D, W, sweeps) -> np.ndarray:
    C, D, W = _f64(C), _f64(D), _f64(W).copy()
    _load().orc_hals_sweeps_w(W.shape[0], W.shape[1], _ptr(C), _ptr(D), _ptr(W), int(sweeps))
    return W


def err2_expanded(fro2_x: float, W, C, D) -> float:
    W, C, D = _f64(W), _f64(C), _f64(D)
    return _load().orc_err2_expanded(float(fro2_x), W.shape[0], W.shape[1], _ptr(W), _ptr(C), _ptr(D))


def err2_direct(X, W, H) -> float:
    X = Matrix.from_any(X)
    W, H = _f64(W), _f64(H)
    return _load().orc_err2_direct(X.ref, W.shape[1], _ptr(W), _ptr(H))


def sweep_counts(m: int, n: int, K: int, r: int, alpha: float = 0.5):
    lw, lh = ct.c_int(), ct.c_int()
    _load().orc_sweep_counts(int(m), int(n), int(K), int(r), float(alpha), ct.byref(lw), ct.byref(lh))
    return lw.value, lh.value


def beta_update(p: Params, s: Scalars, decreased: bool) -> Scalars:
    pc, sc = p.c(), s.c()
    _load().orc_beta_update(ct.byref(pc), ct.byref(sc), int(bool(decreased)))
    return Scalars().load(sc)


class State:
    """Full E-A-HALS state (W, H, W_y, H_y and the Algorithm 3 scalars)."""

    def __init__(self, W, H, Wy=None, Hy=None, scalars: Scalars | None = None):
        self.W = _f64(W).copy()
        self.H = _f64(H).copy()
        self.Wy = _f64(W if Wy is None else Wy).copy()
        self.Hy = _f64(H if Hy is None else Hy).copy()
        self.s = scalars if scalars is not None else Scalars()

    def copy(self) -> "State":
        return State(self.W, self.H, self.Wy, self.Hy, Scalars(**vars(self.s)))


def eahals_init(X, W0, H0, p: Params) -> State:
    X = Matrix.from_any(X)
    st = State(W0, H0)
    sc = st.s.c()
    pc = p.c()
    _load().orc_eahals_init(X.ref, st.W.shape[1], _ptr(st.W), _ptr(st.H), _ptr(st.Wy),
                            _ptr(st.Hy), ct.byref(pc), ct.byref(sc))
    st.s.load(sc)
    return st


def eahals_step(X, st: State, p: Params, force: int = -1, fro2_x: float | None = None,
                line_search: bool = False):
    """One outer iteration in place on ``st``; returns (e_k, beta_k, accepted),
    and the line-search step beta* of Sec. 3 as a fourth value when
    ``line_search``."""
    X = Matrix.from_any(X)
    if fro2_x is None:
        fro2_x = fro2(X)
    sc, pc = st.s.c(), p.c()
    e, b, acc, bs = ct.c_double(), ct.c_double(), ct.c_int(), ct.c_double()
    _load().orc_eahals_step(X.ref, st.W.shape[1], float(fro2_x), _ptr(st.W), _ptr(st.H),
                            _ptr(st.Wy), _ptr(st.Hy), ct.byref(pc), ct.byref(sc), int(force),
                            ct.byref(e), ct.byref(b), ct.byref(acc),
                            ct.byref(bs) if line_search else None)
    st.s.load(sc)
    if line_search:
        return e.value, b.value, bool(acc.value), bs.value
    return e.value, b.value, bool(acc.value)


def nnls(G, b, x0=None, max_iter: int | None = None):
    """Exact min_{x>=0} 1/2 x^T G x - b^T x (block principal pivoting);
    returns (x, exchanges) -- exchanges is -1 on failure."""
    G = _f64(G)
    b = _f64(b)
    r = b.shape[0]
    x = np.zeros(r) if x0 is None else _f64(x0).copy()
    it = _load().orc_nnls(r, _ptr(G), _ptr(b), _ptr(x), 100 * (r + 1) if max_iter is None
                          else int(max_iter))
    return x, it


def nnls_h(A, G, H):
    """Every column of H solved exactly (warm start: H); returns (H, worst)."""
    A, G = _f64(A), _f64(G)
    H = _f64(H).copy()
    st = _load().orc_nnls_h(H.shape[1], H.shape[0], _ptr(A), _ptr(G), _ptr(H))
    return H, st


def nnls_w(C, D, W):
    """Every row of W solved exactly (warm start: W); returns (W, worst)."""
    C, D = _f64(C), _f64(D)
    W = _f64(W).copy()
    st = _load().orc_nnls_w(W.shape[0], W.shape[1], _ptr(C), _ptr(D), _ptr(W))
    return W, st


def line_search_beta(X, W, Wn, Hy) -> float:
    """beta* = <X - Wn Hy, (Wn - W) Hy> / ||(Wn - W) Hy||_F^2 (Sec. 3)."""
    X = Matrix.from_any(X)
    W, Wn, Hy = _f64(W), _f64(Wn), _f64(Hy)
    return _load().orc_line_search_beta(X.ref, W.shape[1], _ptr(W), _ptr(Wn), _ptr(Hy))


def eahals_run(X, st: State, p: Params, iters: int, forced=None):
    """``iters`` outer iterations in place; returns (trace_e, trace_beta, trace_acc)."""
    X = Matrix.from_any(X)
    te, tb = np.zeros(iters), np.zeros(iters)
    ta = np.zeros(iters, dtype=np.uint8)
    fp = None
    if forced is not None:
        forced = np.ascontiguousarray(forced, dtype=np.int8)
        fp = forced.ctypes.data_as(ct.POINTER(ct.c_int8))
    sc, pc = st.s.c(), p.c()
    _load().orc_eahals_run(X.ref, st.W.shape[1], _ptr(st.W), _ptr(st.H), _ptr(st.Wy), _ptr(st.Hy),
                           ct.byref(pc), ct.byref(sc), int(iters), fp, _ptr(te), _ptr(tb),
                           ta.ctypes.data_as(ct.POINTER(ct.c_uint8)))
    st.s.load(sc)
    return te, tb, ta.astype(bool)


def ahals_run(X, W0, H0, lw: int, lh: int, iters: int):
    """Un-extrapolated A-HALS; returns (W, H, trace_e)."""
    X = Matrix.from_any(X)
    W, H = _f64(W0).copy(), _f64(H0).copy()
    te = np.zeros(iters)
    _load().orc_ahals_run(X.ref, W.shape[1], _ptr(W), _ptr(H), int(lw), int(lh), int(iters), _ptr(te))
    return W, H, te
