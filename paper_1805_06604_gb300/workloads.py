"""Seeded synthetic inputs for E-A-HALS.

This module only draws data; it holds none of the factorization's
arithmetic.  The same arrays feed the FP64 oracle (widened to float64) and
the CUDA path, so both sides always see identical inputs.

All draws use ``numpy.random.Generator(PCG64(seed))``.  Products W0 @ H0 are
accumulated as a fixed sequence of elementwise rank-1 updates in float64, so
the data are bit-identical on x86-64 and aarch64 (no BLAS summation order).

Workloads (the paper's data sets are not available; these stand in for
them with the shapes and structure of Sec. 4.1):

* ``low_rank``     -- X = W0 H0 with U[0,1] factors (the "low-rank synthetic"
  data of Sec. 4.1), optionally with additive Gaussian noise.
* ``full_rank``    -- X with i.i.d. U[0,1] entries (the "full-rank synthetic"
  data of Sec. 4.1).
* ``image_like``   -- columns are nonnegative mixtures of smooth 2-D Gaussian
  blobs on a 112 x 92 pixel grid (the ORL/Umist image size of Table 1).
* ``document_like``-- a sparse term-document matrix: Zipf term frequencies,
  lognormal document lengths, log(1+count) * idf values (Table 2's shape).
* ``batch``        -- many small uneven low-rank instances.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _outer_sum(W0: np.ndarray, H0: np.ndarray) -> np.ndarray:
    """W0 @ H0 in float64 as sum_k W0[:,k] H0[k,:], k ascending."""
    W0 = np.asarray(W0, dtype=np.float64)
    H0 = np.asarray(H0, dtype=np.float64)
    X = np.zeros((W0.shape[0], H0.shape[1]))
    tmp = np.empty_like(X)
    for k in range(W0.shape[1]):
        np.multiply(W0[:, k:k + 1], H0[k:k + 1, :], out=tmp)
        X += tmp
    return X


@dataclass
class Problem:
    """One NMF instance: X (dense m x n or CSR), rank r, initial W0, H0."""
    name: str
    m: int
    n: int
    r: int
    W0: np.ndarray                       # m x r, initial W (>= 0)
    H0: np.ndarray                       # r x n, initial H (>= 0)
    X: np.ndarray | None = None          # dense m x n, row-major
    rowptr: np.ndarray | None = None     # CSR (int64, m+1)
    colidx: np.ndarray | None = None     # CSR (int32, nnz)
    val: np.ndarray | None = None        # CSR values
    meta: dict = field(default_factory=dict)

    @property
    def is_csr(self) -> bool:
        return self.rowptr is not None

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if self.is_csr else self.m * self.n

    def dense(self) -> np.ndarray:
        if not self.is_csr:
            return self.X
        D = np.zeros((self.m, self.n), dtype=self.val.dtype)
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        D[rows, self.colidx] = self.val
        return D


def init_factors(m: int, n: int, r: int, seed: int, dtype=np.float32):
    """Initial W (m x r) and H (r x n), i.i.d. U[0,1] (Sec. 4.2)."""
    g = rng(seed)
    W = g.random((m, r))
    H = g.random((r, n))
    return W.astype(dtype), H.astype(dtype)


def low_rank(m: int, n: int, r: int, seed: int = 0, noise: float = 0.0,
             dtype=np.float32, init_seed: int | None = None,
             name: str = "low_rank") -> Problem:
    """X = max(0, W0 H0 + noise * sigma * N(0,1)), W0, H0 ~ U[0,1]; sigma is the
    standard deviation of the entries of W0 H0.  noise = 0 gives the exact
    low-rank X of Sec. 4.1 (no clipping needed)."""
    g = rng(seed)
    W0 = g.random((m, r))
    H0 = g.random((r, n))
    if dtype == np.float32:
        W0 = W0.astype(np.float32)
        H0 = H0.astype(np.float32)
    X = _outer_sum(W0, H0)
    if noise > 0.0:
        sigma = float(X.std())
        X += noise * sigma * g.standard_normal((m, n))
        np.maximum(X, 0.0, out=X)
    X = X.astype(dtype)
    Wi, Hi = init_factors(m, n, r, seed + 1 if init_seed is None else init_seed, dtype)
    return Problem(name, m, n, r, Wi, Hi, X=X,
                   meta={"seed": seed, "noise": noise, "recipe": "W0,H0~U[0,1]; X=max(0,W0H0+noise*sigma*N)"})


def full_rank(m: int = 200, n: int = 200, r: int = 20, seed: int = 0, dtype=np.float32,
              init_seed: int | None = None) -> Problem:
    """The "full-rank synthetic" data of Sec. 4.1: every entry of X i.i.d.
    U[0,1] (m = n = 200, r = 20 in the paper); initial W, H ~ U[0,1]."""
    g = rng(seed)
    X = g.random((m, n)).astype(dtype)
    Wi, Hi = init_factors(m, n, r, seed + 1 if init_seed is None else init_seed, dtype)
    return Problem(f"full_rank_{m}x{n}_r{r}", m, n, r, Wi, Hi, X=X,
                   meta={"seed": seed, "recipe": "X~U[0,1]"})


def oracle_scale(seed: int = 0) -> Problem:
    """m=200, n=150, r=10, X = W0 H0 in float64; initial W,H ~ U[0,1] (seed+1)."""
    return low_rank(200, 150, 10, seed=seed, noise=0.0, dtype=np.float64, name="oracle_scale_200x150_r10")


def dense_noisy(seed: int = 0, m: int = 10000, n: int = 4000, r: int = 50) -> Problem:
    """Dense noisy low-rank: m=10000, n=4000, r=50, noise 0.01 sigma, float32."""
    return low_rank(m, n, r, seed=seed, noise=0.01, dtype=np.float32,
                    name=f"dense_noisy_{m}x{n}_r{r}")


def image_like(seed: int = 0, grid=(112, 92), n: int = 4000, r: int = 64,
               blobs: int = 64) -> Problem:
    """Each column: sum_b w_b B_b + |N(0, 0.02)|, clipped to [0, 1], where
    B_b are Gaussian blobs (centre uniform on the grid, width U[3,15] px) and
    w ~ Dirichlet(0.3).  m = grid[0] * grid[1] pixels."""
    g = rng(seed)
    gy, gx = grid
    m = gy * gx
    yy, xx = np.meshgrid(np.arange(gy, dtype=np.float64), np.arange(gx, dtype=np.float64),
                         indexing="ij")
    B = np.empty((m, blobs))
    for b in range(blobs):
        cy, cx = g.uniform(0, gy), g.uniform(0, gx)
        w = g.uniform(3.0, 15.0)
        B[:, b] = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * w * w)).ravel()
    Wt = g.dirichlet(np.full(blobs, 0.3), size=n).T       # blobs x n
    X = _outer_sum(B, Wt)
    X += np.abs(0.02 * g.standard_normal((m, n)))
    np.clip(X, 0.0, 1.0, out=X)
    X = X.astype(np.float32)
    Wi, Hi = init_factors(m, n, r, seed + 1)
    return Problem(f"image_like_{m}x{n}_r{r}", m, n, r, Wi, Hi, X=X,
                   meta={"seed": seed, "grid": list(grid), "blobs": blobs})


def document_like(seed: int = 0, m: int = 50000, n: int = 20000, r: int = 30,
                  zipf_s: float = 1.1, mu: float = 5.0, sigma: float = 0.8) -> Problem:
    """Sparse term-document matrix (terms = rows, documents = columns).
    Document lengths ~ lognormal(mu, sigma) tokens; each token's term id is
    drawn with probability proportional to 1/(rank+1)^zipf_s; the value of a
    (term, doc) pair is log(1 + count) * log(1 + n / df)."""
    g = rng(seed)
    p = 1.0 / np.arange(1, m + 1, dtype=np.float64) ** zipf_s
    p /= p.sum()
    perm = g.permutation(m)                       # term ranks -> row ids
    lengths = np.maximum(1, np.rint(g.lognormal(mu, sigma, size=n))).astype(np.int64)
    doc = np.repeat(np.arange(n, dtype=np.int64), lengths)
    term = perm[g.choice(m, size=int(lengths.sum()), p=p)]
    key = term * n + doc
    ukey, counts = np.unique(key, return_counts=True)   # sorted: by term, then doc
    rows = ukey // n
    cols = (ukey % n).astype(np.int32)
    df = np.bincount(rows, minlength=m)
    idf = np.log1p(n / np.maximum(df, 1))
    val = (np.log1p(counts.astype(np.float64)) * idf[rows]).astype(np.float32)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=rowptr[1:])
    Wi, Hi = init_factors(m, n, r, seed + 1)
    return Problem(f"document_like_{m}x{n}_r{r}", m, n, r, Wi, Hi, rowptr=rowptr,
                   colidx=cols, val=val,
                   meta={"seed": seed, "nnz": int(rowptr[-1]), "zipf_s": zipf_s,
                         "lognormal": [mu, sigma]})


def csr_from_dense(X: np.ndarray):
    """CSR arrays (rowptr int64, colidx int32, val) of the nonzeros of X."""
    rows, cols = np.nonzero(X)
    rowptr = np.zeros(X.shape[0] + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=X.shape[0]), out=rowptr[1:])
    return rowptr, cols.astype(np.int32), X[rows, cols]


def batch(count: int = 512, seed: int = 0, mn_range=(64, 2048), r_range=(4, 32),
          noise: float = 0.01) -> list[Problem]:
    """`count` independent instances; m, n ~ U{mn_range}, r ~ U{r_range};
    X = (W0 H0) * (1 + noise * U[-1, 1]) with float32 U[0,1] factors."""
    g = rng(seed)
    out = []
    for b in range(count):
        m = int(g.integers(mn_range[0], mn_range[1] + 1))
        n = int(g.integers(mn_range[0], mn_range[1] + 1))
        r = int(g.integers(r_range[0], r_range[1] + 1))
        s = int(g.integers(0, 2**31 - 1))
        gi = rng(s)
        W0 = gi.random((m, r)).astype(np.float32)
        H0 = gi.random((r, n)).astype(np.float32)
        X = _outer_sum(W0, H0) * (1.0 + noise * gi.uniform(-1.0, 1.0, size=(m, n)))
        Wi, Hi = init_factors(m, n, r, s + 1)
        out.append(Problem(f"batch{b}_{m}x{n}_r{r}", m, n, r, Wi, Hi, X=X.astype(np.float32),
                           meta={"seed": s}))
    return out
