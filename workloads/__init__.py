"""Seeded synthetic inputs shaped like the paper's workloads (§5, Table 3).

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no Gram, cross term, rescaling or NNLS step).  Both the
CPU oracle (through the tests) and the CUDA path consume what it returns, so
the two sides always see identical inputs.

The paper's datasets (CBCL Faces, MNIST, Tiny Images, NYTimes bag-of-words,
§5 Table 3) are not available; the generators below stand in for them:

* ``tiny``     - 200x150 dense, exact rank-10 product plus |N(0, 0.01)| noise.
* ``dense``    - 10000x4096 dense image-like matrix in [0, 1] built from a
                 rank-50 product (normalised, noised, clipped).
* ``sparse``   - 100000x50000 CSR bag-of-words counts: Poisson(50) distinct
                 columns per row, Zipf(1.1) column popularity, values
                 Poisson(2)+1.
* ``batched``  - 256 independent dense instances of uneven m, n, r.
* ``serving``  - a fixed column-normalised basis 50000x128 and a stream of
                 CSR request blocks of log-uniform width.

All matrices are row-major.  Factor layout: W is m x r, and H is kept as its
transpose Ht (n x r) so that every NNLS problem is one contiguous r-vector.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng", "tiny", "dense", "sparse", "batched", "serving", "random_nqp",
    "random_csr", "csr_transpose", "zipf_rows", "DenseInstance",
    "SparseInstance",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-free, platform-stable PCG64 stream for ``seed``."""
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


@dataclass
class DenseInstance:
    V: np.ndarray            # m x n
    W0: np.ndarray           # m x r   initial W
    Ht0: np.ndarray          # n x r   initial H^T
    r: int
    alpha_w: float = 0.0
    alpha_h: float = 0.0
    beta_w: float = 0.0
    beta_h: float = 0.0
    outer_iters: int = 50
    name: str = ""

    @property
    def m(self):
        return self.V.shape[0]

    @property
    def n(self):
        return self.V.shape[1]


@dataclass
class SparseInstance:
    rowptr: np.ndarray       # int64, m+1
    colidx: np.ndarray       # int32, nnz
    vals: np.ndarray         # float32 (or float64), nnz
    m: int
    n: int
    W0: np.ndarray
    Ht0: np.ndarray
    r: int
    alpha_w: float = 0.0
    alpha_h: float = 0.0
    beta_w: float = 0.0
    beta_h: float = 0.0
    outer_iters: int = 100
    name: str = ""
    # CSR of V^T (the same matrix stored by columns), filled by csr_transpose
    t_rowptr: np.ndarray | None = None
    t_colidx: np.ndarray | None = None
    t_vals: np.ndarray | None = None

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self, dtype=np.float64):
        D = np.zeros((self.m, self.n), dtype=dtype)
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        D[rows, self.colidx] = self.vals
        return D


def _abs_noise(g: np.random.Generator, shape, sigma=0.01):
    return np.abs(g.normal(0.0, sigma, size=shape))


def tiny(seed: int = 0, r: int = 10, m: int = 200, n: int = 150, r0: int = 10,
         dtype=np.float64) -> DenseInstance:
    """V = W0 H0 + |N(0, 0.01)|, W0 200x10, H0 10x150 ~ U[0,1]; init U[0,1]."""
    g = rng(seed)
    W0 = g.random((m, r0))
    H0 = g.random((r0, n))
    V = W0 @ H0 + _abs_noise(g, (m, n))
    Wi = g.random((m, r))
    Hti = g.random((n, r))
    return DenseInstance(V.astype(dtype), Wi.astype(dtype), Hti.astype(dtype),
                         r, outer_iters=50, name=f"tiny{m}x{n}r{r}")


def dense(seed: int = 0, m: int = 10000, n: int = 4096, r: int = 50, r0: int = 50,
          beta: float = 0.1, dtype=np.float32) -> DenseInstance:
    """Image-like dense matrix in [0, 1].

    The literal recipe (clip W0 H0 + noise to [0, 1]) gives V == 1 because
    every entry of a rank-50 product of U[0,1] factors exceeds 1, so the
    product is first divided by its maximum, then noised and clipped.
    """
    g = rng(seed)
    W0 = g.random((m, r0))
    H0 = g.random((r0, n))
    P = W0 @ H0
    P /= P.max()
    V = np.clip(P + _abs_noise(g, (m, n)), 0.0, 1.0)
    Wi = g.random((m, r))
    Hti = g.random((n, r))
    return DenseInstance(V.astype(dtype), Wi.astype(dtype), Hti.astype(dtype), r,
                         beta_w=beta, beta_h=beta, outer_iters=200,
                         name=f"dense{m}x{n}r{r}")


def zipf_rows(g: np.random.Generator, counts: np.ndarray, n: int, s: float = 1.1,
              chunk: int = 8192) -> list[np.ndarray]:
    """For each entry k of ``counts`` draw k distinct indices in [0, n) without
    replacement, index rank j (0-based) having weight (j+1)^-s.

    Successive weighted sampling without replacement equals keeping the first
    occurrences of i.i.d. weighted draws, which is what is done here.
    """
    w = 1.0 / np.arange(1, n + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    out: list[np.ndarray] = [None] * len(counts)  # type: ignore
    kmax = int(counts.max()) if len(counts) else 0
    for a in range(0, len(counts), chunk):
        b = min(len(counts), a + chunk)
        pending = np.arange(a, b)
        ndraw = max(64, 4 * kmax)   # doubled only for the rows still short
        while len(pending):
            d = np.searchsorted(cdf, g.random((len(pending), ndraw)), side="right")
            d = np.minimum(d, n - 1)
            order = np.argsort(d, axis=1, kind="stable")
            sd = np.take_along_axis(d, order, 1)
            first_sorted = np.ones_like(sd, dtype=bool)
            first_sorted[:, 1:] = sd[:, 1:] != sd[:, :-1]
            first = np.empty_like(first_sorted)
            np.put_along_axis(first, order, first_sorted, 1)
            cum = np.cumsum(first, axis=1)
            need = counts[pending]
            ok = cum[:, -1] >= need
            for j in np.nonzero(ok)[0]:
                keep = first[j] & (cum[j] <= need[j])
                out[pending[j]] = d[j][keep].astype(np.int64)
            pending = pending[~ok]
            ndraw *= 2
    return out


def _csr_from_rows(rows_cols: list[np.ndarray], vals: np.ndarray):
    lens = np.array([len(c) for c in rows_cols], dtype=np.int64)
    rowptr = np.zeros(len(rows_cols) + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    colidx = np.empty(int(rowptr[-1]), dtype=np.int32)
    for i, c in enumerate(rows_cols):
        colidx[rowptr[i]:rowptr[i + 1]] = np.sort(c)
    return rowptr, colidx, vals


def csr_transpose(rowptr, colidx, vals, m: int, n: int):
    """CSR of the transpose (n rows), columns sorted within each row."""
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rowptr))
    order = np.lexsort((rows, colidx.astype(np.int64)))
    t_col = rows[order].astype(np.int32)
    t_val = vals[order]
    cnt = np.bincount(colidx.astype(np.int64), minlength=n)
    t_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=t_ptr[1:])
    return t_ptr, t_col, t_val


def sparse(seed: int = 0, m: int = 100000, n: int = 50000, r: int = 100,
           mean_nnz: float = 50.0, s: float = 1.1, alpha_h: float = 0.01,
           with_transpose: bool = True, dtype=np.float32) -> SparseInstance:
    """Bag-of-words counts: row i has Poisson(mean_nnz) distinct columns,
    drawn with Zipf(s) popularity over column rank; values Poisson(2)+1."""
    g = rng(seed)
    counts = np.minimum(g.poisson(mean_nnz, size=m), n).astype(np.int64)
    cols = zipf_rows(g, counts, n, s)
    nnz = int(counts.sum())
    vals = (g.poisson(2.0, size=nnz) + 1).astype(dtype)
    rowptr, colidx, vals = _csr_from_rows(cols, vals)
    Wi = g.random((m, r)).astype(dtype)
    Hti = g.random((n, r)).astype(dtype)
    inst = SparseInstance(rowptr, colidx, vals, m, n, Wi, Hti, r, alpha_h=alpha_h,
                          outer_iters=100, name=f"sparse{m}x{n}r{r}")
    if with_transpose:
        inst.t_rowptr, inst.t_colidx, inst.t_vals = csr_transpose(rowptr, colidx, vals, m, n)
    return inst


def random_csr(seed: int, m: int, n: int, density: float, empty_rows: int = 0,
               long_rows: int = 0, dtype=np.float32):
    """Small uniform CSR with optional forced empty rows and dense 'head' rows
    (to exercise ragged and long-row paths)."""
    g = rng(seed)
    counts = g.binomial(n, density, size=m).astype(np.int64)
    if empty_rows:
        counts[g.choice(m, size=min(empty_rows, m), replace=False)] = 0
    if long_rows:
        counts[g.choice(m, size=min(long_rows, m), replace=False)] = n
    cols = [np.sort(g.choice(n, size=int(k), replace=False)) for k in counts]
    vals = (g.poisson(2.0, size=int(counts.sum())) + 1).astype(dtype)
    return _csr_from_rows(cols, vals)


def batched(seed: int = 0, count: int = 256, m_range=(100, 4000), n_range=(100, 2000),
            ranks=(8, 16, 32, 64), outer_iters: int = 100,
            workers: int = 1) -> list[DenseInstance]:
    """Independent dense instances of uneven shape, V = W0 H0 + |N(0,0.01)|
    with W0, H0 and the initial factors U[0,1] (all FP32; the noise drawn as
    single-precision normals).  Shapes come from one stream of ``seed``;
    instance i's values from its own child stream, so ``workers`` threads
    give the same instances as one."""
    g = rng(seed)
    shapes = []
    for _ in range(count):
        m = int(g.integers(m_range[0], m_range[1] + 1))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        r = int(ranks[int(g.integers(0, len(ranks)))])
        shapes.append((m, n, r))
    children = np.random.SeedSequence(int(seed)).spawn(count)

    def make(i):
        m, n, r = shapes[i]
        gi = np.random.default_rng(children[i])
        W0 = gi.random((m, r), dtype=np.float32)
        H0 = gi.random((r, n), dtype=np.float32)
        noise = np.abs(gi.standard_normal((m, n), dtype=np.float32)) * np.float32(0.01)
        V = W0 @ H0 + noise
        Wi = gi.random((m, r), dtype=np.float32)
        Hti = gi.random((n, r), dtype=np.float32)
        return DenseInstance(V, Wi, Hti, r, outer_iters=outer_iters, name=f"b{i}_{m}x{n}r{r}")

    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            return list(ex.map(make, range(count)))
    return [make(i) for i in range(count)]


@dataclass
class ServingWorkload:
    W: np.ndarray                          # basis rows x r (float32)
    arrivals: np.ndarray                   # seconds, sorted
    requests: list = field(default_factory=list)   # (rowptr, colidx, vals) per request


def serving(seed: int = 0, rows: int = 50000, r: int = 128, rate: float = 2000.0,
            duration: float = 1.0, max_width: int = 4096, nnz_per_col: int = 100,
            s: float = 1.1, max_requests: int | None = None) -> ServingWorkload:
    """Fixed basis W (U[0,1], columns scaled to unit l2 norm) and Poisson
    arrivals of CSR request blocks; request j has w_j new columns (width
    log-uniform on [1, max_width]); each new column is one CSR row over the
    basis rows with ``nnz_per_col`` distinct entries of Zipf(s) popularity and
    values Poisson(2)+1."""
    g = rng(seed)
    W = g.random((rows, r))
    W /= np.sqrt((W * W).sum(axis=0, keepdims=True))
    W = W.astype(np.float32)
    nreq = int(g.poisson(rate * duration))
    if max_requests is not None:
        nreq = min(nreq, max_requests)
    gaps = g.exponential(1.0 / rate, size=nreq)
    arrivals = np.cumsum(gaps)
    perm = g.permutation(rows)          # popularity rank -> basis row
    reqs = []
    for _ in range(nreq):
        w = int(min(max_width, math.floor(math.exp(g.uniform(0.0, math.log(max_width + 1))))))
        w = max(1, w)
        counts = np.full(w, nnz_per_col, dtype=np.int64)
        cols = zipf_rows(g, counts, rows, s)
        cols = [perm[c] for c in cols]
        vals = (g.poisson(2.0, size=w * nnz_per_col) + 1).astype(np.float32)
        reqs.append(_csr_from_rows(cols, vals))
    return ServingWorkload(W, arrivals, reqs)


def random_nqp(seed: int, r: int, k: int | None = None, beta: float = 0.0,
               rows: int = 1, scale: float = 1.0):
    """Random NNLS data: A (k x r) ~ U[0,1], b_i ~ U[0,1]*scale for ``rows``
    right-hand sides.  Returns (A, B) with B rows x k, so that each problem is
    min 1/2||A x - b_i||^2 (+ beta/2 ||x||^2), x >= 0."""
    g = rng(seed)
    k = k if k is not None else 3 * r + 2
    A = g.random((k, r))
    B = g.random((rows, k)) * scale
    return A, B
