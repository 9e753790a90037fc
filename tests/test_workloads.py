"""The seeded synthetic inputs follow their stated recipes (the stand-ins for
the paper's datasets, §5 Table 3): shapes, value ranges, distributions and
sparsity structure, and reproducibility from the seed.  CPU only."""
import math

import numpy as np
import pytest

import workloads as WL


def test_tiny_recipe_and_seed():
    a = WL.tiny(seed=1)
    b = WL.tiny(seed=1)
    c = WL.tiny(seed=2)
    assert a.V.shape == (200, 150) and a.W0.shape == (200, 10) and a.Ht0.shape == (150, 10)
    assert np.array_equal(a.V, b.V) and np.array_equal(a.W0, b.W0)
    assert not np.array_equal(a.V, c.V)
    # initial factors U[0, 1]; V = W0 H0 + |noise| >= 0
    for x in (a.W0, a.Ht0):
        assert x.min() >= 0.0 and x.max() < 1.0
    assert a.V.min() > 0.0


def test_dense_recipe_not_degenerate():
    # the literal recipe would clip every entry to 1 (rank-50 products of U[0,1]
    # factors exceed 1); the normalised product stays inside [0, 1] with spread
    d = WL.dense(seed=0, m=2000, n=1000)
    V = d.V.astype(np.float64)
    assert d.V.dtype == np.float32 and V.shape == (2000, 1000)
    assert V.min() >= 0.0 and V.max() <= 1.0
    assert V.max() == 1.0                       # the largest entries saturate
    assert np.mean(V >= 1.0) < 1e-3             # ... but only a few of them
    assert V.std() > 0.05 and V.min() < 0.5 < V.mean()   # not constant
    assert d.beta_w == d.beta_h == 0.1 and d.r == 50


def test_dense_noise_is_half_normal_sigma_001():
    # with the product removed the residual is |N(0, 0.01)| (before clipping):
    # mean sigma sqrt(2/pi)
    g = WL.rng(0)
    W0 = g.random((300, 50))
    H0 = g.random((50, 200))
    P = W0 @ H0
    P /= P.max()
    d = WL.dense(seed=0, m=300, n=200)
    resid = d.V.astype(np.float64) - P
    inside = d.V < 1.0
    assert resid[inside].min() >= -1e-6
    assert abs(resid[inside].mean() - 0.01 * math.sqrt(2 / math.pi)) < 5e-4


def test_sparse_recipe():
    m, n = 20000, 10000
    s = WL.sparse(seed=3, m=m, n=n)
    lens = np.diff(s.rowptr)
    # Poisson(50) distinct columns per row
    assert abs(lens.mean() - 50.0) < 0.5 and abs(lens.var() - 50.0) < 5.0
    for i in range(0, m, 997):
        c = s.colidx[s.rowptr[i]:s.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)           # sorted, distinct
        assert c.min() >= 0 and c.max() < n
    # values Poisson(2) + 1: integers >= 1 with mean 3, exact in BF16
    v = s.vals.astype(np.float64)
    assert v.min() >= 1.0 and np.all(v == np.round(v)) and abs(v.mean() - 3.0) < 0.02
    assert v.max() <= 256.0
    # Zipf(1.1) column popularity: the head column sits in nearly every row,
    # and popularity falls with rank
    freq = np.bincount(s.colidx, minlength=n) / m
    assert freq[0] > 0.9
    assert freq[0] > freq[9] > freq[99] > freq[999] > freq[9999]


def test_sparse_transpose_round_trip():
    s = WL.sparse(seed=4, m=3000, n=1500)
    tp, tc, tv = s.t_rowptr, s.t_colidx, s.t_vals
    assert tp[-1] == s.rowptr[-1]
    rp, ci, va = WL.csr_transpose(tp, tc, tv, 1500, 3000)
    assert np.array_equal(rp, s.rowptr) and np.array_equal(ci, s.colidx)
    assert np.array_equal(va, s.vals)


def test_zipf_rows_draws_distinct_columns():
    g = WL.rng(5)
    counts = np.array([0, 1, 5, 64, 200])
    rows = WL.zipf_rows(g, counts, 300)
    for k, r in zip(counts, rows):
        assert len(r) == k and len(np.unique(r)) == k
        assert (r >= 0).all() and (r < 300).all()


def test_batched_shapes_and_thread_independence():
    insts = WL.batched(seed=0, count=64)
    ms = np.array([x.V.shape[0] for x in insts])
    ns = np.array([x.V.shape[1] for x in insts])
    rs = np.array([x.r for x in insts])
    assert ms.min() >= 100 and ms.max() <= 4000 and ns.min() >= 100 and ns.max() <= 2000
    assert set(rs) <= {8, 16, 32, 64} and len(set(rs)) == 4
    for x in insts[:4]:
        assert x.V.dtype == np.float32 and x.W0.shape == (x.V.shape[0], x.r)
        assert x.Ht0.shape == (x.V.shape[1], x.r) and x.V.min() > 0.0
    small = dict(count=12, m_range=(100, 300), n_range=(100, 200))
    one = WL.batched(seed=7, workers=1, **small)
    four = WL.batched(seed=7, workers=4, **small)
    for a, b in zip(one, four):
        assert np.array_equal(a.V, b.V) and np.array_equal(a.W0, b.W0)


def test_serving_recipe():
    w = WL.serving(seed=1, rows=5000, r=32, duration=0.1, max_width=4096)
    assert np.allclose(np.linalg.norm(w.W.astype(np.float64), axis=0), 1.0, atol=1e-5)
    assert np.all(np.diff(w.arrivals) > 0)
    assert abs(len(w.arrivals) - 200) < 50            # Poisson(rate * duration)
    widths = np.array([len(rp) - 1 for rp, _, _ in w.requests])
    assert widths.min() >= 1 and widths.max() <= 4096
    # log-uniform widths: median near sqrt(4097) ~ 64
    assert 25 < np.median(widths) < 160
    rp, ci, va = w.requests[0]
    assert np.all(np.diff(rp) == 100)                 # 100 distinct rows per column
    for i in range(len(rp) - 1):
        assert len(np.unique(ci[rp[i]:rp[i + 1]])) == 100


@pytest.mark.parametrize("seed", [0, 1])
def test_random_nqp_is_reproducible(seed):
    a = WL.random_nqp(seed, 6)
    b = WL.random_nqp(seed, 6)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))
