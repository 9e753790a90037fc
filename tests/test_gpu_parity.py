"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Protocol: both sides get the same seeded inputs (the oracle sees the FP32
values the GPU sees, widened to FP64).  Sizes span several CTAs and end in a
ragged tail.  Every tolerance is a bound computed from the arithmetic:

* each row of an NNLS half-step, in the solver's rescaled variables:
  ||(x_i - x_i*) d|| <= C u (||qt_i|| + ||Qt|| (||y_i*|| + ||y0_i||)) /
  lambda_min(Qt) (tests/gpu_common.py: the solution map is
  1/lambda_min-Lipschitz in the linear term; C = 20, twice the largest
  measured ratio); a fixed-K row may leave it only through a named greedy
  near-tie: the oracle's best and second gains at some step differ by less
  than 16 FP32 resolution units of the gain, and the row's error is at most
  2.5 times the move the swap would make;
* a default set of well-conditioned problems (kappa(Qt) <= 5) where every
  row's relative error is at most 1e-4, the factor tolerance of the target;
* norm-wise over a factor, one NNLS solve: <= 16 sqrt(r) kappa u, u = 2^-24;
* a half-step fed by a factor that carries relative error e inherits
  kappa e on top of its own bound;
* over T outer iterations of a contracting trajectory (successive-difference
  ratio rho measured on the oracle's own run) the per-step bound is summed
  over the horizon 1/(1 - rho);
* the FP64 trace-identity objective evaluated from FP32 Grams and cross
  terms carries an error of order u ||V||^2 / J.
Objectives are compared at 1e-5 wherever the trajectory is not chaotic.
"""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from tests.gpu_common import (assert_nqp_rows, csr_t, dev, elementwise_ok, rel_err,
                               row_rel_err, t32, to_np, torch)

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")


@pytest.fixture(scope="module")
def h():
    import __graft_entry__ as g
    g.build()
    hh = P.Handle(0)
    yield hh
    hh.close()


def nqp_batch(seed, r, rows, beta=0.0, shift=0.45):
    """Rows of NNLS problems sharing Q = A'A + beta I; C rows = A' b_i.
    b_i shifted so that the solutions have mixed active sets."""
    g = WL.rng(seed)
    k = 3 * r + 4
    A = g.random((k, r))
    Bm = g.random((rows, k)) - shift
    Q = O.gram(A, beta)
    Cm = O.cross_dense(Bm, A)
    X0 = g.random((rows, r))
    # round to what the GPU sees
    Q32 = Q.astype(np.float32).astype(np.float64)
    C32 = Cm.astype(np.float32).astype(np.float64)
    X32 = X0.astype(np.float32).astype(np.float64)
    return Q32, C32, X32


RANKS = [1, 4, 7, 8, 10, 31, 32, 33, 50, 64, 65, 96, 100, 128]
U32 = 2.0 ** -24


def nnls_tol(Q, r):
    """Forward-error bound of an FP32 NNLS solve: the error of the passive-set
    solution is (condition number of the rescaled Q) x (backward error); the
    backward error of r-term FP32 dot products grows like sqrt(r) u.  The
    factor 16 covers the constant (measured ratios on these problems: 20-40
    kappa u at sqrt(r) = 3..11)."""
    Qt, _, dead = O.rescale(Q)
    live = ~dead
    ev = np.linalg.eigvalsh(Qt[np.ix_(live, live)])
    kappa = ev[-1] / max(ev[0], 1e-300)
    return max(2e-6, 16.0 * np.sqrt(r) * kappa * U32)


def sparse_nqp_batch(seed, r, rows):
    """Well-conditioned NNLS data: A sparse (10% nonzeros) so columns are
    nearly orthogonal."""
    g = WL.rng(seed)
    k = 20 * r + 4
    A = g.random((k, r)) * (g.random((k, r)) < 0.1)
    Bm = g.random((rows, k)) - 0.3
    Q = O.gram(A, 0.01)
    Cm = O.cross_dense(Bm, A)
    X0 = g.random((rows, r))
    return (Q.astype(np.float32).astype(np.float64), Cm.astype(np.float32).astype(np.float64),
            X0.astype(np.float32).astype(np.float64))


def gpu_nnls(h, Q, Cm, X0, alpha, opts):
    Qt, d, _ = O.rescale(Q)
    X = t32(X0)
    it = torch.empty(X0.shape[0], dtype=torch.int32, device=dev())
    P.nmf_nnls_update(h, t32(Qt), t32(d), t32(Cm), X, alpha=alpha, opts=opts, inner_iters=it)
    h.sync()
    return to_np(X), it.cpu().numpy()


@pytest.mark.parametrize("r", RANKS)
def test_nnls_fixed_iterations(h, r):
    rows = 8 * 37 + 5
    Q, Cm, X0 = nqp_batch(10 + r, r, rows, beta=0.05)
    K = 3
    oo = O.nqp_opts(max_inner=K, eps=0.0)
    Xo, ito, tot, _ = O.nnls_update(Q, Cm, 0.01, X0, oo)
    X, it = gpu_nnls(h, Q, Cm, X0, 0.01, P.nnls_opts(max_inner=K, eps=0.0))
    assert_nqp_rows(X, Xo, Q, Cm, 0.01, X0, fixed_k_opts=oo)
    # with eps = 0 a row stops before K only on an exactly zero projected
    # gradient.  FP32 reaches it more often than FP64: with the unit diagonal
    # of the rescaled Q a coordinate step sets g_p = g_p - g_p = 0 exactly,
    # where FP64 leaves a residue of ~1e-17.  So a count may differ only by an
    # early stop, and a row that stopped early is at the oracle's iterate.
    diff = it != ito
    assert np.all(np.minimum(it, ito)[diff] < K)
    early = it < K
    if early.any():
        assert_nqp_rows(X[early], Xo[early], Q, Cm[early], 0.01, X0[early])


@pytest.mark.parametrize("r", RANKS)
def test_nnls_converges_to_unique_minimiser(h, r):
    rows = 8 * 11 + 3
    Q, Cm, X0 = nqp_batch(200 + r, r, rows, beta=0.1)
    Xo, *_ = O.nnls_update(Q, Cm, 0.0, X0, O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
    X, it = gpu_nnls(h, Q, Cm, X0, 0.0, P.nnls_opts(max_inner=400, eps=1e-12))
    worst = assert_nqp_rows(X, Xo, Q, Cm, 0.0, X0)
    print(f"r={r}: worst row {worst:.3f} of its bound; norm-wise {rel_err(X, Xo):.2e}")
    assert rel_err(X, Xo) < nnls_tol(Q, r)


def layouts(r):
    """Every lanes-per-row setting the solver accepts for rank r."""
    return [g for g in (1, 2, 4, 8, 16, 32) if g * 16 >= r]


@pytest.mark.parametrize("r", [2, 3, 9, 17, 33, 50, 64, 100, 128])
def test_nnls_every_layout(h, r):
    """Each group width (lanes per row) and coordinates-per-lane split: the
    unique minimiser within the FP32 bound, fixed-K iterates row by row."""
    rows = 3 * 8 * 32 + 11
    Q, Cm, X0 = nqp_batch(700 + r, r, rows, beta=0.1)
    Xc, *_ = O.nnls_update(Q, Cm, 0.01, X0, O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
    ok = O.nqp_opts(max_inner=3, eps=0.0)
    Xk, itk, *_ = O.nnls_update(Q, Cm, 0.01, X0, ok)
    for lanes in layouts(r):
        X, it = gpu_nnls(h, Q, Cm, X0, 0.01, P.nnls_opts(max_inner=400, eps=1e-12, lanes=lanes))
        assert_nqp_rows(X, Xc, Q, Cm, 0.01, X0)
        X, it = gpu_nnls(h, Q, Cm, X0, 0.01, P.nnls_opts(max_inner=3, eps=0.0, lanes=lanes))
        assert_nqp_rows(X, Xk, Q, Cm, 0.01, X0, fixed_k_opts=ok)
        assert np.all(it <= 3)


@pytest.mark.parametrize("lanes", [0, 4])
def test_nnls_rows_independent_of_launch(h, lanes):
    """A row's result depends on r and the layout only, not on the rows that
    share its launch: one launch over 20000 rows (balanced CTA ranges, two
    rounds for some warps) equals, bit for bit, launches over uneven
    sub-ranges; the one-launch result is checked against the oracle's fixed-K
    iterates on a sample of rows."""
    r, rows, K = 50, 20000, 3
    Q, Cm, X0 = nqp_batch(808, r, rows, beta=0.1)
    opts = P.nnls_opts(max_inner=K, eps=0.0, lanes=lanes)
    X, it = gpu_nnls(h, Q, Cm, X0, 0.01, opts)
    cuts = [0, 1, 37, 4133, 9000, 19999, 20000]
    parts = [gpu_nnls(h, Q, Cm[lo:hi], X0[lo:hi], 0.01, opts) for lo, hi in zip(cuts, cuts[1:])]
    assert np.array_equal(X, np.concatenate([p[0] for p in parts]))
    assert np.array_equal(it, np.concatenate([p[1] for p in parts]))
    sample = np.r_[0:40, 9990:10010, 19960:20000]
    ok = O.nqp_opts(max_inner=K, eps=0.0)
    Xk, *_ = O.nnls_update(Q, Cm[sample], 0.01, X0[sample], ok)
    assert_nqp_rows(X[sample], Xk, Q, Cm[sample], 0.01, X0[sample], fixed_k_opts=ok)


def test_nnls_layout_rejects_too_few_lanes(h):
    Q, Cm, X0 = nqp_batch(5, 50, 10)
    with pytest.raises(P.NmfError):
        gpu_nnls(h, Q, Cm, X0, 0.0, P.nnls_opts(lanes=2))    # 2 lanes x 16 < 50
    with pytest.raises(P.NmfError):
        gpu_nnls(h, Q, Cm, X0, 0.0, P.nnls_opts(lanes=3))    # not a power of two


def nqp_1e4_batch(seed, r, rows):
    """The default parity set: well-conditioned NNLS data (kappa(Qt) <= 5 at
    every r <= 128) whose FP32 per-row bound stays below the target's 1e-4
    relative factor error.  A is sparse (5% nonzeros up to r = 16, 2% above),
    so its columns overlap little and the rescaled Gram is close to I; the
    targets B are sparse with a negative shift, so solutions have mixed active
    sets and some rows are entirely zero."""
    g = WL.rng(seed)
    p = 0.05 if r <= 16 else 0.02
    k = 40 * r + 4
    A = g.random((k, r)) * (g.random((k, r)) < p)
    A[g.integers(0, k, size=r), np.arange(r)] += 1.0      # no empty column
    Bm = g.random((rows, k)) * (g.random((rows, k)) < 4 * p) - 0.02
    Q = O.gram(A, 0.0)
    Cm = O.cross_dense(Bm, A)
    X0 = g.random((rows, r))
    return (Q.astype(np.float32).astype(np.float64), Cm.astype(np.float32).astype(np.float64),
            X0.astype(np.float32).astype(np.float64))


def assert_rows_1e4(X, Xo, Q, Cm, alpha, X0, fixed_k_opts=None):
    """Every row within 1e-4 relative (row_rel_err), except - for fixed-K
    iterates - rows that are named greedy near-ties."""
    from tests.gpu_common import TIE_SWAP, TIE_UNITS
    n = np.linalg.norm(Xo, axis=1)
    den = np.maximum(n, 0.1 * np.median(n))
    rel = np.linalg.norm(X - Xo, axis=1) / np.maximum(den, 1e-300)
    bad = np.nonzero(rel > 1e-4)[0]
    if len(bad):
        assert fixed_k_opts is not None, f"rows {bad[:8].tolist()} above 1e-4 ({rel.max():.2e})"
        margin, _, swap = O.nqp_min_gaps(Q, Cm[bad], alpha, X0[bad], fixed_k_opts,
                                         tie_units=TIE_UNITS)
        _, d, _ = O.rescale(Q)
        err = np.linalg.norm((X[bad] - Xo[bad]) * d, axis=1)
        tie = (margin < TIE_UNITS) & (err <= TIE_SWAP * swap)
        assert np.all(tie), f"rows {bad[~tie][:8].tolist()} above 1e-4 without a near-tie"
    return float(np.delete(rel, bad).max()) if len(bad) < len(rel) else 0.0


@pytest.mark.parametrize("r", [1, 4, 10, 33, 50, 64, 100, 128])
def test_nnls_default_set_every_row_1e4(h, r):
    """The default parity set at the target's factor tolerance: every row of
    every lane layout, solved to the unique minimiser and after K = 2 fixed
    iterations, within its FP32 bound and within 1e-4 relative of the
    oracle's row."""
    rows = 3 * 8 * 32 + 11
    Q, Cm, X0 = nqp_1e4_batch(900 + r, r, rows)
    assert kappa(Q) <= 5.0
    Xc, *_ = O.nnls_update(Q, Cm, 0.0, X0, O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
    ok = O.nqp_opts(max_inner=2, eps=0.0)
    Xk, *_ = O.nnls_update(Q, Cm, 0.0, X0, ok)
    for lanes in layouts(r):
        X, it = gpu_nnls(h, Q, Cm, X0, 0.0, P.nnls_opts(max_inner=300, eps=1e-12, lanes=lanes))
        assert_nqp_rows(X, Xc, Q, Cm, 0.0, X0)
        wc = assert_rows_1e4(X, Xc, Q, Cm, 0.0, X0)
        X, it = gpu_nnls(h, Q, Cm, X0, 0.0, P.nnls_opts(max_inner=2, eps=0.0, lanes=lanes))
        assert_nqp_rows(X, Xk, Q, Cm, 0.0, X0, fixed_k_opts=ok)
        wk = assert_rows_1e4(X, Xk, Q, Cm, 0.0, X0, fixed_k_opts=ok)
        print(f"r={r} lanes={lanes}: worst row rel err converged {wc:.2e}, fixed K {wk:.2e}")


@pytest.mark.parametrize("r", [4, 10, 50, 100, 128])
def test_nnls_sparse_gram_rows(h, r):
    """Sparse factor columns (10% nonzeros, kappa 1.6 - 18): every row within
    its FP32 bound, to the minimiser and after K = 2 (near-ties named)."""
    rows = 8 * 20 + 7
    Q, Cm, X0 = sparse_nqp_batch(300 + r, r, rows)
    Xo, *_ = O.nnls_update(Q, Cm, 0.02, X0, O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
    X, it = gpu_nnls(h, Q, Cm, X0, 0.02, P.nnls_opts(max_inner=300, eps=1e-12))
    assert_nqp_rows(X, Xo, Q, Cm, 0.02, X0)
    ok = O.nqp_opts(max_inner=2, eps=0.0)
    Xo, ito, *_ = O.nnls_update(Q, Cm, 0.02, X0, ok)
    X, it = gpu_nnls(h, Q, Cm, X0, 0.02, P.nnls_opts(max_inner=2, eps=0.0))
    assert_nqp_rows(X, Xo, Q, Cm, 0.02, X0, fixed_k_opts=ok)


def test_nnls_accelerated_condition_counts(h):
    r, rows = 20, 2000
    Q, Cm, X0 = nqp_batch(5, r, rows)
    Xo, ito, tot, _ = O.nnls_update(Q, Cm, 0.0, X0, O.nqp_opts(max_inner=50, eps=1e-3))
    Qt, d, _ = O.rescale(Q)
    X = t32(X0)
    it = torch.empty(rows, dtype=torch.int32, device=dev())
    P.nmf_nnls_update(h, t32(Qt), t32(d), t32(Cm), X, opts=P.nnls_opts(max_inner=50, eps=1e-3),
                      inner_iters=it)
    h.sync()
    itg = it.cpu().numpy()
    # the stop decision is an FP comparison: all but a few rows agree exactly
    assert np.mean(itg == ito) > 0.98
    assert abs(itg.mean() - ito.mean()) < 0.05 * ito.mean()


@pytest.mark.parametrize("rows", [1, 100, 1023, 20001])
@pytest.mark.parametrize("r", [1, 10, 50, 100, 128])
def test_gram(h, rows, r):
    X = WL.rng(rows + r).random((rows, r)).astype(np.float32)
    Qo = O.gram(X.astype(np.float64), 0.25)
    Q = P.nmf_gram(h, t32(X), beta=0.25)
    h.sync()
    # element by element against the sum of the (nonnegative) products
    elementwise_ok(to_np(Q), Qo, Qo, 2e-6)


# element-wise bounds of one product term, relative to |x_a x_b|: round to
# nearest TF32 (11 significant bits) / BF16 (8) moves each operand by at most
# 2^-11 / 2^-8 of itself, so a product by 2^-10 / 2^-7; the hi + lo BF16
# split represents x to within 2^-8 |x - hi| <= 2^-16 |x| and drops lo lo
# (|lo| <= 2^-8 |x|), so a product moves by at most 3 * 2^-16
GRAM_TOL = {"fp32": 2e-6, "tf32": 2.0 ** -10 + 2e-6, "bf16": 2.0 ** -7 + 2e-6,
            "bf16x2": 3 * 2.0 ** -16 + 2e-6}


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x2"])
@pytest.mark.parametrize("rows,r", [(100, 10), (20001, 50), (3000, 128)])
def test_gram_operand_precisions(h, prec, rows, r):
    """nmf_gram's reduced-precision operand modes against the FP64 Gram of
    the FP32 factor, element by element within the stated worst-case bound
    (each is also well below it on average, and BF16X2 is FP32-grade)."""
    X = WL.rng(rows * 3 + r).random((rows, r)).astype(np.float32)
    Qo = O.gram(X.astype(np.float64), 0.1)
    Q = P.nmf_gram(h, t32(X), beta=0.1, prec=prec)
    h.sync()
    worst = elementwise_ok(to_np(Q), Qo, Qo, GRAM_TOL[prec])
    print(f"gram {prec} rows={rows} r={r}: worst {worst:.3f} x bound, norm-wise "
          f"{rel_err(to_np(Q), Qo):.2e}")


@pytest.mark.parametrize("M,K", [(1, 7), (1007, 3005), (300, 20000)])
@pytest.mark.parametrize("r", [4, 50, 100, 128])
def test_cross_dense(h, M, K, r):
    g = WL.rng(M + K + r)
    A = g.random((M, K)).astype(np.float32)
    B = g.random((K, r)).astype(np.float32)
    Co = O.cross_dense(A.astype(np.float64), B.astype(np.float64))
    Cg = P.nmf_cross(h, t32(A), t32(B))
    h.sync()
    elementwise_ok(to_np(Cg), Co, Co, 2e-6)     # |A||B| = A B: nonnegative inputs


@pytest.mark.parametrize("r", [3, 32, 100, 128])
def test_cross_csr(h, r):
    rp, ci, va = WL.random_csr(7, 3000, 1500, 0.01, empty_rows=40, long_rows=3)
    B = WL.rng(3).random((1500, r)).astype(np.float32)
    Co = O.cross_csr(rp, ci, va.astype(np.float64), B.astype(np.float64))
    rpt, cit, vat = csr_t(rp, ci, va)
    Cg = P.nmf_cross(h, None, t32(B), csr_parts=(rpt, cit, vat, 1500))
    h.sync()
    scale = O.cross_csr(rp, ci, np.abs(va).astype(np.float64), np.abs(B).astype(np.float64))
    elementwise_ok(to_np(Cg), Co, scale, 2e-6)
    empty = np.diff(rp) == 0
    assert np.all(to_np(Cg)[empty] == 0)


def test_cross_csr_bf16_values(h):
    rp, ci, va = WL.random_csr(8, 2000, 900, 0.02)
    B = WL.rng(4).random((900, 64)).astype(np.float32)
    Co = O.cross_csr(rp, ci, va.astype(np.float64), B.astype(np.float64))
    rpt, cit, vat = csr_t(rp, ci, va, dtype=torch.bfloat16)   # counts are exact in BF16
    Cg = P.nmf_cross(h, None, t32(B), csr_parts=(rpt, cit, vat, 900))
    h.sync()
    scale = O.cross_csr(rp, ci, np.abs(va).astype(np.float64), np.abs(B).astype(np.float64))
    elementwise_ok(to_np(Cg), Co, scale, 2e-6)


def test_rescale_with_dead_coordinate(h):
    X = WL.rng(1).random((40, 6))
    X[:, 3] = 0.0
    Q = O.gram(X, 0.0)
    Qt_o, d_o, dead = O.rescale(Q)
    Qt, d = P.nmf_rescale(h, t32(Q))
    h.sync()
    assert dead[3]
    assert np.abs(to_np(Qt) - Qt_o).max() < 1e-6
    assert np.abs(to_np(d) - d_o).max() < 1e-6 * d_o.max()
    assert to_np(d)[3] == 1.0 and np.all(to_np(Qt)[3] == 0)


def test_objective_trace_identity(h):
    inst = WL.tiny(seed=3, r=8, m=300, n=200)
    W = inst.W0.astype(np.float32)
    Ht = inst.Ht0.astype(np.float32)
    V = inst.V.astype(np.float32)
    Wd, Hd, Vd = (a.astype(np.float64) for a in (W, Ht, V))
    Jo = O.objective_dense(Vd, Wd, Hd, 0.1, 0.2, 0.3, 0.4)
    Ch = t32(O.cross_dense(Vd.T, Wd))
    Gw = t32(O.gram(Wd))
    Gh = t32(O.gram(Hd))
    J = P.nmf_objective(h, float(np.sum(Vd * Vd)), t32(W), t32(Ht), Ch, Gw, Gh, 0.1, 0.2, 0.3, 0.4)
    h.sync()
    assert abs(J.item() - Jo) / Jo < 1e-6


@pytest.mark.parametrize("r,rows", [(12, 333), (1, 40), (64, 31), (100, 2049), (128, 777)])
def test_kkt(h, r, rows):
    # tiles of 32 rows (a ragged last tile), one or two columns per thread
    Q, Cm, X0 = nqp_batch(9 + r, r, rows)
    out = P.nmf_kkt(h, t32(Q), t32(Cm), t32(X0), alpha=0.02)
    h.sync()
    ko = O.kkt(Q, Cm, 0.02, X0)
    np.testing.assert_allclose(out.cpu().numpy(), ko, rtol=1e-9)


def run_solve(h, inst, T, K, eps=0.0, use_graph=False, sparse=None, objective="trace"):
    W = t32(inst.W0)
    Ht = t32(inst.Ht0)
    hist = (np.zeros(T)).astype(np.float64)
    import ctypes as C
    hp = hist.ctypes.data_as(C.POINTER(C.c_double))
    o = P.solve_opts(T, alpha_w=inst.alpha_w, alpha_h=inst.alpha_h, beta_w=inst.beta_w,
                     beta_h=inst.beta_h, nnls=P.nnls_opts(max_inner=K, eps=eps),
                     use_graph=use_graph, obj_hist=hp, objective=objective)
    if sparse is None:
        rep = P.nmf_solve(h, t32(inst.V), W, Ht, o)
    else:
        rep = P.nmf_solve(h, None, W, Ht, o, csr_parts=sparse[0], csr_t_parts=sparse[1])
    return W, Ht, hist, rep


def f32_inst(inst):
    for k in ("V", "W0", "Ht0"):
        a = getattr(inst, k)
        if a is not None:
            setattr(inst, k, a.astype(np.float32).astype(np.float64))
    return inst


@pytest.mark.parametrize("r,m,n", [(8, 300, 200), (37, 257, 203), (64, 129, 130)])
def test_objective_direct_matches_oracle(h, r, m, n):
    # 128 x 128 tiles with ragged edges; n % 4 != 0 takes the scalar loads of V;
    # r > 16 spans several staged chunks of the factors
    inst = f32_inst(WL.tiny(seed=3 + r, r=r, m=m, n=n))
    Jo = O.objective_dense(inst.V, inst.W0, inst.Ht0, 0.1, 0.2, 0.3, 0.4)
    J = P.nmf_objective_direct(h, t32(inst.V), t32(inst.W0), t32(inst.Ht0), 0.1, 0.2, 0.3, 0.4)
    h.sync()
    assert abs(J.item() - Jo) / Jo < 1e-7


def kappa(Q):
    Qt, _, dead = O.rescale(Q)
    ev = np.linalg.eigvalsh(Qt[np.ix_(~dead, ~dead)])
    return ev[-1] / max(ev[0], 1e-300)


def step_bounds(Wo, Ho, r, beta_w=0.0, beta_h=0.0):
    """Bounds for one outer iteration: the W-update's own FP32 bound, and the
    H-update's bound plus the W error carried through kappa(Q_H)."""
    tw = nnls_tol(O.gram(Ho, beta_w), r)
    qh = O.gram(Wo, beta_h)
    th = nnls_tol(qh, r) + kappa(qh) * tw
    return tw, th


def assert_iteration_rows(V, W0, Ht0, Wg, Hg, K, aw=0.0, ah=0.0, bw=0.0, bh=0.0):
    """One GPU outer iteration row by row: each W row against the oracle's
    W-update from the same (exact FP32) start, and each Ht row against the
    oracle's H-update computed from the GPU's own W (so every row's check sees
    only its own half-step's arithmetic).  K = None: solved to the
    minimiser; else K fixed iterations (near-ties named).  Returns the
    oracle's W-update rows."""
    o = (O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24) if K is None
         else O.nqp_opts(max_inner=K, eps=0.0))
    fk = None if K is None else o
    Qw = O.gram(Ht0, bw)
    Cw = O.cross_dense(V, Ht0)
    Wo, *_ = O.nnls_update(Qw, Cw, aw, W0, o)
    assert_nqp_rows(Wg, Wo, Qw, Cw, aw, W0, fixed_k_opts=fk)
    ties = assert_nqp_rows.ties
    Wg64 = np.asarray(Wg, dtype=np.float64)
    Qh = O.gram(Wg64, bh)
    Ch = O.cross_dense(np.ascontiguousarray(V.T), Wg64)
    Hs, *_ = O.nnls_update(Qh, Ch, ah, Ht0, o)
    assert_nqp_rows(Hg, Hs, Qh, Ch, ah, Ht0, fixed_k_opts=fk)
    assert_iteration_rows.ties = ties + assert_nqp_rows.ties
    return Wo


def j_bound(inst, Wo, Ho, tw, th):
    """First-order objective bound |dJ| <= ||R|| (||dW|| ||H|| + ||W|| ||dH||)."""
    R = np.sqrt(2 * O.objective_dense(inst.V, Wo, Ho))
    dJ = R * (tw * np.linalg.norm(Wo) * np.linalg.norm(Ho) + th * np.linalg.norm(Wo) *
              np.linalg.norm(Ho))
    return max(1e-5, dJ / O.objective_dense(inst.V, Wo, Ho))


@pytest.mark.parametrize("r,t0", [(10, 0), (10, 5), (10, 20), (4, 0), (4, 10)])
def test_one_iteration_from_oracle_state(h, r, t0):
    """P-step: the oracle runs t0 iterations; from that (FP32-rounded) state
    the oracle and the GPU each run one more iteration with K = 3 fixed."""
    inst = f32_inst(WL.tiny(seed=0, r=r))
    K = 3
    o = O.nqp_opts(max_inner=K, eps=0.0)
    if t0:
        W, Ht, _, _ = O.nmf_solve(inst.W0, inst.Ht0, t0, V=inst.V, opts=o)
        inst.W0, inst.Ht0 = W, Ht
        inst = f32_inst(inst)
    Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, 1, V=inst.V, opts=o)
    W, Ht, hist, rep = run_solve(h, inst, 1, K, objective="direct")
    assert_iteration_rows(inst.V, inst.W0, inst.Ht0, to_np(W), to_np(Ht), K)
    tw, th = step_bounds(Wo, inst.Ht0, r)
    assert rel_err(to_np(W), Wo) < tw
    assert rel_err(to_np(Ht), Ho) < th
    assert abs(hist[0] - ho[1]) / ho[1] < j_bound(inst, Wo, Ho, tw, th)


@pytest.mark.parametrize("r", [64, 80])
def test_converged_iteration_both_preparations(h, r):
    """One outer iteration with every NQP solved to its unique minimiser,
    from the seeded start: at r = 64 the NQP kernel's epilogue prepares the
    solved factor (Gram partials, packed operand) for the next half-step, at
    r = 80 (RP = 128) the separate preparation kernels do; both against the
    oracle's converged iteration within the derived FP32 bounds."""
    inst = f32_inst(WL.tiny(seed=1, r=r, m=300, n=260))
    inst.beta_w = inst.beta_h = 0.1
    Wo, Ho, _, _ = O.nmf_solve(inst.W0, inst.Ht0, 1, V=inst.V, beta_w=0.1, beta_h=0.1,
                               opts=O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
    W, Ht, hist, rep = run_solve(h, inst, 1, 400, eps=1e-12, objective="direct")
    assert_iteration_rows(inst.V, inst.W0, inst.Ht0, to_np(W), to_np(Ht), None, bw=0.1, bh=0.1)
    tw, _ = step_bounds(Wo, inst.Ht0, r, 0.1, 0.1)
    assert rel_err(to_np(W), Wo) < tw
    # the H-update against the oracle's unique minimisers for the GPU's own W
    # (the W error carried through an ill-conditioned Q_H would make a loose bound)
    Wg = to_np(W).astype(np.float64)
    Qh = O.gram(Wg, 0.1)
    Hs, *_ = O.nnls_update(Qh, O.cross_dense(inst.V.T, Wg), 0.0, inst.Ht0,
                           O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
    assert rel_err(to_np(Ht), Hs) < nnls_tol(Qh, r)


def horizon(inst, T, K, **kw):
    """1/(1 - rho), rho = ||W_T - W_{T-1}|| / ||W_{T-1} - W_{T-2}|| on the
    oracle's own trajectory (a contracting iteration sums per-step errors over
    this many steps)."""
    o = O.nqp_opts(max_inner=K, eps=0.0)
    Ws = [O.nmf_solve(inst.W0, inst.Ht0, t, V=inst.V, opts=o, **kw)[0] for t in (T - 2, T - 1, T)]
    rho = np.linalg.norm(Ws[2] - Ws[1]) / max(np.linalg.norm(Ws[1] - Ws[0]), 1e-300)
    return 1.0 / (1.0 - min(rho, 0.99))


def test_solve_stable_run_tight(h):
    """P-run on a non-chaotic instance (L2 weight 10 on both factors: the
    oracle's own trajectory moves < 1e-9 in J for a 1e-7 input
    perturbation), 50 iterations, K = 3: objective at 1e-5, factors at the
    per-step bound summed over the contraction horizon."""
    inst = f32_inst(WL.tiny(seed=0, r=10))
    inst.beta_w = inst.beta_h = 10.0
    T, K = 50, 3
    kw = dict(beta_w=10.0, beta_h=10.0)
    Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V,
                                opts=O.nqp_opts(max_inner=K, eps=0.0), **kw)
    W, Ht, hist, rep = run_solve(h, inst, T, K, objective="direct")
    assert (np.abs(hist - ho[1::2]) / ho[1::2]).max() < 1e-5
    tw, th = step_bounds(Wo, Ho, 10, 10.0, 10.0)
    hz = horizon(inst, T, K, **kw)
    assert rel_err(to_np(W), Wo) < max(tw, th) * hz
    assert rel_err(to_np(Ht), Ho) < max(tw, th) * hz
    assert rep.iters_done == T


@pytest.mark.parametrize("r", [10, 4])
def test_solve_tiny_chaotic_trajectory(h, r):
    """The tiny instance is chaotic: the oracle itself moves by 2e-4 (r=10)
    in J for a 1e-7 relative perturbation of W0, and an FP32 emulation of the
    whole loop drifts to 1.7e-3.  So the trajectory is compared at 5e-2 and
    the per-step parity is carried by test_one_iteration_from_oracle_state."""
    inst = f32_inst(WL.tiny(seed=0, r=r))
    T, K = 50, 3
    Wo, Ho, ho, tot = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V,
                                  opts=O.nqp_opts(max_inner=K, eps=0.0))
    W, Ht, hist, rep = run_solve(h, inst, T, K, objective="direct")
    rel_j = np.abs(hist - ho[1::2]) / ho[1::2]
    assert rel_j.max() < 5e-2, rel_j.max()
    assert np.all(np.diff(hist) <= 1e-9 * hist[1:])
    assert rep.iters_done == T


def test_trace_identity_objective_error(h):
    """The same GPU run evaluated both ways (the factors are bitwise equal):
    the trace identity from FP32 Grams and cross terms differs from the
    element-wise FP64 residual by O(u ||V||^2 / J)."""
    g = WL.rng(42)
    m, n, r = 700, 400, 20
    W0 = g.random((m, r))
    H0 = g.random((r, n))
    V = np.clip(W0 @ H0 / (W0 @ H0).max() + np.abs(g.normal(0, 0.01, (m, n))), 0, 1)
    inst = f32_inst(WL.DenseInstance(V, g.random((m, r)), g.random((n, r)), r, beta_w=0.1,
                                     beta_h=0.1))
    T, K = 20, 2
    Wa, Ha, ha, _ = run_solve(h, inst, T, K, objective="trace")
    Wb, Hb, hb, _ = run_solve(h, inst, T, K, objective="direct")
    assert torch.equal(Wa, Wb) and torch.equal(Ha, Hb)
    vv = float(np.sum(inst.V ** 2))
    bound = 64 * U32 * vv / hb.min()
    assert (np.abs(ha - hb) / hb).max() < bound
    # the direct objective follows the oracle's trajectory (chaotic: compared
    # at 5e-2, see test_solve_tiny_chaotic_trajectory)
    Wo, Ho, ho, tot = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, beta_w=0.1, beta_h=0.1,
                                  opts=O.nqp_opts(max_inner=K, eps=0.0))
    assert abs(hb[0] - ho[1]) / ho[1] < 1e-4
    assert (np.abs(hb - ho[1::2]) / ho[1::2]).max() < 5e-2


def test_solve_sparse_l1(h):
    m, n, r = 1200, 700, 16
    rp, ci, va = WL.random_csr(5, m, n, 0.02, empty_rows=10)
    trp, tci, tva = WL.csr_transpose(rp, ci, va, m, n)
    g = WL.rng(6)
    W0 = g.random((m, r)).astype(np.float32).astype(np.float64)
    H0 = g.random((n, r)).astype(np.float32).astype(np.float64)
    T, K = 10, 2
    Wo, Ho, ho, tot = O.nmf_solve(W0, H0, T, csr=(rp, ci, va), csr_t=(trp, tci, tva),
                                  alpha_h=0.01, opts=O.nqp_opts(max_inner=K, eps=0.0))
    inst = WL.DenseInstance(None, W0, H0, r, alpha_h=0.01)
    sp = ((*csr_t(rp, ci, va), n), (*csr_t(trp, tci, tva), m))
    W, Ht, hist, rep = run_solve(h, inst, T, K, sparse=sp)
    assert (np.abs(hist - ho[1::2]) / ho[1::2]).max() < 1e-5
    # per-step bound (with the W error carried into the H-update) summed over
    # the run (this instance contracts: a 1e-7 input perturbation moves W by
    # 2e-7 over 10 iterations), so the horizon is at most T
    tw = nnls_tol(O.gram(Ho), r)
    qh = O.gram(Wo)
    th = nnls_tol(qh, r) + kappa(qh) * tw
    assert rel_err(to_np(W), Wo) < T * max(tw, th)
    assert rel_err(to_np(Ht), Ho) < T * max(tw, th)


def test_graph_replay_is_bitwise_equal_and_deterministic(h):
    inst = WL.tiny(seed=1, r=10)
    a = run_solve(h, inst, 15, 5, eps=1e-3)
    b = run_solve(h, inst, 15, 5, eps=1e-3, use_graph=True)
    c = run_solve(h, inst, 15, 5, eps=1e-3)
    for x, y in ((a, b), (a, c)):
        assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])
        assert np.array_equal(x[2], y[2])


def test_project_matches_oracle(h):
    g = WL.rng(8)
    rows, r = 3000, 64
    W = g.random((rows, r))
    W /= np.sqrt((W * W).sum(0, keepdims=True))
    W = W.astype(np.float32).astype(np.float64)
    rp, ci, va = WL.random_csr(9, 77, rows, 0.02, empty_rows=2)
    Q = O.gram(W)
    Cm = O.cross_csr(rp, ci, va.astype(np.float64), W)
    Xo, *_ = O.nnls_update(Q, Cm, 0.0, np.zeros((77, r)), O.nqp_opts(max_inner=300, eps=1e-10))
    Qt, d = P.nmf_rescale(h, P.nmf_gram(h, t32(W)))
    Hn = torch.zeros(77, r, device=dev())
    rpt, cit, vat = csr_t(rp, ci, va)
    P.nmf_project(h, Qt, d, t32(W), (rpt, cit, vat, rows), Hn,
                  P.nnls_opts(max_inner=300, eps=1e-10))
    h.sync()
    assert rel_err(to_np(Hn), Xo) < 1e-4
    assert np.all(to_np(Hn)[np.diff(rp) == 0] == 0)


def test_nonfinite_input_is_reported(h):
    Q, Cm, X0 = nqp_batch(3, 8, 64)
    Qt, d, _ = O.rescale(Q)
    Cm[5, 2] = np.nan
    X = t32(X0)
    P.nmf_nnls_update(h, t32(Qt), t32(d), t32(Cm), X)
    with pytest.raises(P.NmfError) as e:
        h.sync()
    assert e.value.status == P.NMF_E_NONFINITE
    assert torch.equal(X[5], t32(X0)[5])       # row left unchanged
    h.sync()                                   # status was cleared


def test_zero_rows_and_bad_rank(h):
    Qt = t32(np.eye(4))
    d = t32(np.ones(4))
    X = torch.empty(0, 4, device=dev())
    P.nmf_nnls_update(h, Qt, d, X, X)
    h.sync()
    with pytest.raises(P.NmfError):
        P.nmf_rescale(h, t32(np.eye(129)))


def test_sharded_schedule_single_rank_on_gpu(h):
    """The multi-GPU schedule's device ops (one rank, no collective) give one
    outer iteration within the per-step FP32 bounds of the oracle's."""
    from paper_1506_08938_gb300.sharded import GpuOps, ShardOpts, sharded_iteration
    inst = f32_inst(WL.tiny(seed=2, r=10))
    K = 3
    ops = GpuOps(h, P.nnls_opts(max_inner=K, eps=0.0))
    V = t32(inst.V)
    W, Ht = sharded_iteration(V, V.t().contiguous(), t32(inst.W0), t32(inst.Ht0), ops,
                              ShardOpts())
    Wo, Ho, _, _ = O.nmf_solve(inst.W0, inst.Ht0, 1, V=inst.V, opts=O.nqp_opts(max_inner=K, eps=0.0))
    tw, th = step_bounds(Wo, inst.Ht0, 10)
    assert rel_err(to_np(W), Wo) < tw
    assert rel_err(to_np(Ht), Ho) < th


def test_solve_fast_break_previous_update(h):
    """maxStop mode 1 inside the solve (Alg. 3's fast break, deterministic
    reading: the threshold of an update is the largest final ||f~||^2 of the
    previous update of the same factor, 0 before the first).  Against the
    oracle's mode 1 on the damped instance: a row near a threshold may stop
    one inner iteration apart in FP32 and FP64, moving J by a fraction of
    that iteration's decrease, so each iteration's J agrees to 5% of the
    oracle's decrease (plus the FP32 objective tolerance 1e-5); the fast
    break must cut the inner iterations, to within 5% of the oracle's count."""
    import ctypes as C
    inst = f32_inst(WL.tiny(seed=0, r=10))
    T, beta = 20, 10.0
    out = {}
    for mode in (0, 1):
        W, Ht = t32(inst.W0), t32(inst.Ht0)
        hist = np.zeros(T)
        o = P.solve_opts(T, beta_w=beta, beta_h=beta, objective="direct",
                         nnls=P.nnls_opts(max_inner=50, eps=1e-3, maxstop_mode=mode),
                         obj_hist=hist.ctypes.data_as(C.POINTER(C.c_double)))
        rep = P.nmf_solve(h, t32(inst.V), W, Ht, o)
        out[mode] = (hist.copy(), rep.inner_total)
    Wo, Ho, ho, tot = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, beta_w=beta, beta_h=beta,
                                  opts=O.nqp_opts(max_inner=50, eps=1e-3, maxstop_mode=1))
    J0 = O.objective_dense(inst.V, inst.W0, inst.Ht0, 0.0, 0.0, beta, beta)
    oj = ho[1::2]
    dec = np.abs(np.diff(np.concatenate([[J0], oj])))
    dev = np.abs(out[1][0] - oj)
    assert np.all(dev <= 0.05 * dec + 1e-5 * oj), (dev, dec)
    assert out[1][1] < out[0][1]
    assert abs(out[1][1] - tot) <= 0.05 * tot


# L1 (a) and L2 (b) weights on either factor or both (§3.5; reading R2: b is
# the paper's 2 mu_2, so its mu_2 = 1e-2 cases are b = 0.02)
PENALTIES = [(0.01, 0.0, 0.0, 0.0), (0.0, 0.01, 0.0, 0.0), (0.01, 0.01, 0.0, 0.0),
             (0.0, 0.0, 0.02, 0.0), (0.0, 0.0, 0.0, 0.02), (0.0, 0.0, 0.02, 0.02),
             (0.01, 0.01, 0.02, 0.02), (1.0, 0.0, 0.0, 0.0), (0.0, 0.5, 0.0, 1.0)]


@pytest.mark.parametrize("aw,ah,bw,bh", PENALTIES)
def test_penalty_grid_one_iteration(h, aw, ah, bw, bh):
    """One outer iteration with L1/L2 weights on W, Ht or both, from the same
    FP32 start: W rows by the fixed-K rule (its inputs are exact), Ht within
    its bound plus kappa(Q_H) times the W error actually made, J within the
    first-order bound of those errors (data and penalty terms)."""
    inst = f32_inst(WL.tiny(seed=7, r=10))
    inst.alpha_w, inst.alpha_h, inst.beta_w, inst.beta_h = aw, ah, bw, bh
    K = 3
    W, Ht, hist, rep = run_solve(h, inst, 1, K, objective="direct")
    Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, 1, V=inst.V, alpha_w=aw, alpha_h=ah,
                                beta_w=bw, beta_h=bh, opts=O.nqp_opts(max_inner=K, eps=0.0))
    Qw = O.gram(inst.Ht0, bw)
    Wg, Hg = to_np(W), to_np(Ht)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert_iteration_rows(inst.V, inst.W0, inst.Ht0, Wg, Hg, K, aw, ah, bw, bh)
    ew = max(nnls_tol(Qw, 10), rel_err(Wg, Wo))
    Qh = O.gram(Wo, bh)
    eh = nnls_tol(Qh, 10) + kappa(Qh) * ew
    assert rel_err(Hg, Ho) < eh
    # first-order bound: the data term as in j_bound, plus the penalty terms'
    # changes (|sum dW| <= sqrt(m r) ||dW||, d||W||^2/2 <= ||W|| ||dW||)
    nw, nh = np.linalg.norm(Wo), np.linalg.norm(Ho)
    pen = (aw * np.sqrt(Wo.size) * ew * nw + ah * np.sqrt(Ho.size) * eh * nh +
           bw * nw * nw * ew + bh * nh * nh * eh)
    jb = j_bound(inst, Wo, Ho, ew, eh) * O.objective_dense(inst.V, Wo, Ho) + pen
    assert abs(hist[0] - ho[1]) < max(1e-5 * ho[1], jb)


def test_peak_probes(h):
    """The measured roofs the benchmark divides by: FP32 FFMA throughput, the
    L2-resident row-gather bandwidth of the sparse cross term, and the dense
    BF16 rate of the library's tcgen05.mma path on an r = 512 contraction
    (152 SMs at their 2.07 GHz maximum clock bound it near 2.6 PFLOP/s: a
    rate above that means MMAs were not issued)."""
    tf = P.nmf_peak_fp32()
    assert 10.0 < tf < 200.0
    gbs = P.nmf_peak_l2_gather(100)
    assert 500.0 < gbs < 100000.0
    with pytest.raises(P.NmfError):
        P.nmf_peak_l2_gather(129)
    tc = P.nmf_peak_tc_bf16(h)
    print(f"tcgen05 bf16 r = 512 probe: {tc:.0f} TFLOP/s")
    assert 100.0 < tc < 2600.0
