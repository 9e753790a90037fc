"""Continuous-batching projection server (nmf_server_*): results against the
oracle, bitwise identity of every request's result alone and inside a
concurrent mix, admission by device-memory budget, and bounded waits."""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from tests.gpu_common import dev, t32, torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")


@pytest.fixture(scope="module")
def basis():
    import __graft_entry__ as g
    g.build()
    wl = WL.serving(seed=3, rows=5000, r=64, rate=1.0, duration=1.0, max_requests=0)
    return wl.W


def requests(seed, count, rows, max_width=300, nnz=20):
    g = WL.rng(seed)
    out = []
    for _ in range(count):
        w = int(g.integers(1, max_width + 1))
        cols = WL.zipf_rows(g, np.full(w, nnz, dtype=np.int64), rows, 1.1)
        rp = np.zeros(w + 1, dtype=np.int64)
        rp[1:] = np.cumsum([len(c) for c in cols])
        ci = np.concatenate([np.sort(c) for c in cols]).astype(np.int32)
        va = (g.poisson(2.0, size=len(ci)) + 1).astype(np.float32)
        out.append((rp, ci, va))
    return out


def test_server_alone_equals_mix_and_matches_oracle(basis):
    W = t32(basis)
    reqs = requests(7, 12, basis.shape[0])
    nn = P.nnls_opts(max_inner=300, eps=1e-10)
    srv = P.Server(W, slots=3, max_batch_cols=600, max_batch_nnz=20000, hbm_budget=1 << 26,
                   nnls=nn)
    alone = []
    for rp, ci, va in reqs:
        t, out = srv.submit(rp, ci, va)
        srv.wait(t)
        alone.append(out.copy())
    tickets = [srv.submit(rp, ci, va) for rp, ci, va in reqs]
    mix = []
    for t, out in tickets:
        srv.wait(t)
        mix.append(out)
    st = srv.stats()
    srv.close()
    for a, b in zip(alone, mix):
        assert np.array_equal(a, b)
    assert st["completed"] == 24 and st["batches"] < 24   # the mix was batched
    # against the oracle's converged NNLS (unique minimiser: the basis Gram is
    # positive definite), bound from its conditioning
    Wd = basis.astype(np.float64)
    Q = O.gram(Wd)
    Qt, _, _ = O.rescale(Q)
    ev = np.linalg.eigvalsh(Qt)
    tol = max(1e-5, 16 * np.sqrt(64) * ev[-1] / ev[0] * 2.0 ** -24)
    for (rp, ci, va), got in list(zip(reqs, alone))[:3]:
        Cm = O.cross_csr(rp, ci, va.astype(np.float64), Wd)
        Xo, *_ = O.nnls_update(Q, Cm, 0.0, np.zeros_like(Cm),
                               O.nqp_opts(max_inner=5000, eps=0.0, abs_tol=1e-24))
        assert np.linalg.norm(got - Xo) / np.linalg.norm(Xo) < tol


def test_server_admission_by_budget(basis):
    W = t32(basis)
    reqs = requests(9, 16, basis.shape[0], max_width=200)
    # budget for about one full batch: the rest must wait for memory to free up
    per = 8 * 201 + 8 * 200 * 20 + 2 * 4 * 200 * 64 + 4 * 256
    srv = P.Server(W, slots=4, max_batch_cols=200, max_batch_nnz=4000, hbm_budget=per)
    tickets = [srv.submit(rp, ci, va) for rp, ci, va in reqs]
    for t, _ in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["completed"] == 16 and st["inflight_bytes"] == 0
    # a request wider than a slot can never be admitted: refused up front
    rp, ci, va = requests(10, 1, basis.shape[0], max_width=1)[0]
    big_rp = np.arange(0, 20 * 301, 20, dtype=np.int64)
    big_ci = np.tile(ci[:1], 20 * 300).astype(np.int32)
    with pytest.raises(P.NmfError) as e:
        srv.submit(big_rp, big_ci, np.ones(20 * 300, dtype=np.float32))
    assert e.value.status == P.NMF_E_BUSY
    # a wait on a ticket that never completes ends with a timeout, not a hang
    with pytest.raises(P.NmfError) as e:
        srv.wait(10 ** 9, timeout=0.2)
    assert e.value.status == P.NMF_E_TIMEOUT
    srv.close()


def test_server_rejects_malformed_requests(basis):
    W = t32(basis)
    srv = P.Server(W, slots=1)
    with pytest.raises(P.NmfError):
        srv.submit(np.array([0, 2], dtype=np.int64), np.array([0, basis.shape[0]], dtype=np.int32),
                   np.ones(2, dtype=np.float32))
    srv.close()
