"""Failure paths, made on the host (the NMF_FAULT injection sites of
include/nmf.h) - nothing here traps, faults or hangs the GPU:

* a bounded device wait runs out: the persistent batched launch's grid
  barrier gets a deadline that has already passed, every waiting CTA gives
  up, NMF_E_TIMEOUT comes back through the device status word, and the next
  call on the same handle runs normally and gives the bitwise result of an
  undisturbed run;
* the server refuses admission (NMF_E_BUSY) or a request's CSR fails
  validation (NMF_E_ARG), and serves normally once the fault is gone;
* a workspace allocation fails (NMF_E_NOMEM) and a later call succeeds.
"""
import numpy as np
import pytest

import workloads as WL
from tests.gpu_common import t32, to_np, torch
from tests.test_gpu_batched import device_instances, make_instances
from tests.test_gpu_serving import requests

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")


@pytest.fixture(scope="module")
def h():
    import __graft_entry__ as g
    g.build()
    hh = P.Handle(0)
    yield hh
    hh.close()


def test_grid_barrier_timeout_reported_and_context_usable(h, monkeypatch):
    insts = make_instances([(300, 120, 5), (90, 130, 50)], seed=2)
    o = P.solve_opts(3, nnls=P.nnls_opts(max_inner=3, eps=0.0), use_graph=False)
    ref = device_instances(insts)
    P.nmf_solve_batched(h, ref, o, mode="persistent")
    dv = device_instances(insts)
    monkeypatch.setenv("NMF_FAULT", "barrier")
    with pytest.raises(P.NmfError) as e:
        P.nmf_solve_batched(h, dv, o, mode="persistent")
    assert e.value.status == P.NMF_E_TIMEOUT
    monkeypatch.delenv("NMF_FAULT")
    dv = device_instances(insts)
    P.nmf_solve_batched(h, dv, o, mode="persistent")     # the status was read and cleared
    for (_, _, W, Ht), (_, _, Wr, Hr) in zip(dv, ref):
        assert torch.equal(W, Wr) and torch.equal(Ht, Hr)


def test_server_admission_and_csr_faults(monkeypatch):
    wl = WL.serving(seed=3, rows=2000, r=16, rate=1.0, duration=1.0, max_requests=0)
    srv = P.Server(t32(wl.W), slots=2, max_batch_cols=1024, max_batch_nnz=1 << 16,
                   hbm_budget=1 << 26)
    rq = requests(4, 1, 2000, max_width=40, nnz=10)[0]
    try:
        monkeypatch.setenv("NMF_FAULT", "admit")
        with pytest.raises(P.NmfError) as e:
            srv.submit(*rq)
        assert e.value.status == P.NMF_E_BUSY
        monkeypatch.setenv("NMF_FAULT", "csr")
        with pytest.raises(P.NmfError) as e:
            srv.submit(*rq)
        assert e.value.status == P.NMF_E_ARG
        monkeypatch.delenv("NMF_FAULT")
        t, out = srv.submit(*rq)
        srv.wait(t)
        assert np.all(np.isfinite(out)) and np.all(out >= 0)
        assert srv.stats()["completed"] == 1
    finally:
        srv.close()


def test_workspace_allocation_fault(monkeypatch):
    hh = P.Handle(0)      # a fresh handle: no workspace yet
    X = t32(WL.rng(1).random((500, 12)))
    try:
        monkeypatch.setenv("NMF_FAULT", "alloc")
        with pytest.raises(P.NmfError) as e:
            P.nmf_gram(hh, X)
        assert e.value.status == P.NMF_E_NOMEM
        monkeypatch.delenv("NMF_FAULT")
        Q = P.nmf_gram(hh, X)
        hh.sync()
        Xd = to_np(X)
        assert np.allclose(to_np(Q), Xd.T @ Xd, rtol=2e-6)
    finally:
        hh.close()
