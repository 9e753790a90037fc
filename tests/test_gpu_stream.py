"""One-pass streamed solve (nmf_solve_streamed: Alg. 2's E-step accumulation
of V_b^T W_b and W_b^T W_b chunk by chunk, V read once per outer iteration)
through the C ABI:

* V in host memory (the limited-internal-memory mode) and V on the device,
  same chunking: bitwise the same factors and objective;
* one iteration from the seeded start against the oracle row by row (W rows
  against the oracle's W-update, Ht rows against its H-update from the GPU's
  own W), with a ragged last chunk, a single chunk, and both cross-term paths
  (tensor cores for n % 4 == 0, CUDA cores otherwise); J by the trace
  identity within its O(u ||V||^2 / J) bound;
* the full dense workload, V in pinned host memory, three iterations with
  every NQP solved to its minimiser: J within 1e-5 of the FP64 oracle's
  converged run (tests/golden).
"""
import ctypes as C
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as WL
from tests.gpu_common import U32, t32, to_np, torch
from tests.test_gpu_parity import assert_iteration_rows, f32_inst

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")
GOLD = os.path.join(os.path.dirname(__file__), "golden", "dense10000x4096_prun.json")


@pytest.fixture(scope="module")
def h():
    import __graft_entry__ as g
    g.build()
    hh = P.Handle(0)
    yield hh
    hh.close()


def streamed(h, V, W0, H0, T, chunk, K=3, eps=0.0, beta=0.0, hist=None, **nn):
    W, Ht = t32(W0), t32(H0)
    hp = hist.ctypes.data_as(C.POINTER(C.c_double)) if hist is not None else None
    o = P.solve_opts(T, beta_w=beta, beta_h=beta, nnls=P.nnls_opts(max_inner=K, eps=eps, **nn),
                     obj_hist=hp)
    rep = P.nmf_solve_streamed(h, V, W, Ht, o, chunk)
    return W, Ht, rep


@pytest.mark.parametrize("m,n,chunk", [(200, 152, 64), (200, 152, 200), (300, 150, 77),
                                       (1000, 600, 256)])
def test_streamed_host_equals_device_and_matches_oracle(h, m, n, chunk):
    inst = f32_inst(WL.tiny(seed=5, r=10, m=m, n=n))
    Vd = t32(inst.V)
    Vh = torch.tensor(inst.V, dtype=torch.float32).pin_memory()
    Wd, Hd, rd = streamed(h, Vd, inst.W0, inst.Ht0, 1, chunk)
    Wh, Hh, rh = streamed(h, Vh, inst.W0, inst.Ht0, 1, chunk)
    assert torch.equal(Wd, Wh) and torch.equal(Hd, Hh) and rd.objective == rh.objective
    assert_iteration_rows(inst.V, inst.W0, inst.Ht0, to_np(Wd), to_np(Hd), 3)
    Jo = O.objective_dense(inst.V, to_np(Wd), to_np(Hd))
    vv = float(np.sum(inst.V ** 2))
    assert abs(rd.objective - Jo) / Jo < 64 * U32 * vv / Jo
    assert rd.iters_done == 1


def test_streamed_several_iterations_host_equals_device(h):
    inst = f32_inst(WL.tiny(seed=6, r=8, m=500, n=300))
    Vh = torch.tensor(inst.V, dtype=torch.float32).pin_memory()
    a = streamed(h, t32(inst.V), inst.W0, inst.Ht0, 6, 128, K=5, eps=1e-3)
    b = streamed(h, Vh, inst.W0, inst.Ht0, 6, 128, K=5, eps=1e-3)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[2].objective == b[2].objective and a[2].inner_total == b[2].inner_total


def test_streamed_dense_host_tracks_oracle_converged(h):
    """Three converged iterations of the dense workload with V in pinned host
    memory; after each, the FP64 element-wise objective of the factors (the
    library's nmf_objective_direct, V copied to the device for it) within
    1e-5 of the oracle's converged run - or of the FP32 error of its
    worst-conditioned half-step so far carried on by the run's sensitivity
    (the bound of tests/test_gpu_prun.py) - and the streamed solve's own trace
    identity within its O(u ||V||^2 / J) bound of that."""
    from tests.test_gpu_prun import propagated
    if not os.path.exists(GOLD):
        pytest.skip("oracle P-run data not generated (oracle/make_dense_prun.py)")
    gold = json.load(open(GOLD))
    cv = gold["converged"]
    Jo = np.array(cv["J"][:3])
    kap = np.maximum(np.array(cv["kappa"][0::2]), np.array(cv["kappa"][1::2]))
    bj = propagated(1e-5, kap, cv["sensitivity"]["J"])
    inst = WL.dense(seed=0)
    Vh = torch.from_numpy(np.ascontiguousarray(inst.V)).pin_memory()
    Vd = Vh.cuda()
    vv = float(np.sum(inst.V.astype(np.float64) ** 2))
    for t in (1, 2, 3):
        W, Ht, rep = streamed(h, Vh, inst.W0, inst.Ht0, t, 1024, K=2000, eps=0.0, beta=0.1,
                              grad_refresh=10)
        J = P.nmf_objective_direct(h, Vd, W, Ht, 0.0, 0.0, 0.1, 0.1)
        h.sync()
        rel = abs(J.item() - Jo[t - 1]) / Jo[t - 1]
        print(f"streamed dense (host V) t={t}: rel J {rel:.2e} (bound {bj[t - 1]:.1e}), "
              f"trace identity {abs(rep.objective - J.item()) / J.item():.2e}")
        assert rel <= bj[t - 1]
        assert abs(rep.objective - J.item()) / J.item() <= 8 * U32 * vv / J.item()
