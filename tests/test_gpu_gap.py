"""The solve's stop at a relative objective gap (A7: the outer loop runs until
(J - J*) / J* <= target): a run with the objective recorded every iteration
gives the trajectory, which a gap-targeted run follows exactly (computing
the objective does not change the factors).

* fixed test interval k: the run stops at the first multiple of k at or
  after the first iteration whose gap meets the target, and reports that
  iteration's objective and gap (J* = the recorded run's final objective,
  the target = its gap after half the iterations);
* adaptive tests (check_every < 0): the run stops with the gap met, never
  before the first iteration that meets it, and at most 20% + 16 iterations
  after it;
* a target that is never met runs all iterations.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as WL
from tests.gpu_common import t32

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")

T = 400


@pytest.fixture(scope="module")
def h():
    import __graft_entry__ as g
    g.build()
    hh = P.Handle(0)
    yield hh
    hh.close()


@pytest.fixture(scope="module")
def traj(h):
    inst = WL.tiny(seed=0, r=10)
    V = t32(inst.V)
    hist = np.zeros(T)
    W, Ht = t32(inst.W0), t32(inst.Ht0)
    o = P.solve_opts(T, nnls=P.nnls_opts(max_inner=50, eps=1e-3), objective="direct",
                     check_every=0, obj_hist=hist.ctypes.data_as(C.POINTER(C.c_double)))
    P.nmf_solve(h, V, W, Ht, o)
    # J* = the run's final objective; the target = the gap the run has after
    # T / 2 iterations, so the first iteration that meets it lies mid-run
    assert np.all(np.diff(hist) <= 0.0)
    fstar = float(hist[-1])
    gap = (hist - fstar) / fstar
    target = float(gap[T // 2 - 1])
    first = int(np.argmax(gap <= target)) + 1   # iterations done when first met
    print(f"trajectory: J* {fstar:.6g}, target {target:.3e}, first iteration at it {first}")
    assert target > 0 and first + 0.2 * first + 16 < T
    return inst, V, hist, fstar, gap, first, target


def gap_run(h, inst, V, fstar, check, target):
    W, Ht = t32(inst.W0), t32(inst.Ht0)
    o = P.solve_opts(T, rel_gap_target=target, f_star=fstar,
                     nnls=P.nnls_opts(max_inner=50, eps=1e-3), objective="direct",
                     check_every=check)
    return P.nmf_solve(h, V, W, Ht, o)


@pytest.mark.parametrize("k", [1, 7])
def test_fixed_interval_stops_at_first_test_past_the_gap(h, traj, k):
    inst, V, hist, fstar, gap, first, target = traj
    rep = gap_run(h, inst, V, fstar, k, target)
    expect = -(-first // k) * k
    assert rep.iters_done == expect
    assert rep.objective == hist[expect - 1]
    assert abs(rep.rel_gap - gap[expect - 1]) <= 1e-12 and rep.rel_gap <= target


def test_adaptive_tests_stop_soon_after_the_gap(h, traj):
    inst, V, hist, fstar, gap, first, target = traj
    rep = gap_run(h, inst, V, fstar, -1, target)
    print(f"first iteration at the gap {first}, adaptive stop {rep.iters_done}")
    assert rep.rel_gap <= target
    assert first <= rep.iters_done <= first + 0.2 * first + 16
    assert rep.objective == hist[rep.iters_done - 1]


def test_unmet_target_runs_every_iteration(h, traj):
    inst, V, hist, fstar, gap, first, target = traj
    # J* 1% below the trajectory's end: every gap is at least ~1e-2
    rep = gap_run(h, inst, V, fstar * (1 - 1e-2), -1, 1e-4)
    assert rep.iters_done == T
    assert rep.rel_gap > 0
