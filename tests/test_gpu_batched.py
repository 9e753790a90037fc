"""Many independent instances in one launch per outer iteration (Alg. 2 per
instance), against the FP64 oracle run instance by instance.

* Every launch shape (persistent with or without a CUDA graph, the
  per-instance loop, the autotuned shape) performs the same arithmetic in
  the same order for every instance, so their results are bitwise equal.
* One iteration from the same FP32 start: the W half-step has exact inputs,
  so its rows are held to the FP32 NNLS bound (a flipped near-tie in a
  greedy step may instead reach the oracle's objective); the H half-step
  carries the W error through kappa(Q_H).
* A damped run (L2 weight 10, a contracting trajectory) stays on the
  oracle's trajectory: objective at 1e-5, factors within the per-step bound
  summed over the contraction horizon.
"""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from tests.gpu_common import rel_err, t32, to_np, torch
from tests.test_gpu_parity import (assert_iteration_rows, horizon, j_bound, kappa, nnls_tol,
                                   step_bounds)

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")

# (m, n, r): ranks on both sides of the 32-wide lane split, one instance
# spanning several Gram (256 rows), cross (64 rows) and NNLS work items
SHAPES = [(40, 33, 1), (300, 120, 5), (97, 280, 8), (1100, 70, 17), (64, 64, 32),
          (150, 211, 33), (90, 130, 50), (257, 300, 64)]


@pytest.fixture(scope="module")
def h():
    import __graft_entry__ as g
    g.build()
    hh = P.Handle(0)
    yield hh
    hh.close()


def make_instances(shapes, seed=0, beta=0.0):
    out = []
    for k, (m, n, r) in enumerate(shapes):
        inst = WL.batched(seed=seed + 7 * k, count=1, m_range=(m, m), n_range=(n, n),
                          ranks=(r,))[0]
        for a in ("V", "W0", "Ht0"):
            setattr(inst, a, getattr(inst, a).astype(np.float32).astype(np.float64))
        inst.beta_w = inst.beta_h = beta
        out.append(inst)
    return out


def device_instances(insts):
    dv = []
    for inst in insts:
        V = t32(inst.V)
        dv.append((V, V.t().contiguous(), t32(inst.W0), t32(inst.Ht0)))
    return dv


def run_batched(h, insts, T, K, mode="persistent", use_graph=True, beta=0.0):
    dv = device_instances(insts)
    o = P.solve_opts(T, beta_w=beta, beta_h=beta, nnls=P.nnls_opts(max_inner=K, eps=0.0),
                     use_graph=use_graph)
    reps = P.nmf_solve_batched(h, dv, o, mode=mode)
    return [(to_np(W), to_np(Ht)) for (_, _, W, Ht) in dv], reps


def test_launch_shapes_are_bitwise_equal(h):
    insts = make_instances(SHAPES * 2, seed=11)
    T, K = 8, 3
    ref, _ = run_batched(h, insts, T, K, "persistent", use_graph=False)
    for mode, graph in (("persistent", True), ("loop", False), ("autotune", True),
                        ("phases", False)):
        got, reps = run_batched(h, insts, T, K, mode, use_graph=graph)
        for (W, Ht), (Wr, Hr) in zip(got, ref):
            assert np.array_equal(W, Wr), mode
            assert np.array_equal(Ht, Hr), mode
        assert all(rp.iters_done == T for rp in reps)


def test_results_do_not_depend_on_instance_order(h):
    """The library orders its device list by cost and CTAs take work items
    in whatever order they finish: an instance's factors and report must be
    bitwise the same wherever it sits in the caller's list."""
    insts = make_instances(SHAPES, seed=13)
    T, K = 6, 3
    ref, rref = run_batched(h, insts, T, K, "persistent")
    perm = [5, 0, 7, 2, 6, 1, 4, 3]
    got, rgot = run_batched(h, [insts[i] for i in perm], T, K, "persistent")
    for j, i in enumerate(perm):
        assert np.array_equal(got[j][0], ref[i][0]) and np.array_equal(got[j][1], ref[i][1]), i
        assert rgot[j].objective == rref[i].objective, i


def test_one_iteration_matches_oracle(h):
    insts = make_instances(SHAPES, seed=3)
    K = 3
    got, reps = run_batched(h, insts, 1, K)
    o = O.nqp_opts(max_inner=K, eps=0.0)
    for inst, (W, Ht), rp in zip(insts, got, reps):
        Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, 1, V=inst.V, opts=o)
        Qw = O.gram(inst.Ht0, 0.0)
        # row by row: W against the oracle's W-update, Ht against the
        # oracle's H-update from this W (near-ties named)
        assert_iteration_rows(inst.V, inst.W0, inst.Ht0, W, Ht, K)
        # the H half-step inherits the W error actually made (a flipped
        # near-tie may exceed the per-row bound) through kappa(Q_H)
        ew = max(nnls_tol(Qw, inst.r), rel_err(W, Wo))
        Qh = O.gram(Wo, 0.0)
        eh = nnls_tol(Qh, inst.r) + kappa(Qh) * ew
        assert rel_err(Ht, Ho) < eh, inst.name
        Jo = ho[1]
        assert abs(rp.objective - Jo) / Jo < j_bound(inst, Wo, Ho, ew, eh), inst.name
        # the reported objective is the element-wise J of the returned factors
        Jr = O.objective_dense(inst.V, W, Ht)
        assert abs(rp.objective - Jr) / Jr < 1e-6


def test_damped_run_stays_on_the_oracle_trajectory(h):
    beta = 10.0
    insts = make_instances(SHAPES[:6], seed=5, beta=beta)
    T, K = 10, 3
    got, reps = run_batched(h, insts, T, K, beta=beta)
    o = O.nqp_opts(max_inner=K, eps=0.0)
    for inst, (W, Ht), rp in zip(insts, got, reps):
        kw = dict(beta_w=beta, beta_h=beta)
        Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, opts=o, **kw)
        assert abs(rp.objective - ho[-1]) / ho[-1] < 1e-5, inst.name
        tw, th = step_bounds(Wo, Ho, inst.r, beta, beta)
        hz = horizon(inst, T, K, **kw)
        assert rel_err(W, Wo) < max(tw, th) * hz, inst.name
        assert rel_err(Ht, Ho) < max(tw, th) * hz, inst.name


def test_rejects_bad_instances(h):
    insts = make_instances([(40, 30, 4)])
    dv = device_instances(insts)
    o = P.solve_opts(1)
    V, Vt, W, Ht = dv[0]
    big = torch.zeros((40, 65), dtype=torch.float32, device=W.device)
    big_h = torch.zeros((30, 65), dtype=torch.float32, device=W.device)
    with pytest.raises(P.NmfError):
        P.nmf_solve_batched(h, [(V, Vt, big, big_h)], o)        # r > 64
    with pytest.raises(ValueError):
        P.nmf_solve_batched(h, [(V, V, W, Ht)], o)              # Vt of the wrong shape
    with pytest.raises(P.NmfError):
        P.nmf_solve_batched(h, [], o)                           # no instances
