"""Many independent instances in one launch per outer iteration (Alg. 2 per
instance), against the FP64 oracle run instance by instance.

* Every launch shape (persistent with or without a CUDA graph, the
  per-instance loop, the autotuned shape) performs the same arithmetic in
  the same order for every instance, so their results are bitwise equal.
* One iteration from the same FP32 start: the W half-step has exact inputs,
  so its rows are held to the FP32 NNLS bound (a flipped near-tie in a
  greedy step may instead reach the oracle's objective); the H half-step
  carries the W error through kappa(Q_H).
* The cross phase alone: with one nonzero per row of H0 the Gram is
  diagonal, the W half-step's NQPs decouple, and their minimiser is the
  cross term divided by the Gram's diagonal - checked element by element
  against the FP64 product.
* Damped runs (L2 weight 10): with converged inner solves (a continuous map)
  every instance stays on the oracle's trajectory, objective at 1e-5 and
  factors within the per-step bound summed over the contraction horizon;
  with K = 3 fixed inner iterations the greedy choices of Alg. 3 can flip on
  near-ties, so the same bar holds on the instances whose own oracle run
  moves less than 1e-7 in J under a 1e-7 relative perturbation of V (the
  others are covered by the converged run and the one-iteration rows).
Each check runs with the cross phase on the tensor cores (prec fp32: 3xTF32
tcgen05 MMAs, each 32-wide k block added into FP32 registers) and on the
CUDA cores (prec fp32_simt: one FFMA per term).
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


PRECS = ["fp32", "fp32_simt"]


def run_batched(h, insts, T, K, mode="persistent", use_graph=True, beta=0.0, prec="fp32"):
    dv = device_instances(insts)
    o = P.solve_opts(T, beta_w=beta, beta_h=beta, nnls=P.nnls_opts(max_inner=K, eps=0.0),
                     use_graph=use_graph, prec=prec)
    reps = P.nmf_solve_batched(h, dv, o, mode=mode)
    return [(to_np(W), to_np(Ht)) for (_, _, W, Ht) in dv], reps


@pytest.mark.parametrize("prec", PRECS)
def test_launch_shapes_are_bitwise_equal(h, prec):
    insts = make_instances(SHAPES * 2, seed=11)
    T, K = 8, 3
    ref, _ = run_batched(h, insts, T, K, "persistent", use_graph=False, prec=prec)
    for mode, graph in (("persistent", True), ("loop", False), ("autotune", True),
                        ("phases", False)):
        got, reps = run_batched(h, insts, T, K, mode, use_graph=graph, prec=prec)
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


@pytest.mark.parametrize("prec", PRECS)
def test_one_iteration_matches_oracle(h, prec):
    insts = make_instances(SHAPES, seed=3)
    K = 3
    got, reps = run_batched(h, insts, 1, K, prec=prec)
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


def cross_tol(K):
    """FP32-grade error of an element of C / diag(Q) (C = A B over K terms):
    a few roundings in the Gram, rescale, NQP and division (measured up to
    5.9e-7 on either arithmetic at K = 33) plus the summation's random walk,
    ~u sqrt(K) / 4 per term scale (measured 1.2e-6 at K = 4000 on the tensor
    cores, 8.4e-7 on the CUDA cores).  A dropped A_lo B_hi or A B_lo term
    (2^-12 of a product on average) or a truncating accumulation over the
    whole k range would exceed it."""
    return 1e-6 + 2.5e-8 * np.sqrt(K)


@pytest.mark.parametrize("prec", PRECS)
def test_cross_phase_against_fp64_product(h, prec):
    shapes = SHAPES + [(129, 1000, 64), (700, 2000, 16), (3000, 4000, 32)]
    insts = make_instances(shapes, seed=21)
    for inst in insts:
        n, r = inst.Ht0.shape
        g = np.random.default_rng(n * 131 + r)
        H = np.zeros((n, r))
        H[np.arange(n), np.arange(n) % r] = g.uniform(0.5, 1.0, n)   # every column used (n >= r)
        inst.Ht0 = H.astype(np.float32).astype(np.float64)
    got, _ = run_batched(h, insts, 1, 20, prec=prec)
    for inst, (W, _) in zip(insts, got):
        q = (inst.Ht0 ** 2).sum(axis=0)
        Wx = (inst.V @ inst.Ht0) / q          # V > 0: every entry positive
        err = np.abs(W - Wx) / Wx
        print(f"{prec} {inst.name}: max {err.max():.2e}, mean {err.mean():.2e}")
        assert err.max() < cross_tol(inst.n), inst.name


def oracle_spread(inst, T, o, kw, level=1e-7, reps=4):
    """The oracle's own J response to a relative `level` perturbation of V."""
    _, _, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, opts=o, **kw)
    g = np.random.default_rng(17)
    out = 0.0
    for _ in range(reps):
        Vp = inst.V * (1 + level * g.standard_normal(inst.V.shape))
        _, _, hp, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=Vp, opts=o, **kw)
        out = max(out, abs(hp[-1] - ho[-1]) / ho[-1])
    return out


def converged_horizon(inst, T, o, kw):
    """horizon() for the converged inner solves of `o` (stopped at its
    absolute tolerance instead of a fixed iteration count)."""
    Ws = [O.nmf_solve(inst.W0, inst.Ht0, t, V=inst.V, opts=o, **kw)[0] for t in (T - 2, T - 1, T)]
    rho = np.linalg.norm(Ws[2] - Ws[1]) / max(np.linalg.norm(Ws[1] - Ws[0]), 1e-300)
    return 1.0 / (1.0 - min(rho, 0.99))


@pytest.mark.parametrize("prec", PRECS)
def test_converged_damped_run_stays_on_the_oracle_trajectory(h, prec):
    beta = 10.0
    insts = make_instances(SHAPES, seed=5, beta=beta)
    T, K = 10, 300
    got, reps = run_batched(h, insts, T, K, beta=beta, prec=prec)
    o = O.nqp_opts(max_inner=20000, eps=0.0, abs_tol=1e-24)
    kw = dict(beta_w=beta, beta_h=beta)
    for inst, (W, Ht), rp in zip(insts, got, reps):
        Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, opts=o, **kw)
        ej = abs(rp.objective - ho[-1]) / ho[-1]
        tw, th = step_bounds(Wo, Ho, inst.r, beta, beta)
        hz = converged_horizon(inst, T, o, kw)
        print(f"{prec} {inst.name}: J {ej:.1e}, W {rel_err(W, Wo):.1e}, H {rel_err(Ht, Ho):.1e}"
              f" (bound {max(tw, th) * hz:.1e})")
        assert ej < 1e-5, inst.name
        # the per-step FP32 bound summed over the horizon, at most 1e-3 (five
        # times the largest error measured on either arithmetic: 1.9e-4 at
        # r = 64, where kappa(Qt) u alone is of order 1e-4)
        tol = max(1e-4, min(max(tw, th) * hz, 1e-3))
        assert rel_err(W, Wo) < tol, inst.name
        assert rel_err(Ht, Ho) < tol, inst.name


@pytest.mark.parametrize("prec", PRECS)
def test_damped_run_stays_on_the_oracle_trajectory(h, prec):
    beta = 10.0
    insts = make_instances(SHAPES[:6], seed=5, beta=beta)
    T, K = 10, 3
    got, reps = run_batched(h, insts, T, K, beta=beta, prec=prec)
    o = O.nqp_opts(max_inner=K, eps=0.0)
    kw = dict(beta_w=beta, beta_h=beta)
    checked = 0
    for inst, (W, Ht), rp in zip(insts, got, reps):
        if oracle_spread(inst, T, o, kw) >= 1e-7:
            print(f"{inst.name}: greedy choices flip under 1e-7 noise, left to the converged run")
            continue
        checked += 1
        Wo, Ho, ho, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, opts=o, **kw)
        assert abs(rp.objective - ho[-1]) / ho[-1] < 1e-5, inst.name
        tw, th = step_bounds(Wo, Ho, inst.r, beta, beta)
        hz = horizon(inst, T, K, **kw)
        assert rel_err(W, Wo) < max(tw, th) * hz, inst.name
        assert rel_err(Ht, Ho) < max(tw, th) * hz, inst.name
    assert checked >= 4


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
    with pytest.raises(P.NmfError):                             # products in BF16
        P.nmf_solve_batched(h, dv, P.solve_opts(1, prec="bf16"))
