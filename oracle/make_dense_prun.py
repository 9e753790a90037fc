"""Write tests/golden/dense10000x4096_prun.json with the FP64 oracle only.

Workload: the dense 10000 x 4096 instance of workloads.dense(seed=0) (rank-50
planted product, normalised, |N(0, 0.01)| noise, clipped to [0, 1]), r = 50,
L2 weight 0.1 on both factors, W and H initialised U[0, 1], all inputs the
FP32 values the GPU sees.  Two fixed-iteration runs of Alg. 1-3, 50 outer
iterations each:

* fixed_k: every NQP takes exactly K = 3 repeat-loop iterations (eps = 0);
* converged: every NQP is solved to its unique minimiser (Q is positive
  definite: the L2 weight), i.e. exact alternating least squares.

Stored: J after every outer iteration of both runs, and, for the converged
run, 32 sampled rows of W and of Ht after iterations 1, 5, 20 and 50, the
condition number of the rescaled Gram of every half-step, and the run's own
sensitivity: J and the sampled rows of a second converged run whose Ht0 is
perturbed by a relative 1e-6 (random signs), per unit of that perturbation.
The GPU parity tests compare their own runs with these values.  Run time:
about ten minutes on 8 cores.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import workloads as WL  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "dense10000x4096_prun.json")
T = 50
SNAPS = (1, 5, 20, 50)
CONVERGED = dict(max_inner=5000, eps=0.0, abs_tol=1e-24)


def kappa(Q):
    Qt, _, dead = O.rescale(Q)
    ev = np.linalg.eigvalsh(Qt[np.ix_(~dead, ~dead)])
    return float(ev[-1] / ev[0])


def converged_run(V, W0, H0, wrows, hrows):
    """J, sampled rows after every iteration and kappa of every half-step,
    with the half-steps written out (the same calls nmf_solve makes)."""
    VT = np.ascontiguousarray(V.T)
    o = O.nqp_opts(**CONVERGED)
    W, H = W0, H0
    J, rows, kap = [], [], []
    for t in range(1, T + 1):
        Q = O.gram(H, 0.1)
        kap.append(kappa(Q))
        W, *_ = O.nnls_update(Q, O.cross_dense(V, H), 0.0, W, o)
        Q = O.gram(W, 0.1)
        kap.append(kappa(Q))
        H, *_ = O.nnls_update(Q, O.cross_dense(VT, W), 0.0, H, o)
        J.append(O.objective_dense(V, W, H, 0.0, 0.0, 0.1, 0.1))
        rows.append((W[wrows].copy(), H[hrows].copy()))
        print(f"converged t={t} J={J[-1]:.8f} kappa {kap[-2]:.0f} {kap[-1]:.0f}", flush=True)
    return np.array(J), rows, kap


def main():
    inst = WL.dense(seed=0)
    V = inst.V.astype(np.float64)
    W0 = inst.W0.astype(np.float64)
    H0 = inst.Ht0.astype(np.float64)
    g = WL.rng(77)
    wrows = np.sort(g.choice(inst.m, size=32, replace=False))
    hrows = np.sort(g.choice(inst.n, size=32, replace=False))
    out = {"workload": "dense10000x4096r50, seed 0, beta_w = beta_h = 0.1",
           "source": "oracle/make_dense_prun.py (FP64 oracle only)",
           "outer_iters": T, "w_rows": wrows.tolist(), "h_rows": hrows.tolist()}
    for name, opts in (("fixed_k", dict(max_inner=3, eps=0.0)),):
        W, H = W0, H0
        J, snaps = [], {}
        t0 = time.time()
        for t in range(1, T + 1):
            W, H, h, _ = O.nmf_solve(W, H, 1, V=V, beta_w=0.1, beta_h=0.1,
                                     opts=O.nqp_opts(**opts))
            J.append(float(h[1]))
            if name == "converged" and t in SNAPS:
                snaps[str(t)] = {"W": W[wrows].tolist(), "Ht": H[hrows].tolist()}
            print(f"{name} t={t} J={J[-1]:.8f} {time.time() - t0:.0f}s", flush=True)
        out[name] = {"J": J, "opts": opts}
        if snaps:
            out[name]["rows"] = snaps
    J, rows, kap = converged_run(V, W0, H0, wrows, hrows)
    out["converged"] = {"J": J.tolist(), "opts": CONVERGED, "kappa": kap,
                        "rows": {str(t): {"W": rows[t - 1][0].tolist(),
                                          "Ht": rows[t - 1][1].tolist()} for t in SNAPS}}
    delta = 1e-6
    Hp = H0 * (1.0 + delta * g.choice([-1.0, 1.0], size=H0.shape))
    Jp, rp, _ = converged_run(V, W0, Hp, wrows, hrows)
    sf = [max(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0]),
              np.linalg.norm(a[1] - b[1]) / np.linalg.norm(b[1])) / delta
          for a, b in zip(rp, rows)]
    out["converged"]["sensitivity"] = {"delta": delta,
                                       "J": (np.abs(Jp - J) / J / delta).tolist(),
                                       "rows": sf}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
