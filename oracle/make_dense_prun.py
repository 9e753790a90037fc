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
run, 32 sampled rows of W and of Ht after iterations 1, 5, 20 and 50.  The
GPU parity tests compare their own runs with these values.  Run time: a few
minutes on 8 cores.
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
    for name, opts in (("fixed_k", dict(max_inner=3, eps=0.0)), ("converged", CONVERGED)):
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
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
