"""Write tests/golden/dense10000x4096_trajectory.json with the FP64 oracle only.

Workload: the dense 10000 x 4096 instance (rank-50 planted product,
normalised, |N(0, 0.01)| noise, clipped to [0, 1]; seed 0), r = 50, L2 weight
0.1 on both factors, W and H initialised U[0, 1].

* reference run: 800 outer iterations (4 x the configured 200) with
  accelerated condition eps = 1e-6; J* = min J over the run.
* plain run: eps = 1e-3 (K_max = 50) until J <= J* (1 + 1e-4) or 1600
  iterations; t_gap = the first such iteration (1-based count of outer
  iterations).

The benchmark's CPU-baseline leg multiplies the oracle's measured time per
outer iteration by t_gap; the GPU tests compare the first iterations of the
GPU trajectory with these values.  Run time: about 1-2 hours on 8 cores.
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

OUT = os.path.join(ROOT, "tests", "golden", "dense10000x4096_trajectory.json")


def run(inst, W, H, iters, eps, chunk=25, stop_at=None):
    hist = []
    t0 = time.time()
    while len(hist) < iters:
        k = min(chunk, iters - len(hist))
        W, H, h, _ = O.nmf_solve(W, H, k, V=inst.V, beta_w=0.1, beta_h=0.1,
                                 opts=O.nqp_opts(max_inner=50, eps=eps))
        hist.extend(h[1::2].tolist())
        print(f"eps={eps:g} t={len(hist)} J={hist[-1]:.6f} {time.time() - t0:.0f}s", flush=True)
        if stop_at is not None and min(hist) <= stop_at:
            break
    return W, H, hist


def main():
    inst = WL.dense(seed=0)
    inst.V = inst.V.astype(np.float64)
    W0 = inst.W0.astype(np.float64)
    H0 = inst.Ht0.astype(np.float64)
    _, _, ref = run(inst, W0, H0, 800, 1e-6)
    jstar = float(min(ref))
    target = jstar * (1 + 1e-4)
    _, _, plain = run(inst, W0, H0, 1600, 1e-3, stop_at=target)
    hit = [i for i, j in enumerate(plain) if j <= target]
    out = {
        "workload": "dense10000x4096r50, seed 0, beta_w = beta_h = 0.1",
        "definition": "J* = min J over 800 outer iterations at eps 1e-6; t_gap = first outer "
                      "iteration of the eps 1e-3 run with J <= J* (1 + 1e-4)",
        "source": "oracle/make_dense_trajectory.py (FP64 oracle only)",
        "J_star": jstar,
        "t_gap": (hit[0] + 1) if hit else None,
        "reference_hist": ref,
        "plain_hist": plain,
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT, "t_gap", out["t_gap"], "J*", jstar)


if __name__ == "__main__":
    main()
