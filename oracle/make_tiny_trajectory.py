"""Write tests/golden/tiny200x150_trajectory.json with the FP64 oracle only.

Workload: workloads.tiny(seed=0, r=10) - V = W0 H0 + |N(0, 0.01)|, W0 200 x 10
and H0 10 x 150 with U[0, 1] entries, no penalties, W and H initialised
U[0, 1] - as the FP32 values the GPU reads.

* reference run: 200 outer iterations (4 x the configured 50) with the
  accelerated condition eps = 1e-6; J* = min J over the run;
* plain run: eps = 1e-3 (K_max = 50) for 400 iterations; t_gap = the first
  iteration with J <= J* (1 + 1e-4).

The benchmark's tiny measurement reads J* from here, so its target does not
move with the build.  Run time: seconds.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import workloads as WL  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "tiny200x150_trajectory.json")


def main():
    inst = WL.tiny(seed=0, r=10)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    V, W0, H0 = f32(inst.V), f32(inst.W0), f32(inst.Ht0)
    _, _, ref, _ = O.nmf_solve(W0, H0, 200, V=V, opts=O.nqp_opts(max_inner=50, eps=1e-6))
    jstar = float(ref[1::2].min())
    _, _, plain, _ = O.nmf_solve(W0, H0, 400, V=V, opts=O.nqp_opts(max_inner=50, eps=1e-3))
    plain = plain[1::2]
    hit = np.nonzero(plain <= jstar * (1 + 1e-4))[0]
    out = {"workload": "tiny200x150r10, seed 0, no penalties",
           "definition": "J* = min J over 200 outer iterations at eps 1e-6; t_gap = first outer "
                         "iteration of the eps 1e-3 run with J <= J* (1 + 1e-4)",
           "source": "oracle/make_tiny_trajectory.py (FP64 oracle only)",
           "J_star": jstar, "t_gap": int(hit[0]) + 1 if len(hit) else None,
           "reference_hist": ref[1::2].tolist(), "plain_hist": plain.tolist()}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT, "J*", jstar, "t_gap", out["t_gap"])


if __name__ == "__main__":
    main()
