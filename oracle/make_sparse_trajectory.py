"""Write tests/golden/sparse100000x50000_trajectory.json with the FP64 oracle.

Workload: workloads.sparse(seed=0) - CSR V 100000 x 50000, Poisson(50)
distinct columns per row drawn with Zipf(1.1) popularity, values
Poisson(2) + 1 (exact in BF16) - r = 100, L1 weight 0.01 on H, W and H
initialised U[0, 1] (the FP32 values the GPU reads).  20 outer iterations of
the plain method (eps = 1e-3, K_max = 50); J after each.

A 4 x 100-iteration reference run of the oracle would take hours on the host,
so the benchmark's sparse line times the GPU to the objective this run
reaches after its 20 iterations (within 1e-4): a target fixed by the oracle.
Run time: about 15 minutes on 8 cores.
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

OUT = os.path.join(ROOT, "tests", "golden", "sparse100000x50000_trajectory.json")
T = 20


def main():
    sp = WL.sparse(seed=0)
    W = sp.W0.astype(np.float32).astype(np.float64)
    H = sp.Ht0.astype(np.float32).astype(np.float64)
    csr = (sp.rowptr, sp.colidx, sp.vals.astype(np.float64))
    csr_t = (sp.t_rowptr, sp.t_colidx, sp.t_vals.astype(np.float64))
    J, inner = [], 0
    t0 = time.time()
    for t in range(T):
        W, H, h, tot = O.nmf_solve(W, H, 1, csr=csr, csr_t=csr_t, alpha_h=sp.alpha_h,
                                   opts=O.nqp_opts(max_inner=50, eps=1e-3))
        J.append(float(h[1]))
        inner += tot
        print(f"t={t + 1} J={J[-1]:.4f} {time.time() - t0:.0f}s", flush=True)
    out = {"workload": "sparse100000x50000r100, seed 0, alpha_h = 0.01",
           "source": "oracle/make_sparse_trajectory.py (FP64 oracle only)",
           "definition": "J after each of 20 outer iterations at eps 1e-3 (K_max 50)",
           "plain_hist": J, "J_target": J[-1], "t_target": T,
           "kbar": inner / (T * (sp.m + sp.n))}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
