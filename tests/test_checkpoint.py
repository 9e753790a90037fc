"""Checkpoint files on the host: what is saved comes back unchanged."""
import numpy as np
import torch

import paper_1506_08938_gb300 as P
from paper_1506_08938_gb300 import checkpoint as CP


def test_checkpoint_round_trip(tmp_path):
    g = torch.Generator().manual_seed(3)
    W = torch.rand(37, 6, generator=g)
    Ht = torch.rand(23, 6, generator=g)
    o = P.solve_opts(7, alpha_w=0.25, beta_h=0.125, prec="bf16",
                     nnls=P.nnls_opts(max_inner=11, eps=1e-4, maxstop_mode=1, grad_refresh=5))
    path = str(tmp_path / "c.npz")
    CP.save(path, W, Ht, 7, o)
    W2, H2, done, meta = CP.load(path, device="cpu")
    assert done == 7
    assert torch.equal(W2, W) and torch.equal(H2, Ht)
    r = CP.resume_opts(meta, 3)
    assert r.outer_iters == 3 and r.prec == P.PREC["bf16"]
    assert (r.alpha_w, r.alpha_h, r.beta_w, r.beta_h) == (0.25, 0.0, 0.0, 0.125)
    for k in ("max_inner", "eps", "cd_steps", "maxstop_mode", "maxstop", "lanes", "grad_refresh"):
        assert getattr(r.nnls, k) == getattr(o.nnls, k)
    assert np.isclose(r.nnls.eps, 1e-4)
