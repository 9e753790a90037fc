"""Checkpoint and resume of an alternating solve: the factors W and Ht, the
outer iterations done and the options that shape the arithmetic, saved as an
.npz file.  A solve carries no state between outer iterations other than the
factors (with the fast break off, its default), so continuing from a
checkpoint gives, bit for bit, the factors of the uninterrupted run; with
maxstop_mode 1 the fast-break threshold restarts at 0, as at a solve's start.
"""
from __future__ import annotations

import json

import numpy as np

_NNLS = ("max_inner", "eps", "cd_steps", "maxstop_mode", "maxstop", "lanes", "grad_refresh")
_SOLVE = ("alpha_w", "alpha_h", "beta_w", "beta_h", "prec")


def save(path: str, W, Ht, iters_done: int, opts) -> None:
    """Write W (m x r) and Ht (n x r) - tensors on any device - with the
    iteration count and the options of `opts` (a SolveOpts) to `path`."""
    meta = {"iters_done": int(iters_done),
            "solve": {k: getattr(opts, k) for k in _SOLVE},
            "nnls": {k: getattr(opts.nnls, k) for k in _NNLS}}
    np.savez(path, W=W.detach().cpu().numpy(), Ht=Ht.detach().cpu().numpy(),
             meta=np.array(json.dumps(meta)))


def load(path: str, device=None):
    """Read a checkpoint: (W, Ht, iters_done, meta) with W and Ht float32
    tensors on `device` (default: the current CUDA device)."""
    import torch
    with np.load(path) as z:
        meta = json.loads(str(z["meta"]))
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        W = torch.tensor(z["W"], dtype=torch.float32, device=dev)
        Ht = torch.tensor(z["Ht"], dtype=torch.float32, device=dev)
    return W, Ht, meta["iters_done"], meta


def resume_opts(meta, outer_iters: int, **overrides):
    """SolveOpts for `outer_iters` more iterations with the saved options."""
    from paper_1506_08938_gb300 import PREC, nnls_opts, solve_opts
    inv = {v: k for k, v in PREC.items()}
    s = dict(meta["solve"])
    s["prec"] = inv.get(s["prec"], "fp32")
    s.update(overrides)
    return solve_opts(outer_iters, nnls=nnls_opts(**meta["nnls"]), **s)
