"""Row-sharded outer iteration of Alg. 2 across P processes.

The independent row problems of §3.2-3.3 shard by rows of V: rank p holds
the row block V_p (m_p x n) and the matching rows W_p of W; Ht (n x r) is
replicated.  One outer iteration:

* W-update, local: Q_W = Ht^T Ht + b_w I from the replicated Ht,
  C_W = V_p Ht, every row of W_p by Alg. 3.
* H-update: the only exchange.  G_W = sum_p W_p^T W_p (r x r) and
  C_H = sum_p V_p^T W_p (n x r) - the Reduce of Fig. 1 (F_i F_i^T and
  F_i V_i^T summed over the map outputs) - travel in one all-reduce of
  r (r + n) floats; every rank then solves all n rows of Ht from identical
  inputs, so Ht stays replicated without a second collective.

The arithmetic is injected through `ops` (GPU kernels through the C ABI by
default, see GpuOps), the exchange through torch.distributed.  On a box
with one GPU the benchmark runs replicas; this schedule is what several
GPUs of one node would run.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class ShardOpts:
    alpha_w: float = 0.0
    alpha_h: float = 0.0
    beta_w: float = 0.0
    beta_h: float = 0.0


class GpuOps:
    """The four steps on device tensors through the C ABI (FP32)."""

    def __init__(self, handle, nnls_opts=None):
        import paper_1506_08938_gb300 as P
        self.P = P
        self.h = handle
        self.nnls_opts = nnls_opts

    def gram(self, X, beta):
        return self.P.nmf_gram(self.h, X, beta=beta)

    def cross(self, A, B):
        return self.P.nmf_cross(self.h, A, B)

    def nnls(self, Q, C, alpha, X0):
        Qt, d = self.P.nmf_rescale(self.h, Q)
        self.P.nmf_nnls_update(self.h, Qt, d, C, X0, alpha=alpha, opts=self.nnls_opts)
        self.h.sync()
        return X0


def sharded_iteration(Vp, Vpt, Wp, Ht, ops, opts: ShardOpts, group=None):
    """One outer iteration on this rank's shard.  Vp (m_p x n) and its
    transpose Vpt, Wp (m_p x r) and the replicated Ht (n x r) are tensors of
    one device; returns the updated (Wp, Ht)."""
    import torch
    import torch.distributed as dist

    r = Ht.shape[1]
    n = Ht.shape[0]
    # W-update: local
    Qw = ops.gram(Ht, opts.beta_w)
    Cw = ops.cross(Vp, Ht)
    Wp = ops.nnls(Qw, Cw, opts.alpha_w, Wp)
    # H-update: this rank's contributions, summed over ranks in one collective.
    # The L2 term enters once, through the first rank's Gram (the library's
    # Q = X^T X + beta I), so the sum is Q_H = sum_p W_p^T W_p + b_h I.
    dist_on = dist.is_available() and dist.is_initialized()
    first = (dist.get_rank(group) if dist_on else 0) == 0
    Gp = ops.gram(Wp, opts.beta_h if first else 0.0)
    Chp = ops.cross(Vpt, Wp)
    buf = torch.cat([Gp.reshape(-1), Chp.reshape(-1)])
    if dist_on:
        dist.all_reduce(buf, group=group)
    Qh = buf[: r * r].reshape(r, r)
    Ch = buf[r * r:].reshape(n, r)
    Ht = ops.nnls(Qh, Ch, opts.alpha_h, Ht)
    return Wp, Ht


def row_block(m: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [lo, hi) of rank `rank` when m rows are cut into `world` blocks
    whose sizes differ by at most one."""
    base, extra = divmod(m, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)
