"""Row-sharded outer iteration (the multi-GPU schedule) on two and three gloo ranks on
the CPU, with the FP64 oracle supplying the arithmetic: the concatenated
W blocks and the replicated Ht must equal the unsharded oracle run up to
summation order (the exchanged Gram and cross term are sums of per-rank
partial sums instead of one), and every rank must hold the same Ht bit for
bit."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

import oracle as O  # noqa: E402
import workloads as WL  # noqa: E402
from paper_1506_08938_gb300.sharded import ShardOpts, row_block, sharded_iteration  # noqa: E402

T, K, BETA = 8, 3, 10.0


class OracleOps:
    """The four steps of the schedule by the oracle, on CPU float64 tensors."""

    def __init__(self):
        self.o = O.nqp_opts(max_inner=K, eps=0.0)

    def gram(self, X, beta):
        return torch.from_numpy(O.gram(X.numpy(), beta))

    def cross(self, A, B):
        return torch.from_numpy(O.cross_dense(A.numpy(), B.numpy()))

    def nnls(self, Q, C, alpha, X0):
        X, *_ = O.nnls_update(Q.numpy(), C.numpy(), alpha, X0.numpy(), self.o)
        return torch.from_numpy(X)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def instance():
    inst = WL.tiny(seed=4, r=6, m=61, n=37)
    return inst


def worker(rank, world, port, outdir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    inst = instance()
    lo, hi = row_block(inst.m, world, rank)
    Vp = torch.from_numpy(np.ascontiguousarray(inst.V[lo:hi]))
    Vpt = Vp.t().contiguous()
    Wp = torch.from_numpy(np.ascontiguousarray(inst.W0[lo:hi]))
    Ht = torch.from_numpy(np.ascontiguousarray(inst.Ht0))
    ops = OracleOps()
    so = ShardOpts(beta_w=BETA, beta_h=BETA)
    for _ in range(T):
        Wp, Ht = sharded_iteration(Vp, Vpt, Wp, Ht, ops, so)
    np.save(os.path.join(outdir, f"W{rank}.npy"), Wp.numpy())
    np.save(os.path.join(outdir, f"H{rank}.npy"), Ht.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_row_block_partition():
    for m in (1, 7, 61, 1000):
        for world in (1, 2, 3, 8):
            blocks = [row_block(m, world, p) for p in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == m
            assert all(blocks[p][1] == blocks[p + 1][0] for p in range(world - 1))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_match_unsharded_oracle(world):
    # 61 rows over 3 ranks: uneven blocks (21, 20, 20)
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(worker, args=(world, free_port(), d), nprocs=world, join=True)
        Ws = [np.load(os.path.join(d, f"W{p}.npy")) for p in range(world)]
        Hs = [np.load(os.path.join(d, f"H{p}.npy")) for p in range(world)]
    for p in range(1, world):
        assert np.array_equal(Hs[0], Hs[p])
    inst = instance()
    Wo, Ho, _, _ = O.nmf_solve(inst.W0, inst.Ht0, T, V=inst.V, beta_w=BETA, beta_h=BETA,
                               opts=O.nqp_opts(max_inner=K, eps=0.0))
    W = np.concatenate(Ws)
    assert np.abs(W - Wo).max() <= 1e-9 * np.abs(Wo).max()
    assert np.abs(Hs[0] - Ho).max() <= 1e-9 * np.abs(Ho).max()
