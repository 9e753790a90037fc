"""nmf_gram_noalloc: the Gram matrix with no device allocation in the library.

For callers that cannot call cudaMalloc (an allocator that must own every
device byte, a fixed memory budget reserved up front, code that may not take
the allocation path): their split-K partial sums go to a fixed device array
inside the library.  Checked through the C ABI against nmf_gram (within the
FP32 rounding of a different split of the sums), two calls in a row (the
second smaller, so stale contents from the first would show), plus the edge
cases: no rows (Q = beta I), a padded row pitch, a row count whose split
leaves trailing partial slices unwritten (they must be cleared), and one case
element by element against an FP64 Gram computed on the host.  This file
sorts last so a stop-at-first-failure run has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call(L, P, X, beta, Q, stream):
    d = P.dense(X)
    return L.nmf_gram_noalloc(C.byref(d), C.c_float(beta), C.c_void_p(Q.data_ptr()),
                              C.c_void_p(stream.cuda_stream))


def test_gram_noalloc_matches_gram_twice():
    import __graft_entry__ as g
    g.build()
    import paper_1506_08938_gb300 as P
    L = P.lib()
    dev = torch.device("cuda:0")
    h = P.Handle(0)
    stream = torch.cuda.current_stream(dev)
    for rows, r, beta in ((20001, 100, 0.25), (777, 37, 0.0)):
        X = torch.tensor(WL.rng(rows + r).random((rows, r)), dtype=torch.float32, device=dev)
        Qref = P.nmf_gram(h, X, beta=beta)
        Q = torch.full((r, r), float("nan"), dtype=torch.float32, device=dev)
        assert _call(L, P, X, beta, Q, stream) == P.NMF_OK
        torch.cuda.synchronize()
        a = Q.double().cpu().numpy()
        b = Qref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-6
    # sizes beyond the array's maximum are refused before any launch
    X = torch.zeros(10, 129, dtype=torch.float32, device=dev)
    Q = torch.zeros(129, 129, dtype=torch.float32, device=dev)
    assert _call(L, P, X, 0.0, Q, stream) == P.NMF_E_SHAPE
    # host memory is refused: the kernels run on the current device
    Xh = torch.zeros(10, 8, dtype=torch.float32)
    Qd = torch.zeros(8, 8, dtype=torch.float32, device=dev)
    assert _call(L, P, Xh, 0.0, Qd, stream) == P.NMF_E_ARG
    h.close()


def test_gram_noalloc_edge_cases():
    import paper_1506_08938_gb300 as P
    L = P.lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    # no rows: every slice is cleared and Q = beta I exactly
    X = torch.empty(0, 16, dtype=torch.float32, device=dev)
    Q = torch.full((16, 16), float("nan"), dtype=torch.float32, device=dev)
    assert _call(L, P, X, 0.5, Q, stream) == P.NMF_OK
    torch.cuda.synchronize()
    assert np.array_equal(Q.cpu().numpy(), 0.5 * np.eye(16, dtype=np.float32))
    # 4033 rows: 63 slices of 96-row chunks are requested but 43 CTAs cover
    # the rows, so the trailing 20 slices must be cleared; a padded row pitch
    # (a 24-wide view of 40-wide rows); FP64 host reference element by element
    base = torch.tensor(WL.rng(4033).random((4033, 40)), dtype=torch.float32, device=dev)
    X = base[:, :24]
    assert X.stride(0) == 40
    Q = torch.full((24, 24), float("nan"), dtype=torch.float32, device=dev)
    assert _call(L, P, X, 0.125, Q, stream) == P.NMF_OK
    torch.cuda.synchronize()
    Xd = X.double().cpu().numpy()
    ref = Xd.T @ Xd + 0.125 * np.eye(24)
    err = np.abs(Q.double().cpu().numpy() - ref)
    assert np.all(err <= 2e-6 * ref)
