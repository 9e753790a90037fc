"""nmf_gram_noalloc: the Gram matrix with no device allocation in the library.

For callers that cannot call cudaMalloc (an allocator that must own every
device byte, a fixed memory budget reserved up front, code that may not take
the allocation path): their split-K partial sums go to a fixed device array
inside the library.  Checked through the C ABI against nmf_gram, two calls in
a row (the second smaller, so stale contents from the first would show).
This file sorts last so a stop-at-first-failure run has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
        d = P.dense(X)
        st = L.nmf_gram_noalloc(C.byref(d), C.c_float(beta), C.c_void_p(Q.data_ptr()),
                                C.c_void_p(stream.cuda_stream))
        assert st == P.NMF_OK
        torch.cuda.synchronize()
        a = Q.double().cpu().numpy()
        b = Qref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-6
    # sizes beyond the array's maximum are refused before any launch
    X = torch.zeros(10, 129, dtype=torch.float32, device=dev)
    Q = torch.zeros(129, 129, dtype=torch.float32, device=dev)
    d = P.dense(X)
    assert L.nmf_gram_noalloc(C.byref(d), C.c_float(0.0), C.c_void_p(Q.data_ptr()),
                              C.c_void_p(stream.cuda_stream)) == P.NMF_E_SHAPE
    h.close()
