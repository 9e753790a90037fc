"""tcgen05 tensor-core cross term C = A B (through nmf_cross) against the FP64
oracle.  Shapes cover partial row tiles, K not a multiple of the 32-wide k
block, every padded width (r -> 16, 32, 64, 128) and stream-K splits where a
row tile is shared by several CTAs.

Bounds, element by element against |A||B| (= A B here: the inputs are
nonnegative): FP32 (3xTF32 split with the TMEM accumulator drained into FP32
registers every k block, the small terms in columns of their own; measured
1.2e-7 norm-wise at K = 10000) 2e-6; TF32 truncates both operands to a 10-bit
mantissa, so each product is off by less than 2^-9 of itself: 2^-9 + 2e-6;
BF16 with A already BF16 (the oracle sees the same A) and B rounded to
nearest BF16 inside the kernel (8 significant bits: off by at most 2^-8 of
itself), each product off by at most 2^-8 of itself: 2^-8 + 2e-6; BF16X2
with the same A and B split into hi = rn(B) and lo = rn(B - hi), so that
|B - hi - lo| <= 2^-8 |B - hi| <= 2^-16 |B| (BF16 products are exact in the
FP32 accumulator): 2^-16 + 2e-6.  These are worst-case bounds, not fits.
"""
import numpy as np
import pytest

import oracle as O
import workloads as WL
from tests.gpu_common import dev, elementwise_ok, rel_err, t32, to_np, torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1506_08938_gb300")


@pytest.fixture(scope="module")
def h():
    import __graft_entry__ as g
    g.build()
    hh = P.Handle(0)
    yield hh
    hh.close()


SHAPES = [(1, 32), (127, 64), (129, 96), (1000, 3008), (300, 20000), (4096, 10000)]


@pytest.mark.parametrize("M,K", SHAPES)
@pytest.mark.parametrize("r", [4, 16, 50, 64, 100, 128])
def test_tc_cross_fp32_split(h, M, K, r):
    g = WL.rng(M * 7 + K + r)
    A = g.random((M, K)).astype(np.float32)
    B = g.random((K, r)).astype(np.float32)
    Co = O.cross_dense(A.astype(np.float64), B.astype(np.float64))
    Cg = P.nmf_cross(h, t32(A), t32(B), prec="fp32")
    h.sync()
    err = rel_err(to_np(Cg), Co)
    bias = float(np.mean((to_np(Cg) - Co) / Co))
    worst = elementwise_ok(to_np(Cg), Co, Co, 2e-6)
    print(f"tc fp32 M={M} K={K} r={r}: rel {err:.3e} bias {bias:.3e} worst {worst:.3f} x bound")


@pytest.mark.parametrize("M,K", [(129, 96), (1000, 3008), (4096, 10000)])
@pytest.mark.parametrize("r", [16, 50, 128])
def test_tc_cross_tf32(h, M, K, r):
    g = WL.rng(M + K + r + 1)
    A = g.random((M, K)).astype(np.float32)
    B = g.random((K, r)).astype(np.float32)
    Co = O.cross_dense(A.astype(np.float64), B.astype(np.float64))
    Cg = P.nmf_cross(h, t32(A), t32(B), prec="tf32")
    h.sync()
    err = rel_err(to_np(Cg), Co)
    worst = elementwise_ok(to_np(Cg), Co, Co, 2.0 ** -9 + 2e-6)
    print(f"tc tf32 M={M} K={K} r={r}: rel {err:.3e} worst {worst:.3f} x bound")


BF16_BOUND = {"bf16": 2.0 ** -8 + 2e-6, "bf16x2": 2.0 ** -16 + 2e-6}


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
@pytest.mark.parametrize("M,K", [(1, 64), (129, 96), (1000, 3008), (300, 20000), (4096, 10000)])
@pytest.mark.parametrize("r", [4, 16, 50, 128])
def test_tc_cross_bf16(h, M, K, r, prec):
    g = WL.rng(M + K + r + 2)
    A = g.random((M, K)).astype(np.float32)
    B = g.random((K, r)).astype(np.float32)
    Ab = torch.tensor(A, device=dev()).to(torch.bfloat16)
    # the oracle sees the BF16-rounded A; B is rounded (split) inside the kernel
    Co = O.cross_dense(Ab.float().cpu().numpy().astype(np.float64), B.astype(np.float64))
    Cg = P.nmf_cross(h, Ab, t32(B), prec=prec)
    h.sync()
    err = rel_err(to_np(Cg), Co)
    worst = elementwise_ok(to_np(Cg), Co, Co, BF16_BOUND[prec])
    print(f"tc {prec} M={M} K={K} r={r}: rel {err:.3e} worst {worst:.3f} x bound")


def test_tc_cross_unaligned_falls_back(h):
    g = WL.rng(5)
    A = g.random((300, 3005)).astype(np.float32)    # row pitch not a multiple of 16 B
    B = g.random((3005, 50)).astype(np.float32)
    Co = O.cross_dense(A.astype(np.float64), B.astype(np.float64))
    Cg = P.nmf_cross(h, t32(A), t32(B), prec="fp32")
    h.sync()
    elementwise_ok(to_np(Cg), Co, Co, 2e-6)
    with pytest.raises(P.NmfError):
        P.nmf_cross(h, t32(A), t32(B), prec="tf32")


def test_tc_and_simt_solves_agree(h):
    """The dense solve with tensor-core FP32 and with CUDA-core FP32 cross
    terms: both are FP32-accurate, so the first iterations agree to the FP32
    per-step bound."""
    import ctypes as C
    inst = WL.tiny(seed=0, r=10)
    V = t32(inst.V)
    out = []
    for prec in ("fp32", "fp32_simt"):
        W = t32(inst.W0)
        Ht = t32(inst.Ht0)
        hist = np.zeros(3)
        o = P.solve_opts(3, prec=prec, nnls=P.nnls_opts(max_inner=3, eps=0.0), objective="direct",
                         obj_hist=hist.ctypes.data_as(C.POINTER(C.c_double)))
        P.nmf_solve(h, V, W, Ht, o)
        out.append((to_np(W), to_np(Ht), hist.copy()))
    assert np.abs(out[0][2] - out[1][2]).max() / out[1][2].max() < 1e-4


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x2"])
def test_reduced_precision_solves_track_fp32(h, prec):
    """Solve with TF32 / BF16 cross terms (FP32 accumulation; Grams and NNLS
    in FP32) against the FP32 solve from the same start, on the non-chaotic
    instance (L2 weight 10).  Stated bound: the products carry relative
    errors up to 6.5e-4 (TF32) and 2e-4 (BF16, measured above); the
    objectives over 20 iterations agree to 2e-3.  Each half-step minimises
    the problem with the perturbed cross term, so the true objective
    decreases only up to that perturbation: a rise between iterations stays
    within the same 2e-3 of J, and the run ends below its start."""
    import ctypes as C
    inst = WL.tiny(seed=0, r=10, m=200, n=152)     # n multiple of 8 for BF16 rows
    Vd = t32(inst.V)
    out = {}
    for p_ in ("fp32", prec):
        W = t32(inst.W0)
        Ht = t32(inst.Ht0)
        hist = np.zeros(20)
        o = P.solve_opts(20, beta_w=10.0, beta_h=10.0, prec=p_, objective="direct",
                         nnls=P.nnls_opts(max_inner=3, eps=0.0),
                         obj_hist=hist.ctypes.data_as(C.POINTER(C.c_double)))
        P.nmf_solve(h, Vd, W, Ht, o)
        out[p_] = hist.copy()
    rel = np.abs(out[prec] - out["fp32"]) / out["fp32"]
    print(f"{prec} vs fp32 max rel J {rel.max():.3e}")
    assert rel.max() < 2e-3, rel
    assert np.all(np.diff(out[prec]) <= 2e-3 * out[prec][1:])
    assert out[prec][-1] < out[prec][0]
