"""Python binding of libnmf.so (the C ABI declared in include/nmf.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  If the library is
missing or cannot be loaded, every call raises - there is no fallback.

Names follow the C ABI: ``nmf_gram``, ``nmf_cross``, ``nmf_rescale``,
``nmf_nnls_update``, ``nmf_solve``, ``nmf_project``, ``nmf_objective``,
``nmf_kkt``; ``Handle`` wraps ``nmf_create``/``nmf_destroy``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnmf.so")

# status codes (nmf_status)
NMF_OK, NMF_E_ARG, NMF_E_SHAPE, NMF_E_DTYPE, NMF_E_NOMEM, NMF_E_CUDA = 0, 1, 2, 3, 4, 5
NMF_E_NONFINITE, NMF_E_TIMEOUT, NMF_E_BUSY, NMF_E_NOTIMPL = 6, 7, 8, 9
# dtypes / precisions
NMF_F32, NMF_BF16, NMF_F64 = 0, 1, 2
PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x2": 3, "fp32_simt": 4}


class NmfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class Dense(C.Structure):
    _fields_ = [("rows", C.c_int64), ("cols", C.c_int64), ("ld", C.c_int64), ("dt", C.c_int),
                ("data", C.c_void_p)]


class Csr(C.Structure):
    _fields_ = [("rows", C.c_int64), ("cols", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("vals", C.c_void_p),
                ("dt", C.c_int)]


class Matrix(C.Structure):
    _fields_ = [("is_sparse", C.c_int), ("d", Dense), ("s", Csr)]


class NnlsOpts(C.Structure):
    _fields_ = [("max_inner", C.c_int), ("eps", C.c_double), ("cd_steps", C.c_int),
                ("maxstop_mode", C.c_int), ("maxstop", C.c_float), ("lanes", C.c_int),
                ("grad_refresh", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("rel_gap_target", C.c_double), ("f_star", C.c_double),
                ("alpha_w", C.c_float), ("alpha_h", C.c_float), ("beta_w", C.c_float),
                ("beta_h", C.c_float), ("prec", C.c_int), ("nnls", NnlsOpts),
                ("check_every", C.c_int), ("use_graph", C.c_int), ("objective", C.c_int),
                ("obj_hist", C.POINTER(C.c_double))]


class Report(C.Structure):
    _fields_ = [("iters_done", C.c_int), ("objective", C.c_double), ("rel_gap", C.c_double),
                ("kbar", C.c_double), ("kkt_max", C.c_double), ("ms_total", C.c_double),
                ("inner_total", C.c_int64)]


class Instance(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("r", C.c_int), ("V", C.c_void_p),
                ("Vt", C.c_void_p), ("W", C.c_void_p), ("Ht", C.c_void_p)]


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int), ("max_batch_cols", C.c_int64), ("max_batch_nnz", C.c_int64),
                ("hbm_budget", C.c_size_t), ("nnls", NnlsOpts)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("completed_cols", C.c_int64), ("batches", C.c_int64),
                ("queued", C.c_int64), ("max_queue", C.c_int64), ("inflight_bytes", C.c_int64)]


_lib = None
_lock = threading.Lock()
_P = C.c_void_p


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    L.nmf_status_string.restype = C.c_char_p
    L.nmf_status_string.argtypes = [C.c_int]
    L.nmf_create.argtypes = [C.POINTER(_P), C.c_int, _P]
    L.nmf_destroy.argtypes = [_P]
    L.nmf_set_stream.argtypes = [_P, _P]
    L.nmf_sync.argtypes = [_P]
    L.nmf_nnls_opts_default.argtypes = [C.POINTER(NnlsOpts)]
    L.nmf_nnls_opts_default.restype = None
    L.nmf_launch_count.restype = C.c_int64
    L.nmf_gram.argtypes = [_P, C.POINTER(Dense), C.c_float, C.c_int, _P]
    L.nmf_cross.argtypes = [_P, C.POINTER(Matrix), _P, C.c_int, C.c_int, _P]
    L.nmf_rescale.argtypes = [_P, _P, C.c_int, _P, _P]
    L.nmf_nnls_update.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_int, C.c_float, _P,
                                  C.POINTER(NnlsOpts), _P]
    L.nmf_objective.argtypes = [_P, C.c_double, _P, C.c_int64, _P, C.c_int64, C.c_int, _P, _P,
                                _P, C.c_float, C.c_float, C.c_float, C.c_float, _P]
    L.nmf_kkt.argtypes = [_P, _P, _P, C.c_int64, C.c_int, C.c_float, _P, _P]
    L.nmf_objective_direct.argtypes = [_P, C.POINTER(Dense), _P, _P, C.c_int, C.c_float,
                                       C.c_float, C.c_float, C.c_float, _P]
    L.nmf_peak_tc_bf16.argtypes = [_P, C.POINTER(C.c_double)]
    L.nmf_solve.argtypes = [_P, C.POINTER(Matrix), C.POINTER(Matrix), C.c_int, _P, _P,
                            C.POINTER(SolveOpts), C.POINTER(Report)]
    L.nmf_solve_streamed.argtypes = [_P, C.POINTER(Dense), C.c_int, _P, _P,
                                     C.POINTER(SolveOpts), C.c_int64, C.POINTER(Report)]
    L.nmf_solve_batched.argtypes = [_P, C.c_int, C.POINTER(Instance), C.POINTER(SolveOpts),
                                    C.c_int, C.POINTER(Report)]
    L.nmf_project.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_int, C.POINTER(Csr), _P,
                              C.POINTER(NnlsOpts)]
    L.nmf_gram_noalloc.argtypes = [C.POINTER(Dense), C.c_float, _P, _P]
    L.nmf_server_create.argtypes = [C.POINTER(_P), C.c_int, _P, C.c_int64, C.c_int,
                                    C.POINTER(ServerOpts)]
    L.nmf_server_submit.argtypes = [_P, C.c_int64, C.c_int64, _P, _P, _P, _P,
                                    C.POINTER(C.c_int64)]
    L.nmf_server_wait.argtypes = [_P, C.c_int64, C.c_double, C.POINTER(C.c_double)]
    L.nmf_server_stats.argtypes = [_P, C.POINTER(ServerStats)]
    L.nmf_server_destroy.argtypes = [_P]
    L.nmf_peak_fp32.argtypes = [C.POINTER(C.c_double)]
    L.nmf_peak_l2_gather.argtypes = [C.c_int, C.POINTER(C.c_double)]
    L.nmf_fault_armed.argtypes = [C.c_char_p]
    L.nmf_fault_armed.restype = C.c_int
    L.nmf_profile_enable.argtypes = [C.c_int]
    L.nmf_profile_read.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    return L


KCLASS = {"gram": 0, "cross": 1, "spmm": 2, "rescale": 3, "nnls": 4, "objective": 5, "other": 6}


def nmf_peak_tc_bf16(h: "Handle") -> float:
    """Dense BF16 TFLOP/s of the library's tcgen05.mma path on an r = 512
    contraction from shared memory (the tensor-pipe roofline)."""
    t = C.c_double()
    _check(lib().nmf_peak_tc_bf16(h.h, C.byref(t)), "nmf_peak_tc_bf16")
    return t.value


def nmf_peak_fp32() -> float:
    """Measured FP32 FFMA throughput of the current device, TFLOP/s."""
    v = C.c_double(0.0)
    _check(lib().nmf_peak_fp32(C.byref(v)), "nmf_peak_fp32")
    return v.value


def nmf_peak_l2_gather(r: int) -> float:
    """Measured L2-resident gather bandwidth for rows of r floats, GB/s."""
    v = C.c_double(0.0)
    _check(lib().nmf_peak_l2_gather(int(r), C.byref(v)), "nmf_peak_l2_gather")
    return v.value


def nmf_profile_enable(enable: bool = True):
    _check(lib().nmf_profile_enable(int(bool(enable))), "nmf_profile_enable")


def nmf_profile_read(kclass: str):
    """(device ms, launches) of one kernel class since profiling was enabled."""
    ms = C.c_double()
    n = C.c_int64()
    _check(lib().nmf_profile_read(KCLASS[kclass], C.byref(ms), C.byref(n)), "nmf_profile_read")
    return ms.value, n.value


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load()
    return _lib


def status_string(s: int) -> str:
    return lib().nmf_status_string(int(s)).decode()


def _check(st: int, where: str):
    if st != NMF_OK:
        raise NmfError(st, where)


def launch_count() -> int:
    return int(lib().nmf_launch_count())


# ---------------------------------------------------------------- helpers
def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dt(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return NMF_F32
    if t.dtype == torch.bfloat16:
        return NMF_BF16
    if t.dtype == torch.float64:
        return NMF_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensor must live on the GPU")


def dense(t) -> Dense:
    """Describe a row-major 2-D tensor (stride(1) must be 1)."""
    assert t.dim() == 2 and (t.stride(1) == 1 or t.shape[1] <= 1)
    return Dense(t.shape[0], t.shape[1], t.stride(0) if t.shape[0] > 1 else t.shape[1], _dt(t),
                 t.data_ptr())


def csr(rowptr, colidx, vals, ncols: int) -> Csr:
    return Csr(rowptr.numel() - 1, int(ncols), vals.numel(), rowptr.data_ptr(), colidx.data_ptr(),
               vals.data_ptr(), _dt(vals))


def matrix_dense(t) -> Matrix:
    m = Matrix()
    m.is_sparse = 0
    m.d = dense(t)
    return m


def matrix_csr(rowptr, colidx, vals, ncols: int) -> Matrix:
    m = Matrix()
    m.is_sparse = 1
    m.s = csr(rowptr, colidx, vals, ncols)
    return m


def nnls_opts(max_inner=50, eps=1e-3, cd_steps=-1, maxstop_mode=0, maxstop=0.0,
              lanes=0, grad_refresh=0) -> NnlsOpts:
    return NnlsOpts(int(max_inner), float(eps), int(cd_steps), int(maxstop_mode), float(maxstop),
                    int(lanes), int(grad_refresh))


def solve_opts(outer_iters, rel_gap_target=0.0, f_star=0.0, alpha_w=0.0, alpha_h=0.0,
               beta_w=0.0, beta_h=0.0, prec="fp32", nnls: NnlsOpts | None = None,
               check_every=1, use_graph=False, obj_hist=None, objective="trace") -> SolveOpts:
    o = SolveOpts()
    o.outer_iters = int(outer_iters)
    o.rel_gap_target = float(rel_gap_target)
    o.f_star = float(f_star)
    o.alpha_w, o.alpha_h, o.beta_w, o.beta_h = (float(alpha_w), float(alpha_h), float(beta_w),
                                                float(beta_h))
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.nnls = nnls or nnls_opts()
    o.check_every = int(check_every)
    o.use_graph = int(bool(use_graph))
    o.objective = {"trace": 0, "direct": 1}[objective]
    o.obj_hist = obj_hist
    return o


class Handle:
    """nmf_create / nmf_destroy.  The stream defaults to torch's current
    stream on ``device``."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._stream = stream
        h = C.c_void_p()
        _check(lib().nmf_create(C.byref(h), self.device, C.c_void_p(stream.cuda_stream)),
               "nmf_create")
        self.h = h

    def set_stream(self, stream):
        self._stream = stream
        _check(lib().nmf_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "nmf_set_stream")

    def sync(self):
        _check(lib().nmf_sync(self.h), "nmf_sync")

    def close(self):
        if getattr(self, "h", None):
            lib().nmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points
def nmf_gram(h: Handle, X, beta=0.0, prec="fp32", Q=None):
    import torch
    _need_cuda(X)
    r = X.shape[1]
    Q = Q if Q is not None else torch.empty(r, r, device=X.device, dtype=torch.float32)
    d = dense(X)
    _check(lib().nmf_gram(h.h, C.byref(d), float(beta), PREC[prec], _ptr(Q)), "nmf_gram")
    return Q


def nmf_gram_noalloc(X, beta=0.0, Q=None, stream=None):
    """Gram without any allocation inside the library (no handle needed); Q
    must be preallocated by the caller when it cannot allocate either.  The
    call runs with X's device current; Q and the stream must belong to it."""
    import torch
    _need_cuda(X)
    r = X.shape[1]
    Q = Q if Q is not None else torch.empty(r, r, device=X.device, dtype=torch.float32)
    if Q.shape != (r, r) or Q.dtype != torch.float32 or Q.device != X.device or \
            not Q.is_contiguous():
        raise ValueError("Q must be a contiguous (r, r) float32 tensor on X's device")
    with torch.cuda.device(X.device):
        stream = stream if stream is not None else torch.cuda.current_stream(X.device)
        if stream.device != X.device:
            raise ValueError("the stream must belong to X's device")
        d = dense(X)
        _check(lib().nmf_gram_noalloc(C.byref(d), float(beta), _ptr(Q),
                                      C.c_void_p(stream.cuda_stream)), "nmf_gram_noalloc")
    return Q


def nmf_cross(h: Handle, V, B, prec="fp32", C_out=None, csr_parts=None):
    """C = V B.  V: dense 2-D tensor, or pass csr_parts=(rowptr, colidx, vals, ncols)."""
    import torch
    r = B.shape[1]
    if csr_parts is not None:
        rp, ci, va, ncols = csr_parts
        _need_cuda(rp, ci, va, B)
        M = matrix_csr(rp, ci, va, ncols)
        rows = rp.numel() - 1
    else:
        _need_cuda(V, B)
        M = matrix_dense(V)
        rows = V.shape[0]
    C_out = C_out if C_out is not None else torch.empty(rows, r, device=B.device,
                                                        dtype=torch.float32)
    _check(lib().nmf_cross(h.h, C.byref(M), _ptr(B), r, PREC[prec], _ptr(C_out)), "nmf_cross")
    return C_out


def nmf_rescale(h: Handle, Q, Qt=None, d=None):
    import torch
    _need_cuda(Q)
    r = Q.shape[0]
    Qt = Qt if Qt is not None else torch.empty_like(Q)
    d = d if d is not None else torch.empty(r, device=Q.device, dtype=torch.float32)
    _check(lib().nmf_rescale(h.h, _ptr(Q), r, _ptr(Qt), _ptr(d)), "nmf_rescale")
    return Qt, d


def nmf_nnls_update(h: Handle, Qt, d, C_in, X, alpha=0.0, opts: NnlsOpts | None = None,
                    inner_iters=None):
    """Solve every row of X in place (Alg. 3); X is the warm start."""
    _need_cuda(Qt, d, C_in, X)
    rows, r = X.shape
    _check(lib().nmf_nnls_update(h.h, _ptr(Qt), _ptr(d), _ptr(C_in), rows, r, float(alpha),
                                 _ptr(X), C.byref(opts) if opts else None, _ptr(inner_iters)),
           "nmf_nnls_update")
    return X


def nmf_objective(h: Handle, vv, W, Ht, Ch, Gw, Gh, alpha_w=0.0, alpha_h=0.0, beta_w=0.0,
                  beta_h=0.0, J=None):
    import torch
    J = J if J is not None else torch.empty(1, device=W.device, dtype=torch.float64)
    _check(lib().nmf_objective(h.h, float(vv), _ptr(W), W.shape[0], _ptr(Ht), Ht.shape[0],
                               W.shape[1], _ptr(Ch), _ptr(Gw), _ptr(Gh), float(alpha_w),
                               float(alpha_h), float(beta_w), float(beta_h), _ptr(J)),
           "nmf_objective")
    return J


def nmf_objective_direct(h: Handle, V, W, Ht, alpha_w=0.0, alpha_h=0.0, beta_w=0.0,
                         beta_h=0.0, J=None):
    import torch
    _need_cuda(V, W, Ht)
    J = J if J is not None else torch.empty(1, device=W.device, dtype=torch.float64)
    d = dense(V)
    _check(lib().nmf_objective_direct(h.h, C.byref(d), _ptr(W), _ptr(Ht), W.shape[1],
                                      float(alpha_w), float(alpha_h), float(beta_w),
                                      float(beta_h), _ptr(J)), "nmf_objective_direct")
    return J


def nmf_kkt(h: Handle, Q, C_in, X, alpha=0.0, out=None):
    import torch
    out = out if out is not None else torch.empty(2, device=X.device, dtype=torch.float64)
    _check(lib().nmf_kkt(h.h, _ptr(Q), _ptr(C_in), X.shape[0], X.shape[1], float(alpha), _ptr(X),
                         _ptr(out)), "nmf_kkt")
    return out


def nmf_solve(h: Handle, V, W, Ht, opts: SolveOpts, Vt=None, csr_parts=None, csr_t_parts=None):
    """Alternating solve in place on W (m x r) and Ht (n x r).

    Dense: V (m x n tensor), optional Vt.  Sparse: csr_parts and csr_t_parts
    = (rowptr, colidx, vals, ncols) of V and V^T.  Tensors may live on the GPU
    or in (preferably pinned) host memory; the library stages host inputs and
    copies W, Ht back.  Returns the Report."""
    r = W.shape[1]
    if csr_parts is not None:
        Mv = matrix_csr(*csr_parts)
        Mt = matrix_csr(*csr_t_parts)
        pt = C.byref(Mt)
    else:
        Mv = matrix_dense(V)
        pt = C.byref(matrix_dense(Vt)) if Vt is not None else None
    rep = Report()
    _check(lib().nmf_solve(h.h, C.byref(Mv), pt, r, _ptr(W), _ptr(Ht), C.byref(opts),
                           C.byref(rep)), "nmf_solve")
    return rep


def nmf_solve_streamed(h: Handle, V, W, Ht, opts: SolveOpts, chunk_rows: int):
    """One-pass solve with V streamed in row chunks (Alg. 2's E-step
    accumulation); V a contiguous float32 tensor on the GPU or in (pinned)
    host memory, W and Ht on the GPU (updated in place).  Returns the Report."""
    _need_cuda(W, Ht)
    if not V.is_contiguous():
        raise ValueError("V must be contiguous")
    rep = Report()
    d = dense(V)
    _check(lib().nmf_solve_streamed(h.h, C.byref(d), W.shape[1], _ptr(W), _ptr(Ht),
                                    C.byref(opts), int(chunk_rows), C.byref(rep)),
           "nmf_solve_streamed")
    return rep


_BATCH_MODES = {"persistent": 0, "loop": 1, "autotune": 2, "phases": 3}


def nmf_solve_batched(h: Handle, instances, opts: SolveOpts, mode="persistent"):
    """Advance independent instances, each a tuple (V, Vt, W, Ht) of device
    tensors (V m x n, Vt its n x m transpose, W m x r, Ht n x r, r <= 64), by
    opts.outer_iters outer iterations, in place.  mode: "persistent" (one
    cooperative launch per iteration for all instances), "loop" (launches per
    instance and phase), "autotune", or "phases" (one launch per phase over
    all instances).  Returns one Report per instance."""
    arr = (Instance * len(instances))()
    for k, (V, Vt, W, Ht) in enumerate(instances):
        _need_cuda(V, Vt, W, Ht)
        m, n = V.shape
        r = W.shape[1]
        if Vt.shape != (n, m) or W.shape != (m, r) or Ht.shape != (n, r):
            raise ValueError(f"instance {k}: inconsistent shapes")
        for t in (V, Vt, W, Ht):
            if _dt(t) != NMF_F32 or not t.is_contiguous():
                raise ValueError(f"instance {k}: tensors must be contiguous float32")
        arr[k] = Instance(m, n, r, _ptr(V), _ptr(Vt), _ptr(W), _ptr(Ht))
    reps = (Report * len(instances))()
    _check(lib().nmf_solve_batched(h.h, len(instances), arr, C.byref(opts),
                                   _BATCH_MODES[mode], reps), "nmf_solve_batched")
    return list(reps)


def nmf_project(h: Handle, Qt, d, W, csr_parts, Hnew, opts: NnlsOpts | None = None):
    rp, ci, va, ncols = csr_parts
    _need_cuda(Qt, d, W, rp, ci, va, Hnew)
    cs = csr(rp, ci, va, ncols)
    _check(lib().nmf_project(h.h, _ptr(Qt), _ptr(d), _ptr(W), W.shape[0], W.shape[1],
                             C.byref(cs), _ptr(Hnew), C.byref(opts) if opts else None),
           "nmf_project")
    return Hnew


class Server:
    """nmf_server_*: continuous-batching projection onto a fixed basis W
    (device tensor, kept referenced here).  Requests are host CSR blocks
    (numpy int64 rowptr, int32 colidx, float32 vals); results land in host
    numpy arrays."""

    def __init__(self, W, slots=4, max_batch_cols=8192, max_batch_nnz=1 << 20,
                 hbm_budget=1 << 30, nnls: NnlsOpts | None = None, device=0):
        _need_cuda(W)
        self._W = W
        o = ServerOpts(int(slots), int(max_batch_cols), int(max_batch_nnz), int(hbm_budget),
                       nnls or nnls_opts())
        s = C.c_void_p()
        _check(lib().nmf_server_create(C.byref(s), int(device), _ptr(W), W.shape[0], W.shape[1],
                                       C.byref(o)), "nmf_server_create")
        self.s = s
        self.r = W.shape[1]
        self._keep = {}

    def submit(self, rowptr, colidx, vals, out=None):
        import numpy as np
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float32)
        w = len(rowptr) - 1
        out = out if out is not None else np.zeros((w, self.r), dtype=np.float32)
        t = C.c_int64()
        _check(lib().nmf_server_submit(self.s, w, len(vals), rowptr.ctypes.data_as(C.c_void_p),
                                       colidx.ctypes.data_as(C.c_void_p),
                                       vals.ctypes.data_as(C.c_void_p),
                                       out.ctypes.data_as(C.c_void_p), C.byref(t)),
               "nmf_server_submit")
        self._keep[t.value] = out
        return t.value, out

    def wait(self, ticket, timeout=60.0):
        lat = C.c_double()
        _check(lib().nmf_server_wait(self.s, int(ticket), float(timeout), C.byref(lat)),
               "nmf_server_wait")
        self._keep.pop(ticket, None)
        return lat.value

    def stats(self):
        st = ServerStats()
        _check(lib().nmf_server_stats(self.s, C.byref(st)), "nmf_server_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "s", None):
            lib().nmf_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
