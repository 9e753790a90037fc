"""FP64 CPU oracle of the paper's alternating NNLS method (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never links or calls it;
the two share no code.  The arithmetic lives in ``oracle.c`` (plain C, FP64,
loops written from the definitions of §3.2-§3.5 and Alg. 1-3); this module
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (OpenMP if gcc has it)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _OUT)
    return _OUT


class NqpOpts(C.Structure):
    _fields_ = [("max_inner", C.c_int), ("eps", C.c_double), ("abs_tol", C.c_double),
                ("cd_steps", C.c_int), ("rescale", C.c_int), ("pg", C.c_int),
                ("maxstop_mode", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("alpha_w", C.c_double), ("alpha_h", C.c_double),
                ("beta_w", C.c_double), ("beta_h", C.c_double), ("nqp", NqpOpts)]


def nqp_opts(max_inner=50, eps=1e-3, abs_tol=0.0, cd_steps=-1, rescale=1, pg=1,
             maxstop_mode=0) -> NqpOpts:
    return NqpOpts(int(max_inner), float(eps), float(abs_tol), int(cd_steps), int(rescale),
                   int(pg), int(maxstop_mode))


_P = C.c_void_p


def load(path: str):
    """Load a compiled oracle library from ``path`` with its signatures set."""
    L = C.CDLL(path)
    L.oracle_gram.argtypes = [_P, C.c_int64, C.c_int, C.c_double, _P]
    L.oracle_cross_dense.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, _P, C.c_int, _P]
    L.oracle_cross_csr.argtypes = [_P, _P, _P, C.c_int64, _P, C.c_int, _P]
    L.oracle_rescale.argtypes = [_P, C.c_int, _P, _P, _P]
    L.oracle_nqp.argtypes = [_P, _P, C.c_int, _P, C.POINTER(NqpOpts), _P, _P]
    L.oracle_nqp.restype = C.c_int
    L.oracle_nqp_min_gap.argtypes = [_P, _P, C.c_int, _P, C.POINTER(NqpOpts), C.c_double, _P]
    L.oracle_nqp_min_gap.restype = C.c_int
    L.oracle_nnls_update.argtypes = [_P, _P, C.c_int64, C.c_int, C.c_double, _P,
                                     C.POINTER(NqpOpts), C.c_double, _P, _P]
    L.oracle_nnls_update.restype = C.c_int64
    L.oracle_objective_dense.argtypes = [_P, C.c_int64, C.c_int64, _P, _P, C.c_int,
                                         C.c_double, C.c_double, C.c_double, C.c_double]
    L.oracle_objective_dense.restype = C.c_double
    L.oracle_objective_csr.argtypes = [_P, _P, _P, C.c_int64, C.c_int64, _P, _P, C.c_int,
                                       C.c_double, C.c_double, C.c_double, C.c_double]
    L.oracle_objective_csr.restype = C.c_double
    L.oracle_kkt.argtypes = [_P, _P, C.c_int64, C.c_int, C.c_double, _P, _P]
    L.oracle_nmf_solve.argtypes = [_P, _P, _P, _P, _P, _P, _P, C.c_int64, C.c_int64,
                                   C.c_int, _P, _P, C.POINTER(SolveOpts), _P]
    L.oracle_nmf_solve.restype = C.c_int64
    L.oracle_num_threads.restype = C.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def num_threads() -> int:
    return lib().oracle_num_threads()


def gram(X, beta=0.0):
    X = _f64(X)
    rows, r = X.shape
    Q = np.empty((r, r))
    lib().oracle_gram(_ptr(X), rows, r, beta, _ptr(Q))
    return Q


def cross_dense(A, B):
    A = _f64(A)
    B = _f64(B)
    rows, k = A.shape
    r = B.shape[1]
    Cm = np.empty((rows, r))
    lib().oracle_cross_dense(_ptr(A), rows, k, k, _ptr(B), r, _ptr(Cm))
    return Cm


def cross_csr(rowptr, colidx, vals, B):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    va = _f64(vals)
    B = _f64(B)
    rows = len(rp) - 1
    r = B.shape[1]
    Cm = np.empty((rows, r))
    lib().oracle_cross_csr(_ptr(rp), _ptr(ci), _ptr(va), rows, _ptr(B), r, _ptr(Cm))
    return Cm


def rescale(H):
    H = _f64(H)
    r = H.shape[0]
    Qt = np.empty((r, r))
    d = np.empty(r)
    dead = np.empty(r, dtype=np.uint8)
    lib().oracle_rescale(_ptr(H), r, _ptr(Qt), _ptr(d), _ptr(dead))
    return Qt, d, dead.astype(bool)


def nqp(H, h, x0, opts: NqpOpts | None = None, maxstop=None):
    """Alg. 3 on one problem; returns (x, iterations, s_final[, maxstop])."""
    H = _f64(H)
    h = _f64(h)
    x = _f64(x0).copy()
    r = H.shape[0]
    o = opts or nqp_opts()
    ms = C.c_double(0.0 if maxstop is None else maxstop)
    sf = C.c_double(0.0)
    k = lib().oracle_nqp(_ptr(H), _ptr(h), r, _ptr(x), C.byref(o), C.addressof(ms),
                         C.addressof(sf))
    if maxstop is None:
        return x, k, sf.value
    return x, k, sf.value, ms.value


def nqp_min_gaps(Q, Cm, alpha, X0, opts: NqpOpts | None = None, tie_units=16.0):
    """Greedy-choice margins of each row of a half-step (as nnls_update, no
    fast break), over the row's coordinate steps (see nqp_core in oracle.c):
    returns (margin, rel_margin, swap) arrays - the smallest gap between the
    two largest gains in units of the gain difference an FP32 gradient cannot
    resolve, the smallest gap relative to the best gain, and the largest move
    |dx_p| + |dx_s| (rescaled variables) of a step whose gap is below
    tie_units such units.  Instrumentation for the parity tests: a row may
    legitimately take another coordinate in FP32 only at such a step, and the
    move swapped there bounds what that choice changes."""
    Q = _f64(Q)
    Cm = _f64(Cm)
    X0 = _f64(X0)
    rows, r = X0.shape
    o = opts or nqp_opts()
    out = np.empty((rows, 3))
    g = (C.c_double * 3)()
    for i in range(rows):
        h = np.ascontiguousarray(-Cm[i] + alpha)
        x = X0[i].copy()
        lib().oracle_nqp_min_gap(_ptr(Q), _ptr(h), r, _ptr(x), C.byref(o), float(tie_units),
                                 C.addressof(g))
        out[i] = g[:]
    return out[:, 0], out[:, 1], out[:, 2]


def nnls_update(Q, Cm, alpha, X0, opts: NqpOpts | None = None, maxstop_in=0.0):
    """One half-step: each row i of X solves min 1/2 x'Qx + (-C_i + alpha)'x,
    x >= 0, from warm start X0_i.  Returns (X, iters per row, total, maxstop_out)."""
    Q = _f64(Q)
    Cm = _f64(Cm)
    X = _f64(X0).copy()
    rows, r = X.shape
    it = np.empty(rows, dtype=np.int32)
    mo = C.c_double(0.0)
    o = opts or nqp_opts()
    tot = lib().oracle_nnls_update(_ptr(Q), _ptr(Cm), rows, r, alpha, _ptr(X), C.byref(o),
                                   maxstop_in, C.addressof(mo), _ptr(it))
    return X, it, int(tot), mo.value


def objective_dense(V, W, Ht, aw=0.0, ah=0.0, bw=0.0, bh=0.0):
    V = _f64(V)
    W = _f64(W)
    Ht = _f64(Ht)
    m, n = V.shape
    return lib().oracle_objective_dense(_ptr(V), m, n, _ptr(W), _ptr(Ht), W.shape[1],
                                        aw, ah, bw, bh)


def objective_csr(rowptr, colidx, vals, m, n, W, Ht, aw=0.0, ah=0.0, bw=0.0, bh=0.0):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    va = _f64(vals)
    W = _f64(W)
    Ht = _f64(Ht)
    return lib().oracle_objective_csr(_ptr(rp), _ptr(ci), _ptr(va), m, n, _ptr(W), _ptr(Ht),
                                      W.shape[1], aw, ah, bw, bh)


def kkt(Q, Cm, alpha, X):
    Q = _f64(Q)
    Cm = _f64(Cm)
    X = _f64(X)
    out = np.empty(2)
    lib().oracle_kkt(_ptr(Q), _ptr(Cm), X.shape[0], X.shape[1], alpha, _ptr(X), _ptr(out))
    return out


def nmf_solve(W0, Ht0, outer_iters, V=None, csr=None, csr_t=None, alpha_w=0.0, alpha_h=0.0,
              beta_w=0.0, beta_h=0.0, opts: NqpOpts | None = None):
    """Alg. 1/2.  V dense (m x n) or csr=(rowptr, colidx, vals) with its
    transpose csr_t.  Returns (W, Ht, hist, total_inner) where hist[2t] and
    hist[2t+1] are J after the W- and H-update of iteration t."""
    W = _f64(W0).copy()
    Ht = _f64(Ht0).copy()
    m, r = W.shape
    n = Ht.shape[0]
    so = SolveOpts(int(outer_iters), alpha_w, alpha_h, beta_w, beta_h, opts or nqp_opts())
    hist = np.empty(2 * outer_iters)
    if V is not None:
        Vd = _f64(V)
        tot = lib().oracle_nmf_solve(_ptr(Vd), None, None, None, None, None, None, m, n, r,
                                     _ptr(W), _ptr(Ht), C.byref(so), _ptr(hist))
    else:
        rp, ci, va = (np.ascontiguousarray(csr[0], np.int64), np.ascontiguousarray(csr[1], np.int32),
                      _f64(csr[2]))
        trp, tci, tva = (np.ascontiguousarray(csr_t[0], np.int64),
                         np.ascontiguousarray(csr_t[1], np.int32), _f64(csr_t[2]))
        tot = lib().oracle_nmf_solve(None, _ptr(rp), _ptr(ci), _ptr(va), _ptr(trp), _ptr(tci),
                                     _ptr(tva), m, n, r, _ptr(W), _ptr(Ht), C.byref(so),
                                     _ptr(hist))
    return W, Ht, hist, int(tot)
