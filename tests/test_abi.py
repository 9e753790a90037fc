"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/nmf.h declares; host-side argument checks return before any
launch.  No GPU is needed."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nmf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1506_08938_gb300 import build as B
    B.build()
    import paper_1506_08938_gb300 as P
    return P.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(nmf_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("nmf_gram", "nmf_cross", "nmf_rescale", "nmf_nnls_update", "nmf_solve",
              "nmf_project", "nmf_create", "nmf_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (nmf_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"not exported: {missing}"
    for n in declared_functions():
        getattr(lib, n)


def test_build_targets_sm103a_only():
    from paper_1506_08938_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    import paper_1506_08938_gb300 as P
    for s in range(10):
        assert P.status_string(s)
    assert P.status_string(0) == "ok"


def test_argument_errors_return_before_launch(lib):
    import paper_1506_08938_gb300 as P
    before = P.launch_count()
    assert lib.nmf_gram(None, None, C.c_float(0.0), 0, None) == P.NMF_E_ARG
    assert lib.nmf_rescale(None, None, 4, None, None) == P.NMF_E_ARG
    assert lib.nmf_nnls_update(None, None, None, None, 1, 4, C.c_float(0.0), None, None,
                               None) == P.NMF_E_ARG
    assert lib.nmf_solve(None, None, None, 4, None, None, None, None) == P.NMF_E_ARG
    assert lib.nmf_project(None, None, None, None, 0, 4, None, None, None) == P.NMF_E_ARG
    assert lib.nmf_solve_batched(None, 1, None, None, 0, None) == P.NMF_E_ARG
    assert lib.nmf_destroy(None) == P.NMF_E_ARG
    assert lib.nmf_create(None, 0, None) == P.NMF_E_ARG
    assert P.launch_count() == before


def test_default_nnls_options(lib):
    import paper_1506_08938_gb300 as P
    o = P.NnlsOpts()
    lib.nmf_nnls_opts_default(C.byref(o))
    assert o.max_inner == 50 and abs(o.eps - 1e-3) < 1e-15 and o.cd_steps == -1
    assert o.grad_refresh == 0


def test_fault_sites_parse_from_the_environment(lib, monkeypatch):
    """NMF_FAULT is a comma-separated list of injection sites, read at each
    call (no GPU involved): exact names only, no prefixes."""
    monkeypatch.delenv("NMF_FAULT", raising=False)
    assert lib.nmf_fault_armed(b"admit") == 0
    monkeypatch.setenv("NMF_FAULT", "admit,barrier")
    assert lib.nmf_fault_armed(b"admit") == 1
    assert lib.nmf_fault_armed(b"barrier") == 1
    assert lib.nmf_fault_armed(b"alloc") == 0
    assert lib.nmf_fault_armed(b"adm") == 0
    assert lib.nmf_fault_armed(b"") == 0
    monkeypatch.setenv("NMF_FAULT", "csr")
    assert lib.nmf_fault_armed(b"csr") == 1 and lib.nmf_fault_armed(b"admit") == 0
