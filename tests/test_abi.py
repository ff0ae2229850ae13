"""The C-ABI library loads and exports every symbol include/spaqr.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import paper_2010_06807_gb300 as sq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "spaqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spaqr_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(spaqr_lib):
    names = _declared()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(spaqr_lib, nm), nm
    assert sorted(sq.EXPORTS) == names


def test_host_only_calls_without_gpu(spaqr_lib):
    # option defaults and error reporting are host-only
    import ctypes
    o = sq._Opts()
    spaqr_lib.spaqr_opts_default(ctypes.byref(o))
    assert o.eps == 1e-2 and o.skip == 2 and o.scaling == 1
    h = ctypes.c_void_p()
    rc = spaqr_lib.spaqr_order(None, None, 0, ctypes.byref(h))
    assert rc == -1
    assert b"NULL" in spaqr_lib.spaqr_last_error()
    sq.spaqr_stats_reset()
    tot, st = sq.spaqr_stats()
    assert tot == 0 and "cpqr" in st


def test_plain_c_program(spaqr_lib, tmp_path):
    """The header compiles as strict C99 (-pedantic -Werror) and a C program
    linked against libspaqr.so orders a matrix through the ABI alone
    (tests/c_abi_host.c: host-only calls)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    libdir = os.path.dirname(os.path.abspath(spaqr_lib._name))
    exe = str(tmp_path / "c_abi_host")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_host.c"),
                        "-L", libdir, "-lspaqr", "-Wl,-rpath," + libdir, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok n=1600 ")


def test_host_only_error_paths(spaqr_lib):
    """Bad arguments of the host-only calls come back as INVALID_ARG with a
    message (no crash, no handle): NULL handles, nnz < n, nlevels out of
    range, an empty batch; destroying NULL is a no-op."""
    import ctypes

    import numpy as np
    from synth.convdiff import config_problem
    INVALID = -1
    info = sq._OrdInfo()
    assert spaqr_lib.spaqr_ordering_info(None, ctypes.byref(info)) == INVALID
    assert spaqr_lib.spaqr_ordering_rows(None, None) == INVALID
    assert spaqr_lib.spaqr_ordering_get(None, None, None, None, None, None) == INVALID
    assert spaqr_lib.spaqr_last_error()
    spaqr_lib.spaqr_ordering_destroy(None)
    p = config_problem("2d_uniform_a", n=6)
    csr, keep = sq._make_csr(p.rowptr, p.colind, p.val)
    g = sq._Grid(2, 6, 6, 1)
    h = ctypes.c_void_p()
    assert spaqr_lib.spaqr_order(ctypes.byref(csr), ctypes.byref(g), 41, ctypes.byref(h)) == INVALID
    assert spaqr_lib.spaqr_order(ctypes.byref(csr), ctypes.byref(g), -1, ctypes.byref(h)) == INVALID
    short = sq._CSR(csr.n, csr.n - 1, csr.rowptr, csr.colind, csr.val, 0)
    assert spaqr_lib.spaqr_order(ctypes.byref(short), ctypes.byref(g), 0, ctypes.byref(h)) == INVALID
    assert spaqr_lib.spaqr_order_batch(0, ctypes.byref(csr), ctypes.byref(g), ctypes.byref(h)) == INVALID
    assert not h.value
    # a grid whose size does not match n
    g2 = sq._Grid(2, 6, 5, 1)
    assert spaqr_lib.spaqr_order(ctypes.byref(csr), ctypes.byref(g2), 0, ctypes.byref(h)) == INVALID
    assert b"grid" in spaqr_lib.spaqr_last_error()
    del keep


def test_csr_location_flag_checked(spaqr_lib):
    """A->on_device must say where the arrays are: host arrays flagged as
    device memory are refused (INVALID_ARG) before anything reads them."""
    import ctypes

    from synth.convdiff import config_problem
    p = config_problem("2d_uniform_a", n=6)
    csr, keep = sq._make_csr(p.rowptr, p.colind, p.val)
    csr.on_device = 1
    g = sq._Grid(2, 6, 6, 1)
    h = ctypes.c_void_p()
    assert spaqr_lib.spaqr_order(ctypes.byref(csr), ctypes.byref(g), 0, ctypes.byref(h)) == -1
    assert b"host memory" in spaqr_lib.spaqr_last_error()
    assert spaqr_lib.spaqr_order_general(ctypes.byref(csr), 0, 0, ctypes.byref(h)) == -1
    assert not h.value
    del keep
