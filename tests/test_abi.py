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
