"""The C-ABI library loads and exports every symbol include/gapla.h declares
(no compute calls: this runs on machines without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gapla.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(la_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("la_load_grid", "la_load_nets", "la_assign_round", "la_elmore", "la_elmore_backward"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2507_13375_gb300 as la
    from paper_2507_13375_gb300 import build as libbuild

    libbuild.build()
    lib = ctypes.CDLL(la.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(la.EXPORTS) == _declared()


def test_create_fails_cleanly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2507_13375_gb300 as la

    lib = la.library()
    h = ctypes.c_void_p()
    st = lib.la_create(ctypes.byref(h), 0, None)
    assert st != la.LA_OK and not h.value
    assert lib.la_last_error(None)
