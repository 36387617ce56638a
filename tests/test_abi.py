"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/mapi.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mapi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mapi_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_core_entry_points():
    syms = declared_symbols()
    for name in ("mapi_create", "mapi_destroy", "mapi_iterate", "mapi_pca_topk",
                 "mapi_pagerank", "mapi_matrix_upload", "mapi_status_str"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    from paper_2110_12065_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    import paper_2110_12065_gb300 as M
    for s in declared_symbols():
        assert hasattr(M, s), s


def test_status_strings_without_gpu():
    import paper_2110_12065_gb300 as M
    M.load()
    assert M.mapi_status_str(0) == "ok"
    assert M.mapi_status_str(4) == "zero norm"


def test_create_rejects_bad_device_without_gpu():
    import paper_2110_12065_gb300 as M
    with pytest.raises(M.MapiError):
        M.mapi_create(device=999, stream=0)
