"""CPU-only checks of the C ABI: the library loads and exports every symbol
the public header declares; non-compute entry points behave."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(dsd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1906_00341_gb300 import build as b
    b.build()
    from paper_1906_00341_gb300 import _lib
    return _lib.load()


def test_header_declares_core_calls():
    names = declared_functions()
    for want in ("dsd_graph_from_edges", "dsd_clique_degrees", "dsd_core_decompose",
                 "dsd_core_app", "dsd_graph_destroy", "dsd_status_string"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1906_00341_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings_and_limits(lib):
    from paper_1906_00341_gb300 import _lib
    assert _lib.dsd_status_string(0) == "ok"
    assert "timed out" in _lib.dsd_status_string(4)
    with pytest.raises(_lib.DSDError) as ei:
        _lib.dsd_set_wait_limit_ms(0)
    assert ei.value.name == "DSD_ERR_INVALID"
    _lib.dsd_set_wait_limit_ms(20000)
    assert "sm_103a" in _lib.dsd_version()


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1906_00341_gb300 import _lib
    # argument validation happens before any CUDA call
    rc = lib.dsd_graph_from_edges(3, 1, None, None, 0, None, None)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    rc = lib.dsd_core_app(None, 3, None, None, 0, None)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    rc = lib.dsd_core_exact(None, 3, None, 0, None)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    rc = lib.dsd_pattern_degrees(None, 1, 2, None, None, 0)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    rc = lib.dsd_pattern_core_decompose(None, 2, 0, None, None, None, None, None, 0, None, 0)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    rc = lib.dsd_pattern_core_app(None, 1, 3, None, None, 0, None)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    lib.dsd_graph_destroy(None)   # NULL-safe
