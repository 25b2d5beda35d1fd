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


# The boundary's contract: status codes, the prototypes of the calls the
# problem statement names (Problem 1, Defs. 3-6, Algorithms 3, 5 and 6), and
# the CoreApp result record.
BOUNDARY_STATUS = {"DSD_OK": 0, "DSD_ERR_INVALID": 1, "DSD_ERR_NOMEM": 2, "DSD_ERR_CUDA": 3,
                   "DSD_ERR_TIMEOUT": 4, "DSD_ERR_OVERFLOW": 5, "DSD_ERR_INTERNAL": 6}

BOUNDARY_CALLS = {
    "dsd_graph_from_edges": "uint32_t, uint64_t, const uint32_t*, const uint32_t*, int, void*, "
                            "dsd_graph**",
    "dsd_graph_from_csr": "uint32_t, const uint64_t*, const uint32_t*, int, void*, dsd_graph**",
    "dsd_graph_destroy": "dsd_graph*",
    "dsd_graph_info": "const dsd_graph*, uint32_t*, uint64_t*",
    "dsd_clique_degrees": "dsd_graph*, int, uint64_t*, uint64_t*, int",
    "dsd_core_decompose": "dsd_graph*, int, uint64_t*, uint64_t*, int",
    "dsd_core_app": "dsd_graph*, int, uint32_t*, uint32_t*, int, dsd_core_app_result*",
    "dsd_core_app_seeded": "dsd_graph*, int, const dsd_model*, uint32_t*, uint32_t*, int, "
                           "dsd_core_app_result*",
    "dsd_batch_run": "int, dsd_graph* const*, const int*, dsd_core_app_result*, "
                     "uint64_t* const*, const char*",
    "dsd_status_string": "dsd_status",
}


def _header_text():
    text = open(os.path.join(HEADER_DIR, "dsd.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def _param_types(decl):
    types = []
    for p in decl.split(","):
        p = " ".join(p.split())
        # drop the parameter name (the last identifier), keep the type
        m = re.match(r"^(.*?[\*\s])(\w+)$", p)
        t = m.group(1) if m else p
        types.append(re.sub(r"\s*\*", "*", " ".join(t.split())).strip())
    return ", ".join(types)


def test_status_values_follow_the_boundary():
    text = _header_text()
    body = re.search(r"typedef enum \{(.*?)\} dsd_status;", text, flags=re.S).group(1)
    vals = {k: int(v) for k, v in re.findall(r"(DSD_\w+)\s*=\s*(\d+)", body)}
    for k, v in BOUNDARY_STATUS.items():
        assert vals[k] == v, k
    assert len(set(vals.values())) == len(vals)
    from paper_1906_00341_gb300 import _lib
    assert all(_lib.STATUS[v] == k for k, v in vals.items())


def test_boundary_prototypes():
    text = _header_text()
    for name, want in BOUNDARY_CALLS.items():
        m = re.search(r"\b%s\s*\(([^;]*?)\)\s*;" % name, text, flags=re.S)
        assert m, name
        assert _param_types(m.group(1)) == want, (name, _param_types(m.group(1)))


def test_core_app_result_layout(tmp_path):
    """The ctypes record the binding uses has the C struct's size and field
    offsets (compiled with the host compiler), and carries the boundary's
    fields."""
    import shutil
    import subprocess
    from paper_1906_00341_gb300 import _lib
    fields = [f for f, _ in _lib.CoreAppResult._fields_]
    for want in ("kmax", "kmax_core_size", "kmax_core_mu", "best_k", "densest_size",
                 "densest_mu", "seeded_accepted", "seed_k"):
        assert want in fields
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "layout.c"
    body = "".join('printf("%s %%zu\\n", offsetof(dsd_core_app_result, %s));\n' % (f, f)
                   for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "dsd.h"\n'
                   'int main(void) {\nprintf("size %zu\\n", sizeof(dsd_core_app_result));\n'
                   + body + "return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True,
                                                          capture_output=True,
                                                          text=True).stdout.splitlines())
    import ctypes as C
    assert int(got["size"]) == C.sizeof(_lib.CoreAppResult)
    for f in fields:
        assert int(got[f]) == getattr(_lib.CoreAppResult, f).offset, f


def test_checked_mode_switch_without_gpu(lib):
    from paper_1906_00341_gb300 import _lib
    _lib.dsd_set_checked(True)
    _lib.dsd_set_checked(False)
    rc = lib.dsd_checked_add_selftest(0, None, 1, None, None)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"
    rc = lib.dsd_batch_run(-1, None, None, None, None, None)
    assert _lib.STATUS[rc] == "DSD_ERR_INVALID"


def test_tuning_switches_without_gpu(lib):
    from paper_1906_00341_gb300 import _lib
    # the peel's item thresholds: warp_max outside 2..32 is rejected, the
    # defaults are restored; the PeelApp queue placement never fails
    for bad in (0, 1, 33):
        with pytest.raises(_lib.DSDError) as ei:
            _lib.dsd_set_peel_items(bad, 16)
        assert ei.value.name == "DSD_ERR_INVALID"
    _lib.dsd_set_peel_items(2, 0)
    _lib.dsd_set_peel_items(4, 1 << 20)
    _lib.dsd_set_peel_app_queue(0, 0)
    _lib.dsd_set_peel_app_queue(12288, 1 << 26)
