"""Host-side checks of the C-ABI library (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "apsp.h")


def _declared():
    hdr = open(HEADER).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(apsp_[a-z0-9_]+)\s*\(", hdr)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1902_04446_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    import paper_1902_04446_gb300 as apsp
    assert apsp._lib.ENTRY_POINTS == _declared()


def test_strerror_and_defaults_are_host_only():
    import paper_1902_04446_gb300 as apsp
    assert apsp.lib.apsp_strerror(0) == b"ok"
    assert apsp.lib.apsp_strerror(4) == b"value out of range"
    cfg = apsp._lib.apsp_config()
    apsp.lib.apsp_config_default(ctypes.byref(cfg))
    assert cfg.max_batch == 64 and cfg.queue_depth == 4096 and cfg.dtype == 0


def test_null_arguments_are_rejected_without_a_gpu():
    import paper_1902_04446_gb300 as apsp
    L = apsp.lib
    assert L.apsp_solve_t(None, 0, None, 4, 4, None, None) == 1           # null handle
    assert L.apsp_create(None, None) == 1
    assert L.apsp_destroy(None) == 0
    assert L.apsp_pack_u16(None, 4, None, 4, 4, None) == 1                 # null matrices
    assert L.apsp_unpack_u16(None, 2, None, 4, 4, None) == 1               # ld < n


def test_dtype_names():
    import paper_1902_04446_gb300 as apsp
    assert apsp.dtype_code("int32") == apsp.APSP_I32
    assert apsp.dtype_code("u16x2") == apsp.APSP_U16
    assert apsp.dtype_code("fp32") == apsp.APSP_F32
    assert apsp.dtype_code("auto") == apsp.APSP_AUTO
    torch = pytest.importorskip("torch")
    assert apsp.dtype_code(torch.int16) == apsp.APSP_U16
