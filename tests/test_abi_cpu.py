"""CPU checks of the C ABI: the library loads and exports every symbol the
header declares; the binding mirrors the header.  No compute calls."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(hase_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2604_27162_gb300 import build, hase

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hase.EXPORTS) == names


def test_binding_struct_sizes_match_header():
    from paper_2604_27162_gb300 import hase

    assert ctypes.sizeof(hase.hase_env_desc) == 32
    assert ctypes.sizeof(hase.hase_config) == 56
    assert ctypes.sizeof(hase.hase_layout) == 88
    assert ctypes.sizeof(hase.hase_digest_out) == 32
    assert ctypes.sizeof(hase.hase_request) == 56
    assert ctypes.sizeof(hase.hase_serve_config) == 24
    assert ctypes.sizeof(hase.hase_request_result) == 56
    assert ctypes.sizeof(hase.hase_serve_stats) == 24


def test_missing_library_fails_loudly(tmp_path):
    import pytest

    from paper_2604_27162_gb300 import hase

    saved = hase._lib
    hase._lib = None
    try:
        with pytest.raises(RuntimeError):
            hase.load(str(tmp_path / "nope.so"))
    finally:
        hase._lib = saved
