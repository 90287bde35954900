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


def test_binding_struct_sizes_match_header(tmp_path):
    """Every struct of the binding has the size the C compiler gives the
    header's declaration."""
    import os
    import subprocess

    from paper_2604_27162_gb300 import hase

    structs = [n for n in dir(hase) if n.startswith("hase_") and isinstance(getattr(hase, n), type)
               and issubclass(getattr(hase, n), ctypes.Structure)]
    assert "hase_config" in structs and "hase_server_config" in structs
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "hase.h"\n#include "hase_serve.h"\nint main(void) {\n'
                   + "".join('    printf("%%s %%zu\\n", "%s", sizeof(%s));\n' % (n, n) for n in structs)
                   + "    return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for n in structs:
        assert ctypes.sizeof(getattr(hase, n)) == int(got[n]), n


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
