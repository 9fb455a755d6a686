"""The C ABI library builds for sm_103a, loads, and exports every symbol its header declares.

No compute calls: this runs without a GPU.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(hedap_\w+)\s*\(", text, re.M))
    return names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_2606_10477_gb300 import build, hedap
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(hedap.EXPORTED) <= names


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_is_plain_c_and_cpp(tmp_path, lang, std):
    """include/hedap.h compiles on its own as C99 and as C++17 with every warning an error: plain types, no torch
    or CUDA types in the signatures."""
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "hedap.h"\nint main(void) { return 0; }\n')
    cmd = ["gcc" if lang == "c" else "g++", "-x", lang, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
           "-I", os.path.join(ROOT, "include"), str(src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
