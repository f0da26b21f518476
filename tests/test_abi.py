"""The C-ABI library builds, loads and exports every entry point include/rara.h declares.
No compute calls: these run without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rara_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2506_20202_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("rara_preprocess", "rara_bin", "rara_render", "rara_render_frame", "rara_ctx_create"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rara_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2506_20202_gb300 import rara
    assert set(rara.SIGNATURES) == set(declared_functions())
    lib = rara.load(lib_path)
    for name in rara.SIGNATURES:
        assert getattr(lib, name).argtypes is not None


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2506_20202_gb300 import rara
    saved = rara._lib
    rara._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            rara.load(str(tmp_path / "missing.so"))
    finally:
        rara._lib = saved


def test_product_package_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2506_20202_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liborc" not in text, f
