"""The C-ABI library builds, loads, and exports every entry point that
include/ftn.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^FTN_API\s+[\w\s\*]+?\b(ftn_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2410_02215_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 19
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2410_02215_gb300 import ftn

    monkeypatch.setattr(ftn, "_lib", None)
    monkeypatch.setattr(ftn, "LIB_PATH", str(tmp_path / "missing.so"))
    try:
        ftn.lib()
    except ImportError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected ImportError")


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2410_02215_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
