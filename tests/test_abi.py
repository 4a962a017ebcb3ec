"""The C-ABI library builds for sm_103a, loads, and exports every function
include/pic.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import paper_1704_01202_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    """Both builds (FP32 and FP64 arithmetic) export the whole ABI and say
    which arithmetic type they were built with."""
    pkg.build()
    names = _declared()
    assert len(names) >= 15
    for path, nbytes in ((pkg.LIB_PATH, 4), (pkg.LIB64_PATH, 8)):
        lib = ctypes.CDLL(path)
        missing = [n for n in names if not hasattr(lib, n)]
        assert not missing, (path, missing)
        assert lib.pic_real_bytes() == nbytes
    assert sorted(pkg.ABI_FUNCTIONS) == names


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    try:
        pkg.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("binding loaded a missing library")
