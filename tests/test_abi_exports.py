"""The C-ABI library builds for sm_103a, loads without a GPU, and exports exactly the entry
points that include/te_gb300.h declares (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "te_gb300.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(te_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1401_4068_gb300 import build
    return build.build()


def test_header_declares_the_five_hot_path_calls():
    names = declared()
    for n in ("te_embed", "te_knn_maxnorm", "te_range_count", "te_estimate", "te_surrogate_test"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1401_4068_gb300 import te
    assert sorted(te.EXPORTS) == declared()


def test_only_te_symbols_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if l.split() and l.split()[1] in ("T", "t")]
    extra = [s for s in syms if not s.startswith("te_") and not s.startswith("_")]
    assert not [s for s in syms if s.startswith("te_") and s not in declared()]
    assert not extra, extra[:10]


def test_library_built_for_sm_103a(libpath):
    from paper_1401_4068_gb300 import build
    flags = " ".join(build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert "-use_fast_math" not in flags and "-fmad=false" in flags and "-ftz=false" in flags


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1401_4068_gb300 import te
    monkeypatch.setattr(te, "_lib", None)
    monkeypatch.setattr(te, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        te.load()
