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


def test_instance_array_has_the_c_struct_layout():
    """te_estimate's prepared descriptor array is byte for byte the te_instance array the
    C ABI reads (series, t_start, window, perm as int32)."""
    import numpy as np
    from paper_1401_4068_gb300 import inputs as I
    from paper_1401_4068_gb300 import te
    insts = [I.Instance(0, 5, 3, -1), I.Instance(1, 7, 2, 4), I.Instance(2, 9, 1, 0)]
    arr = te.instance_array(insts)
    ref = (te.te_instance * 3)(*[te.te_instance(i.series, i.t_start, i.window, i.perm) for i in insts])
    assert arr.shape == (3, 4) and arr.tobytes() == bytes(ref)
    assert te.instance_array(arr) is arr
    with pytest.raises(ValueError):
        te.instance_array(arr.astype(np.int64))
    with pytest.raises(ValueError):
        te.instance_array(np.asfortranarray(np.zeros((3, 4), np.int32)))
    empty = te.instance_array([])
    keep, ptr = te._instance_ptr(empty)
    assert empty.shape == (0, 4) and keep.shape == (1, 4) and ptr


def test_te_estimate_marshals_objects_and_prepared_arrays_alike():
    """The binding hands the C call the same descriptors (and sizes its optional outputs from the
    same point count) whether the instances are objects or a prepared int32 [n, 4] array."""
    import numpy as np
    import torch
    from paper_1401_4068_gb300 import inputs as I
    from paper_1401_4068_gb300 import te

    class FakeLib:
        def te_estimate(self, hh, ser, n_ser, ins, n, k, te_p, err_p, counts_p, eps_p, stream):
            self.got = [(ins[i].series, ins[i].t_start, ins[i].window, ins[i].perm) for i in range(n)]
            self.n_ser, self.k = n_ser, k
            return 0

    class FakeHandle:
        h = None
        lib = FakeLib()

        def check(self, status):
            assert status == 0

    series = [te.DeviceSeries(torch.zeros((7, 50)), torch.zeros((7, 50)), 2, 1, 3),
              te.DeviceSeries(torch.zeros((4, 50)), torch.zeros((4, 50)), 1, 1, 2)]
    insts = [I.Instance(0, 10, 3, -1), I.Instance(1, 12, 5, -1), I.Instance(0, 20, 1, -1)]
    h = FakeHandle()
    results = []
    for arg in (insts, te.instance_array(insts)):
        out = te.te_estimate(h, series, arg, 4, want_counts=True, stream=0)
        results.append(list(h.lib.got))
        assert out["counts"].numel() == 3 * (7 * 3 + 4 * 5 + 7 * 1)
        assert out["eps"].numel() == 7 * 3 + 4 * 5 + 7 * 1
    assert results[0] == results[1] == [(0, 10, 3, -1), (1, 12, 5, -1), (0, 20, 1, -1)]
    assert h.lib.n_ser == 2 and h.lib.k == 4
