"""Host-side pieces of the benchmark and the binding that need no GPU: the source hash that keys
each kernel's committed DRAM-traffic capture, and the sharing-mode argument check."""
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _copy_tree(tmp_path):
    for sub in ("include", os.path.join("paper_1401_4068_gb300", "csrc")):
        shutil.copytree(os.path.join(ROOT, sub), tmp_path / sub,
                        ignore=shutil.ignore_patterns("__pycache__"))
    return tmp_path


def test_kernel_hashes_are_stable_and_distinct():
    hashes = {k: bench.kernel_source_hash(k) for k in bench.KERNEL_UNITS}
    assert all(len(h) == 16 and int(h, 16) >= 0 for h in hashes.values())
    assert len(set(hashes.values())) == len(hashes)
    assert hashes == {k: bench.kernel_source_hash(k) for k in bench.KERNEL_UNITS}


def test_kernel_hash_follows_the_include_closure(tmp_path, monkeypatch):
    """A change to a file a kernel's units include changes its hash; a change to another kernel's
    own header does not."""
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    before = {k: bench.kernel_source_hash(k) for k in bench.KERNEL_UNITS}
    csrc = root / "paper_1401_4068_gb300" / "csrc"
    with open(csrc / "te_bundle.cuh", "a") as f:
        f.write("\n// edit\n")
    after = {k: bench.kernel_source_hash(k) for k in bench.KERNEL_UNITS}
    assert after["bundle_kernel"] != before["bundle_kernel"]
    assert after["lane_kernel"] == before["lane_kernel"]
    assert after["batched_kernel"] == before["batched_kernel"]
    with open(csrc / "te_device.cuh", "a") as f:  # shared by every search kernel
        f.write("\n// edit\n")
    shared = {k: bench.kernel_source_hash(k) for k in bench.KERNEL_UNITS}
    assert all(shared[k] != after[k] for k in bench.KERNEL_UNITS)
    with open(root / "include" / "te_gb300.h", "a") as f:  # reached through te_internal.h
        f.write("\n/* edit */\n")
    assert bench.kernel_source_hash("lane_kernel") != shared["lane_kernel"]


def test_traffic_needs_a_known_kernel():
    w = type("W", (), {"instances": []})()
    assert bench.traffic_per_launch(w, "no_such_kernel") is None


def test_sharing_mode_must_be_an_integer():
    """A fraction passed as a mode would truncate to 0 (no sharing) without this check."""
    from paper_1401_4068_gb300 import te
    with pytest.raises(TypeError):
        te.te_set_sharing(None, 0.5)
    with pytest.raises(TypeError):
        te.te_set_sharing(None, "auto")
