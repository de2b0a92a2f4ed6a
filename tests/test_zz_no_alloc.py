"""te_surrogate_test_static: the surrogate test for callers that cannot allocate GPU memory
(for example a host whose device memory belongs to another runtime's pool or a fixed budget).
It keeps its scratch in a static device array instead of calling cudaMalloc.

Called here through the C ABI (ctypes on the shared library) and checked against the
allocating entry point te_surrogate_test and against the CPU oracle on the same inputs, for two
different calls in a row, so that a call that reuses the array left by the previous one is
covered too; and a call after the first allocates no device memory (torch's allocator counters
and the driver's free-memory figure are unchanged around it). This file sorts last so that a
run stopping at its first failure has run every other test first."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
TOL = 1e-6  # the TE tolerance of the parity tests


def _static_fn():
    lib = te.load()
    fn = lib.te_surrogate_test_static
    P, i32 = C.c_void_p, C.c_int32
    fn.argtypes = [C.POINTER(te.te_series), P, i32, i32, i32, i32, P, P, P, P, C.c_char_p, i32]
    fn.restype = i32
    return fn


def _outputs(nt, S, dev):
    return {"te_orig": torch.full((nt,), -1.0, dtype=torch.float64, device=dev),
            "te_surr": torch.full((nt, max(S, 1)), -1.0, dtype=torch.float64, device=dev),
            "p": torch.full((nt,), -1.0, dtype=torch.float64, device=dev)}


def _call_static(ds, t_starts, window, S, k, out=None):
    fn = _static_fn()
    nt = len(t_starts)
    if out is None:
        out = _outputs(nt, S, ds.src.device)
    ts = (C.c_int32 * nt)(*t_starts)
    msg = C.create_string_buffer(256)
    desc = ds.desc()
    st = fn(C.byref(desc), C.cast(ts, C.c_void_p), nt, window, S, k, out["te_orig"].data_ptr(),
            out["te_surr"].data_ptr(), out["p"].data_ptr(), torch.cuda.current_stream().cuda_stream,
            msg, 256)
    return st, msg.value.decode(), out


CASES = [
    # surrogate-test shapes: 400 trials, d = 3, window 3 (N = 1200, 7-D), 3 start points x (1 + 40)
    dict(cid=3, kw=dict(n_t=3, S=40), k=4),
    # a different shape right after: 200 trials, d = 2, window 5 (N = 1000, 5-D), 2 x (1 + 25), k = 3
    dict(cid=1, kw={}, k=3),
]


def _workload(case):
    w = I.config(case["cid"], **case["kw"])
    if case["cid"] == 1:
        s = w.series[0]
        s.perms = I.permutations(np.random.default_rng(77), 25, s.R)
        return s, [40, 150], 5, 25
    return w.series[0], w.t_starts[0], w.window, w.S


def test_static_scratch_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    h = te.Handle(0)
    try:
        for case in CASES:  # two calls in a row
            s, t_starts, window, S = _workload(case)
            ds = te.to_device([s])
            ref = te.te_surrogate_test(h, ds, t_starts, window, S, case["k"])
            st, msg, got = _call_static(ds[0], t_starts, window, S, case["k"])
            torch.cuda.synchronize()
            assert st == te.TE_OK, msg
            assert torch.max(torch.abs(got["te_orig"] - ref["te_orig"][0])).item() <= TOL
            assert torch.max(torch.abs(got["te_surr"][:, :S] - ref["te_surr"][0])).item() <= TOL
            assert torch.equal(got["p"], ref["p"][0])
            # and directly against the oracle: TE within the tolerance, p-values equal
            insts = [I.Instance(0, t, window, m) for t in t_starts for m in range(-1, S)]
            o = oracle.te_batch([s], insts, case["k"]).reshape(len(t_starts), S + 1)
            assert np.max(np.abs(got["te_orig"].cpu().numpy() - o[:, 0])) <= TOL
            assert np.max(np.abs(got["te_surr"][:, :S].cpu().numpy() - o[:, 1:])) <= TOL
            for j in range(len(t_starts)):
                assert got["p"][j].item() == oracle.pvalue(o[j, 0], o[j, 1:])
    finally:
        h.close()


def test_a_call_after_the_first_allocates_nothing():
    """The property the entry point exists for: once a device is set up (first call), a call
    changes neither torch's allocator counters nor the device's free memory."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s, t_starts, window, S = _workload(CASES[0])
    ds = te.to_device([s])[0]
    st, msg, first = _call_static(ds, t_starts, window, S, 4)  # first call on the device: set-up
    torch.cuda.synchronize()
    assert st == te.TE_OK, msg
    out = _outputs(len(t_starts), S, ds.src.device)  # outputs allocated before the measurement
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    st, msg, second = _call_static(ds, t_starts, window, S, 4, out)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    assert st == te.TE_OK, msg
    assert after == before
    assert torch.equal(first["te_orig"], second["te_orig"]) and torch.equal(first["p"], second["p"])


def test_static_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    s = I.Series(np.zeros((3000, 20), np.float32), np.zeros((3000, 20), np.float32), d=1, tau=1, u=1)
    ds = te.to_device([s])[0]
    st, msg, _ = _call_static(ds, [5], 3, 0, 4)  # N = 9000 > 8192
    assert st == te.TE_ENOTIMPL and "static scratch" in msg
