"""Python binding of the C ABI in ``include/te_gb300.h`` (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and does no arithmetic of the
method: it checks tensor devices/dtypes/layouts, allocates outputs with torch when the caller
passes none, converts descriptors to the C structs and raises ``TEError`` on a non-zero
status. PyTorch supplies device memory and the current CUDA stream.

The shared library is the in-tree ``_lib/libte_gb300.so`` built by ``build.build()``; there is
no other implementation to fall back to, so a missing library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

TE_OK, TE_EINVAL, TE_ERANGE, TE_ENOMEM, TE_ECUDA, TE_ETIMEOUT, TE_ENOTIMPL = range(7)
_STATUS = {0: "TE_OK", 1: "TE_EINVAL", 2: "TE_ERANGE", 3: "TE_ENOMEM", 4: "TE_ECUDA",
           5: "TE_ETIMEOUT", 6: "TE_ENOTIMPL"}

# every symbol the header declares (checked by the tests against include/te_gb300.h)
EXPORTS = ["te_create", "te_destroy", "te_last_error", "te_sync_status", "te_embed",
           "te_knn_maxnorm", "te_range_count", "te_estimate", "te_surrogate_test",
           "te_set_profiling", "te_last_kernel_ms", "te_last_launch_count", "te_set_launch_config",
           "te_set_batching", "te_surrogate_test_static", "te_autotune", "te_delay_scan",
           "te_set_search", "te_last_work", "te_set_sharing", "te_last_alu_ops", "te_last_pass_work",
           "te_last_paths"]


class TEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class te_params(C.Structure):
    _fields_ = [("d", C.c_int32), ("tau", C.c_int32), ("u", C.c_int32), ("k", C.c_int32),
                ("t_start", C.c_int32), ("window", C.c_int32)]


class te_series(C.Structure):
    _fields_ = [("src", C.c_void_p), ("tgt", C.c_void_p), ("R", C.c_int32), ("T", C.c_int32),
                ("d", C.c_int32), ("tau", C.c_int32), ("u", C.c_int32), ("S", C.c_int32),
                ("perms", C.c_void_p)]


class te_instance(C.Structure):
    _fields_ = [("series", C.c_int32), ("t_start", C.c_int32), ("window", C.c_int32),
                ("perm", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path} missing): run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, i32 = C.c_void_p, C.c_int32
    lib.te_create.argtypes = [C.POINTER(P), i32]
    lib.te_create.restype = i32
    lib.te_destroy.argtypes = [P]
    lib.te_destroy.restype = None
    lib.te_last_error.argtypes = [P]
    lib.te_last_error.restype = C.c_char_p
    lib.te_sync_status.argtypes = [P, P]
    lib.te_embed.argtypes = [P, P, P, i32, i32, C.POINTER(te_params), P, P, i32, P]
    lib.te_knn_maxnorm.argtypes = [P, P, i32, i32, i32, i32, P, P, P]
    lib.te_range_count.argtypes = [P, P, i32, i32, i32, i32, P, P, P]
    lib.te_estimate.argtypes = [P, C.POINTER(te_series), i32, C.POINTER(te_instance), i32, i32,
                                P, P, P, P, P]
    lib.te_surrogate_test.argtypes = [P, C.POINTER(te_series), i32, P, i32, i32, i32, i32, P, P,
                                      P, P]
    lib.te_set_profiling.argtypes = [P, i32]
    lib.te_last_kernel_ms.argtypes = [P, C.POINTER(C.c_float)]
    lib.te_last_launch_count.argtypes = [P]
    lib.te_set_launch_config.argtypes = [P, i32, i32]
    lib.te_set_batching.argtypes = [P, i32]
    lib.te_set_search.argtypes = [P, i32]
    lib.te_last_work.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(i32)]
    lib.te_set_sharing.argtypes = [P, i32]
    lib.te_last_alu_ops.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(i32)]
    lib.te_last_pass_work.argtypes = [P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    lib.te_last_paths.argtypes = [P, C.POINTER(i32)]
    lib.te_delay_scan.argtypes = [P, C.POINTER(te_series), P, i32, i32, i32, i32, i32, i32, P, P, P, P]
    lib.te_autotune.argtypes = [P, C.POINTER(te_series), i32, C.POINTER(te_instance), i32, i32,
                                C.c_char_p, C.POINTER(i32), C.POINTER(i32), P]
    for name in ("te_sync_status", "te_embed", "te_knn_maxnorm", "te_range_count", "te_estimate",
                 "te_surrogate_test", "te_set_profiling", "te_last_kernel_ms",
                 "te_last_launch_count", "te_set_launch_config", "te_set_batching", "te_autotune", "te_delay_scan",
                 "te_set_search", "te_last_work", "te_set_sharing", "te_last_alu_ops", "te_last_pass_work",
                 "te_last_paths"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


# ------------------------------------------------------------------------------- helpers
def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _need_out(t, dtype, numel: int, dev, name: str):
    """A caller-supplied output: a contiguous CUDA tensor of `dtype` on `dev` with room for
    `numel` elements (the library writes that many)."""
    _need(t, dtype, name)
    if t.device != torch.device(dev):
        raise ValueError(f"{name} must be on {dev}, got {t.device}")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the call writes {numel}")


class Handle:
    """Owner of a ``te_handle*`` (device workspace, cached plans and graphs)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.te_create(C.byref(h), int(device))
        if st != TE_OK:
            raise TEError(st, self.lib.te_last_error(None).decode())
        self.h = h
        self.device = int(device)

    def check(self, st: int):
        if st != TE_OK:
            raise TEError(st, self.lib.te_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.te_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def te_create(device: int = 0) -> Handle:
    return Handle(device)


def te_destroy(h: Handle):
    h.close()


def te_last_error(h: Optional[Handle]) -> str:
    lib = load()
    return lib.te_last_error(None if h is None else h.h).decode()


def te_sync_status(h: Handle, stream=None):
    h.check(h.lib.te_sync_status(h.h, _stream(stream)))


def te_embed(h: Handle, src: torch.Tensor, tgt: torch.Tensor, d: int, tau: int, u: int,
             t_start: int, window: int, perm: Optional[torch.Tensor] = None,
             points: Optional[torch.Tensor] = None, ld: Optional[int] = None, stream=None):
    """Points [D][ld] (SoA) of one estimate; returns (points, N, D, ld)."""
    _need(src, torch.float32, "src")
    _need(tgt, torch.float32, "tgt")
    R, T = src.shape
    N = R * window
    D = 1 + 2 * d
    ld = ld or ((N + 3) // 4) * 4
    if tgt.shape != src.shape:
        raise ValueError(f"src {tuple(src.shape)} and tgt {tuple(tgt.shape)} differ")
    if points is None:
        points = torch.full((D, ld), float("nan"), dtype=torch.float32, device=src.device)
    _need_out(points, torch.float32, D * ld, src.device, "points")
    if perm is not None:
        _need_out(perm, torch.int32, R, src.device, "perm")
    p = te_params(d, tau, u, 0, t_start, window)
    h.check(h.lib.te_embed(h.h, _ptr(src), _ptr(tgt), R, T, C.byref(p), _ptr(perm), _ptr(points),
                           ld, _stream(stream)))
    return points, N, D, ld


def te_knn_maxnorm(h: Handle, points: torch.Tensor, N: int, D: int, ld: int, k: int,
                   eps: Optional[torch.Tensor] = None, want_nn: bool = False, stream=None):
    _need_out(points, torch.float32, D * ld, points.device, "points")
    if eps is None:
        eps = torch.full((N,), float("nan"), dtype=torch.float32, device=points.device)
    _need_out(eps, torch.float32, N, points.device, "eps")
    nn = torch.full((N, k), -1, dtype=torch.int32, device=points.device) if want_nn else None
    h.check(h.lib.te_knn_maxnorm(h.h, _ptr(points), N, D, ld, k, _ptr(eps), _ptr(nn),
                                 _stream(stream)))
    return (eps, nn) if want_nn else eps


def te_range_count(h: Handle, points: torch.Tensor, N: int, d_y: int, d_x: int, ld: int,
                   eps: torch.Tensor, counts: Optional[torch.Tensor] = None, stream=None):
    _need_out(points, torch.float32, (1 + d_y + d_x) * ld, points.device, "points")
    _need_out(eps, torch.float32, N, points.device, "eps")
    if counts is None:
        counts = torch.full((3, N), -1, dtype=torch.int32, device=points.device)
    _need_out(counts, torch.int32, 3 * N, points.device, "counts")
    h.check(h.lib.te_range_count(h.h, _ptr(points), N, d_y, d_x, ld, _ptr(eps), _ptr(counts),
                                 _stream(stream)))
    return counts


@dataclass
class DeviceSeries:
    """Device copies of one series (and its permutations) plus the C descriptor."""
    src: torch.Tensor
    tgt: torch.Tensor
    d: int
    tau: int
    u: int
    perms: Optional[torch.Tensor] = None

    @property
    def S(self) -> int:
        return 0 if self.perms is None else int(self.perms.shape[0])

    def desc(self) -> te_series:
        return te_series(self.src.data_ptr(), self.tgt.data_ptr(), self.src.shape[0],
                         self.src.shape[1], self.d, self.tau, self.u, self.S,
                         None if self.perms is None else self.perms.data_ptr())


def to_device(series: Sequence, device="cuda", non_blocking: bool = False) -> List[DeviceSeries]:
    """Copy host series (objects with src, tgt, d, tau, u, perms as numpy or torch) to the GPU."""
    out = []
    for s in series:
        def dev(a, dt):
            if a is None:
                return None
            t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
            return t.to(device=device, dtype=dt, non_blocking=non_blocking).contiguous()
        out.append(DeviceSeries(dev(s.src, torch.float32), dev(s.tgt, torch.float32), int(s.d),
                                int(s.tau), int(s.u), dev(s.perms, torch.int32)))
    return out


def _series_array(series: Sequence[DeviceSeries]):
    arr = (te_series * len(series))()
    for i, s in enumerate(series):
        arr[i] = s.desc()
    return arr


def instance_array(instances) -> np.ndarray:
    """The te_instance descriptors of `instances` (objects with series, t_start, window, perm) as
    a C-contiguous int32 [n, 4] array, the struct's memory layout. te_estimate and te_autotune
    accept such an array in place of the objects, so a caller that repeats a batch builds it once
    (an already built array is returned as it is)."""
    if isinstance(instances, np.ndarray):
        if instances.dtype != np.int32 or instances.ndim != 2 or instances.shape[1] != 4 \
                or not instances.flags.c_contiguous:
            raise ValueError("an instance array is C-contiguous int32 [n, 4]: series, t_start, window, perm")
        return instances
    return np.array([(int(it.series), int(it.t_start), int(it.window), int(it.perm)) for it in instances],
                    dtype=np.int32).reshape(-1, 4)


def _instance_ptr(arr: np.ndarray):
    """te_instance* for an instance array (a one-element dummy when it is empty)."""
    if arr.shape[0] == 0:
        arr = np.zeros((1, 4), dtype=np.int32)
    return arr, arr.ctypes.data_as(C.POINTER(te_instance))


def te_estimate(h: Handle, series: Sequence[DeviceSeries], instances: Sequence, k: int,
                te: Optional[torch.Tensor] = None, want_err: bool = False,
                want_counts: bool = False, stream=None):
    """TE of every instance (objects with series, t_start, window, perm) in one batched launch.
    Returns te [n] (float64) or a dict with te, err_bound, counts, eps when asked."""
    dev = series[0].src.device
    arr = instance_array(instances)
    n = arr.shape[0]
    ser = _series_array(series)
    keep, ins = _instance_ptr(arr)
    npts = 0
    if want_counts:  # points of the valid instances; the library validates the rest
        sid = arr[:, 0].astype(np.int64)
        ok = (sid >= 0) & (sid < len(series))
        rows = np.array([s.src.shape[0] for s in series], dtype=np.int64)
        npts = int((rows[sid[ok]] * np.maximum(arr[ok, 2], 0).astype(np.int64)).sum())
    if te is None:
        te = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    else:
        _need_out(te, torch.float64, n, dev, "te")
    err = torch.full((n,), float("nan"), dtype=torch.float64, device=dev) if want_err else None
    # sentinels (-1, NaN): a point the library failed to write can never pass for a result
    counts = torch.full((3 * npts,), -1, dtype=torch.int32, device=dev) if want_counts else None
    eps = torch.full((npts,), float("nan"), dtype=torch.float32, device=dev) if want_counts else None
    h.check(h.lib.te_estimate(h.h, ser, len(series), ins, n, int(k), _ptr(te), _ptr(err),
                              _ptr(counts), _ptr(eps), _stream(stream)))
    if not (want_err or want_counts):
        return te
    return {"te": te, "err_bound": err, "counts": counts, "eps": eps}


def te_surrogate_test(h: Handle, series: Sequence[DeviceSeries], t_starts: Sequence[int],
                      window: int, S: int, k: int, out=None, stream=None):
    """Original TE, S surrogate TEs and the p-value per (series, t_start)."""
    dev = series[0].src.device
    ns, nt = len(series), len(t_starts)
    ser = _series_array(series)
    ts = (C.c_int32 * max(1, nt))(*[int(t) for t in t_starts])
    if out is None:
        out = {"te_orig": torch.full((ns, nt), float("nan"), dtype=torch.float64, device=dev),
               "te_surr": torch.full((ns, nt, max(S, 1)), float("nan"), dtype=torch.float64, device=dev),
               "p": torch.full((ns, nt), float("nan"), dtype=torch.float64, device=dev)}
    else:
        _need_out(out["te_orig"], torch.float64, ns * nt, dev, "te_orig")
        _need_out(out["te_surr"], torch.float64, ns * nt * max(S, 0), dev, "te_surr")
        _need_out(out["p"], torch.float64, ns * nt, dev, "p")
    h.check(h.lib.te_surrogate_test(h.h, ser, ns, C.cast(ts, C.c_void_p), nt, int(window),
                                    int(S), int(k), _ptr(out["te_orig"]), _ptr(out["te_surr"]),
                                    _ptr(out["p"]), _stream(stream)))
    return out


def te_set_profiling(h: Handle, enable: bool):
    h.check(h.lib.te_set_profiling(h.h, 1 if enable else 0))


def te_last_kernel_ms(h: Handle) -> float:
    ms = C.c_float()
    h.check(h.lib.te_last_kernel_ms(h.h, C.byref(ms)))
    return float(ms.value)


def te_last_launch_count(h: Handle) -> int:
    return int(h.lib.te_last_launch_count(h.h))


def te_set_launch_config(h: Handle, threads: int = 0, qpt: int = 0):
    h.check(h.lib.te_set_launch_config(h.h, int(threads), int(qpt)))


def te_set_batching(h: Handle, per_instance: bool):
    h.check(h.lib.te_set_batching(h.h, 1 if per_instance else 0))


def te_autotune(h: Handle, series: Sequence[DeviceSeries], instances: Sequence, k: int,
                cache_path: Optional[str] = None, stream=None):
    """Measure and keep the batched kernel's launch shape for this batch signature.
    Returns (threads, queries_per_thread)."""
    ser = _series_array(series)
    arr = instance_array(instances)
    n = arr.shape[0]
    keep, ins = _instance_ptr(arr)
    t, q = C.c_int32(), C.c_int32()
    h.check(h.lib.te_autotune(h.h, ser, len(series), ins, n, int(k),
                              None if cache_path is None else cache_path.encode(),
                              C.byref(t), C.byref(q), _stream(stream)))
    return int(t.value), int(q.value)


def te_delay_scan(h: Handle, series: DeviceSeries, t_starts: Sequence[int], window: int, u_lo: int,
                  u_hi: int, S: int, k: int, out=None, stream=None):
    """TE for every scanned delay u_lo..u_hi and start, p-values, and the argmax delay per start."""
    dev = series.src.device
    n_u, n_t = u_hi - u_lo + 1, len(t_starts)
    ser = _series_array([series])
    ts = (C.c_int32 * max(1, n_t))(*[int(t) for t in t_starts])
    if out is None:  # sizes clamped to >= 1 so that the library, not torch, rejects bad ranges
        out = {"te": torch.full((max(n_u, 1), max(n_t, 1)), float("nan"), dtype=torch.float64, device=dev),
               "p": torch.full((max(n_u, 1), max(n_t, 1)), float("nan"), dtype=torch.float64, device=dev),
               "u_best": torch.full((max(n_t, 1),), -1, dtype=torch.int32, device=dev)}
    else:
        _need_out(out["te"], torch.float64, max(n_u, 0) * n_t, dev, "te")
        _need_out(out["p"], torch.float64, max(n_u, 0) * n_t, dev, "p")
        _need_out(out["u_best"], torch.int32, n_t, dev, "u_best")
    h.check(h.lib.te_delay_scan(h.h, ser, C.cast(ts, C.c_void_p), n_t, int(window), int(u_lo), int(u_hi),
                                int(S), int(k), _ptr(out["te"]), _ptr(out["p"]), _ptr(out["u_best"]),
                                _stream(stream)))
    return out


def te_set_search(h: Handle, sweep: bool):
    """True: sorted sweep (default); False: exhaustive search over all pairs."""
    h.check(h.lib.te_set_search(h.h, 1 if sweep else 0))


def te_last_work(h: Handle):
    """(pair evaluations, FP32 ops, swept) of the last batched call."""
    pr, op, sw = C.c_uint64(), C.c_uint64(), C.c_int32()
    h.check(h.lib.te_last_work(h.h, C.byref(pr), C.byref(op), C.byref(sw)))
    return int(pr.value), int(op.value), bool(sw.value)


SHARE_NONE, SHARE_AUTO, SHARE_BUNDLES, SHARE_LANES = 0, 1, 2, 3


def te_set_sharing(h: Handle, mode):
    """Target-part sharing: 1 or True (default) = one estimate per lane for groups of at least 32
    estimates with one target part and d = 3..8, bundles of up to 3 for other groups; 3 = the lane
    kernel for every group of at least 8 with d = 2..8; 2 = bundles only; 0 or False = none."""
    if not isinstance(mode, (bool, int)):
        raise TypeError(f"te_set_sharing: mode must be an int or bool, got {type(mode).__name__}")
    h.check(h.lib.te_set_sharing(h.h, int(mode)))


def te_last_paths(h: Handle):
    """(estimates on the lane kernel, in bundles, unshared) of the last batched call."""
    v = (C.c_int32 * 3)()
    h.check(h.lib.te_last_paths(h.h, v))
    return int(v[0]), int(v[1]), int(v[2])


def te_last_pass_work(h: Handle):
    """((pass-1 pairs, pass-2 pairs), (pass-1 warp cycles, pass-2 warp cycles)) of the last
    batched call; cycles are 0 for the exhaustive search."""
    pr, cy = (C.c_uint64 * 2)(), (C.c_uint64 * 2)()
    h.check(h.lib.te_last_pass_work(h.h, pr, cy))
    return (int(pr[0]), int(pr[1])), (int(cy[0]), int(cy[1]))


def te_last_alu_ops(h: Handle):
    """(FP32 ops the kernels executed, bundles) of the last batched call."""
    op, nb = C.c_uint64(), C.c_int32()
    h.check(h.lib.te_last_alu_ops(h.h, C.byref(op), C.byref(nb)))
    return int(op.value), int(nb.value)
