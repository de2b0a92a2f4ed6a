"""CPU oracle for the ensemble KSG transfer-entropy hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
leg may import this package.  The library's compute path never does, and the two share no
code: the oracle is plain C (``te_oracle.c``) compiled with gcc, called here through ctypes.

Every function cites the passage of Wollstadt et al. (PLoS ONE 2014) it follows in the C
source; this wrapper only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "te_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no fast-math, no FP
    contraction).  Rebuilds when the source is newer than the library."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "te_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Series(C.Structure):
    _fields_ = [("src", C.c_void_p), ("tgt", C.c_void_p), ("R", C.c_int32), ("T", C.c_int32),
                ("d", C.c_int32), ("tau", C.c_int32), ("u", C.c_int32), ("S", C.c_int32),
                ("perms", C.c_void_p)]


class _Instance(C.Structure):
    _fields_ = [("series", C.c_int32), ("t_start", C.c_int32), ("window", C.c_int32),
                ("perm", C.c_int32)]


def configure(lib):
    """Declare the C signatures on a loaded oracle library (also used to load test builds)."""
    P = C.c_void_p
    i = C.c_int
    lib.oracle_embed.argtypes = [P, P, i, i, i, i, i, i, i, i, P, P]
    lib.oracle_knn.argtypes = [P, i, i, i, P, P]
    lib.oracle_range_count.argtypes = [P, i, i, i, P, P]
    lib.oracle_digamma.argtypes = [i]
    lib.oracle_digamma.restype = C.c_double
    lib.oracle_te_points.argtypes = [P, i, i, i, i, P, P, P]
    lib.oracle_te_batch.argtypes = [P, i, P, i, i, i, P, P, P]
    lib.oracle_pvalue.argtypes = [C.c_double, P, i]
    lib.oracle_pvalue.restype = C.c_double
    lib.oracle_points_at.argtypes = [P, i, i, i, i, P, i, i, P, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = configure(C.CDLL(_LIB))
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def embed(src: np.ndarray, tgt: np.ndarray, d: int, tau: int, u: int, t_start: int, window: int,
          perm: Optional[np.ndarray] = None, dy: Optional[int] = None,
          dx: Optional[int] = None) -> np.ndarray:
    """Points [N][D] (N = R*window, D = 1+dy+dx) of one estimate (Eq. 6, 7, 10)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.float32)
    tgt = np.ascontiguousarray(tgt, dtype=np.float32)
    R, T = src.shape
    dy = d if dy is None else dy
    dx = d if dx is None else dx
    p = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    out = np.empty((R * window, 1 + dy + dx), dtype=np.float32)
    rc = lib.oracle_embed(_ptr(src), _ptr(tgt), R, T, dy, dx, tau, u, t_start, window, _ptr(p),
                          _ptr(out))
    if rc == 2:
        raise IndexError("embedding reaches outside the recorded samples")
    _check(rc, "embed")
    return out


def knn(points: np.ndarray, k: int, want_nn: bool = False):
    """eps[N] (float32) and optionally nn[N][k] (int32)."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    N, D = pts.shape
    eps = np.empty(N, dtype=np.float32)
    nn = np.empty((N, k), dtype=np.int32) if want_nn else None
    _check(lib.oracle_knn(_ptr(pts), N, D, k, _ptr(eps), _ptr(nn)), "knn")
    return (eps, nn) if want_nn else eps


def range_count(points: np.ndarray, dy: int, dx: int, eps: np.ndarray) -> np.ndarray:
    """counts[3][N]: n_z (y-), n_yz (y_t, y-), n_xz (y-, x-)."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    N = pts.shape[0]
    assert pts.shape[1] == 1 + dy + dx
    e = np.ascontiguousarray(eps, dtype=np.float32)
    out = np.empty((3, N), dtype=np.int32)
    _check(lib.oracle_range_count(_ptr(pts), N, dy, dx, _ptr(e), _ptr(out)), "range_count")
    return out


def points_at(points: np.ndarray, dy: int, dx: int, k: int, idx, n_threads: Optional[int] = None):
    """(eps[n], counts[3][n]) of the query points ``idx`` only (same definitions as knn and
    range_count), for point sets too large to evaluate whole."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    N = pts.shape[0]
    assert pts.shape[1] == 1 + dy + dx
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    eps = np.empty(len(ix), dtype=np.float32)
    out = np.empty((3, len(ix)), dtype=np.int32)
    _check(lib.oracle_points_at(_ptr(pts), N, dy, dx, k, _ptr(ix), len(ix), n_threads or default_threads(),
                                _ptr(eps), _ptr(out)), "points_at")
    return eps, out


def digamma(n: int) -> float:
    return float(_load().oracle_digamma(int(n)))


def te_points(points: np.ndarray, dy: int, dx: int, k: int):
    """(te, eps, counts) of one point set (Eq. 9 / 10)."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    N = pts.shape[0]
    te = np.zeros(1, dtype=np.float64)
    eps = np.empty(N, dtype=np.float32)
    counts = np.empty((3, N), dtype=np.int32)
    _check(lib.oracle_te_points(_ptr(pts), N, dy, dx, k, _ptr(te), _ptr(eps), _ptr(counts)),
           "te_points")
    return float(te[0]), eps, counts


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def te_batch(series: Sequence, instances: Sequence, k: int, n_threads: Optional[int] = None,
             want_counts: bool = False):
    """TE of many instances.  ``series`` items need .src .tgt .d .tau .u .perms (numpy);
    ``instances`` items need .series .t_start .window .perm.  Returns te [n] (float64) and,
    if asked, the concatenated counts [3*sum N] and eps [sum N]."""
    lib = _load()
    keep = []
    ser = (_Series * len(series))()
    for i, s in enumerate(series):
        src = np.ascontiguousarray(s.src, dtype=np.float32)
        tgt = np.ascontiguousarray(s.tgt, dtype=np.float32)
        perms = None if s.perms is None else np.ascontiguousarray(s.perms, dtype=np.int32)
        keep += [src, tgt, perms]
        ser[i] = _Series(src.ctypes.data, tgt.ctypes.data, src.shape[0], src.shape[1], s.d, s.tau,
                         s.u, 0 if perms is None else perms.shape[0],
                         None if perms is None else perms.ctypes.data)
    ins = (_Instance * max(1, len(instances)))()
    npts = 0
    for i, it in enumerate(instances):
        ins[i] = _Instance(it.series, it.t_start, it.window, it.perm)
        npts += series[it.series].src.shape[0] * it.window
    te = np.zeros(len(instances), dtype=np.float64)
    counts = np.empty(3 * npts, dtype=np.int32) if want_counts else None
    eps = np.empty(npts, dtype=np.float32) if want_counts else None
    nt = n_threads or default_threads()
    rc = lib.oracle_te_batch(C.cast(ser, C.c_void_p), len(series), C.cast(ins, C.c_void_p),
                             len(instances), k, nt, _ptr(te), _ptr(counts), _ptr(eps))
    _check(rc, "te_batch")
    del keep
    return (te, counts, eps) if want_counts else te


def pvalue(te_orig: float, te_surr: np.ndarray) -> float:
    ts = np.ascontiguousarray(te_surr, dtype=np.float64)
    return float(_load().oracle_pvalue(float(te_orig), _ptr(ts), ts.shape[0]))
