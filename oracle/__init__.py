"""Serial CPU oracle for the RCM ordering (plain C, loaded with ctypes).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg. The GPU library never imports it and shares no code with it.

The C source (``rcm_oracle.c``) follows Sec. II-A of the paper: Alg. 2 for the pseudo-peripheral
root, Alg. 1 for the Cuthill-McKee labelling, one reversal at the end, components in start-rule
order. Pins that tie it to the paper and to mathematics rather than to itself live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librcm_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", -1: "bad argument", -2: "bad csr", -3: "out of memory"}


def build(src: str = _SRC, out: str = _LIB_PATH, extra=()) -> str:
    """Compile the oracle with gcc (portable flags only: it runs on x86-64 and aarch64 hosts)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", out, src, *extra]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    lib.oracle_rcm.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i64p]
    lib.oracle_rcm.restype = ctypes.c_int
    lib.oracle_rcm_ex.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i64p, ctypes.c_int]
    lib.oracle_rcm_ex.restype = ctypes.c_int
    lib.oracle_bandwidth_profile.argtypes = [ctypes.c_int32, i32p, i32p, i32p,
                                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_bandwidth_profile.restype = ctypes.c_int
    lib.oracle_pseudo_peripheral.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p]
    lib.oracle_pseudo_peripheral.restype = ctypes.c_int
    lib.oracle_degrees.argtypes = [ctypes.c_int32, i32p, i32p, i32p]
    lib.oracle_degrees.restype = None
    lib.oracle_check_csr.argtypes = [ctypes.c_int32, i32p, i32p]
    lib.oracle_check_csr.restype = ctypes.c_int
    lib.oracle_cm_from_root.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p]
    lib.oracle_cm_from_root.restype = ctypes.c_int32
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library. ``path`` loads another build, e.g. a
    mutant compiled by the tests."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
                build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _arrays(rowptr, colidx):
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    if len(ci) == 0:
        ci = np.zeros(1, np.int32)
    return rp, ci


def rcm(n, rowptr, colidx, lib=None, with_stats=False, row_order=0):
    """RCM permutation perm (new -> old) of the symmetric pattern; raises on a bad input.
    row_order=1: the sort-free variant (children numbered in stored row order)."""
    lib = lib or load()
    rp, ci = _arrays(rowptr, colidx)
    perm = np.empty(max(n, 1), dtype=np.int32)
    stats = np.zeros(8, dtype=np.int64)
    rc = lib.oracle_rcm_ex(int(n), rp, ci, perm, stats, int(row_order)) if row_order else \
        lib.oracle_rcm(int(n), rp, ci, perm, stats)
    if rc != 0:
        raise ValueError(f"oracle_rcm: {STATUS.get(rc, rc)}")
    perm = perm[:n]
    if with_stats:
        return perm, {"components": int(stats[0]), "sweeps": int(stats[1]), "levels": int(stats[2]),
                      "max_ecc": int(stats[3]), "isolated": int(stats[4])}
    return perm


def check_csr(n, rowptr, colidx, lib=None) -> int:
    lib = lib or load()
    rp, ci = _arrays(rowptr, colidx)
    return int(lib.oracle_check_csr(int(n), rp, ci))


def degrees(n, rowptr, colidx, lib=None):
    lib = lib or load()
    rp, ci = _arrays(rowptr, colidx)
    deg = np.empty(max(n, 1), dtype=np.int32)
    lib.oracle_degrees(int(n), rp, ci, deg)
    return deg[:n]


def pseudo_peripheral(n, rowptr, colidx, r0, lib=None):
    """(root, sweeps, ecc(root)) of Alg. 2 started at r0."""
    lib = lib or load()
    rp, ci = _arrays(rowptr, colidx)
    out = np.zeros(3, dtype=np.int32)
    rc = lib.oracle_pseudo_peripheral(int(n), rp, ci, int(r0), out)
    if rc != 0:
        raise ValueError(f"oracle_pseudo_peripheral: {STATUS.get(rc, rc)}")
    return int(out[0]), int(out[1]), int(out[2])


def cm_from_root(n, rowptr, colidx, root, lib=None):
    """Alg. 1 labels of root's component from the given root (others -1)."""
    lib = lib or load()
    rp, ci = _arrays(rowptr, colidx)
    label = np.empty(max(n, 1), dtype=np.int32)
    cnt = lib.oracle_cm_from_root(int(n), rp, ci, int(root), label)
    if cnt < 0:
        raise ValueError("oracle_cm_from_root: bad input")
    return label[:n]


def bandwidth_profile(n, rowptr, colidx, perm, lib=None):
    lib = lib or load()
    rp, ci = _arrays(rowptr, colidx)
    bw, prof = ctypes.c_int64(0), ctypes.c_int64(0)
    pm = np.ascontiguousarray(perm, dtype=np.int32)
    if len(pm) == 0:
        pm = np.zeros(1, np.int32)
    rc = lib.oracle_bandwidth_profile(int(n), rp, ci, pm, ctypes.byref(bw), ctypes.byref(prof))
    if rc != 0:
        raise ValueError(f"oracle_bandwidth_profile: {STATUS.get(rc, rc)}")
    return int(bw.value), int(prof.value)


def rcm_batch(goff, rowptr, colidx, threads: int | None = None, indices=None, with_stats=False):
    """Per-graph oracle orderings of a block-diagonal batch (local ids per segment), one graph per
    thread (ctypes releases the GIL during the C call). Returns a dict index -> perm, or index ->
    (perm, stats) with ``with_stats``."""
    lib = load()
    goff = np.asarray(goff, dtype=np.int64)
    idx = range(len(goff) - 1) if indices is None else indices

    def one(g):
        a, b = int(goff[g]), int(goff[g + 1])
        e0, e1 = int(rowptr[a]), int(rowptr[b])
        rp = (rowptr[a:b + 1] - e0).astype(np.int32)
        ci = (colidx[e0:e1] - a).astype(np.int32)
        return g, rcm(b - a, rp, ci, lib=lib, with_stats=with_stats)

    threads = threads or len(os.sched_getaffinity(0))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return dict(ex.map(one, idx))
