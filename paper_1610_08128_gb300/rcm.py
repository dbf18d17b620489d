"""Thin Python binding of the C ABI in include/rcm.h (argument marshalling only).

Every function has the C name and argument order, takes torch tensors (or raw pointers as ints)
and returns the C status code. All ordering work runs in the CUDA library; if the library is not
built this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

RCM_OK = 0
RCM_ERR_INVALID_ARG = 1
RCM_ERR_BAD_CSR = 2
RCM_ERR_OOM = 3
RCM_ERR_TOO_LARGE = 4
RCM_ERR_CUDA = 5
RCM_ERR_TIMEOUT = 6
RCM_ERR_NOT_READY = 7
RCM_ERR_UNKNOWN_TICKET = 8


class RcmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


class rcm_options(ctypes.Structure):
    _fields_ = [
        ("narrow_threshold", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("fused_sweeps", ctypes.c_int32),
        ("spin_limit_ns", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("debug_stall_barrier", ctypes.c_int32),
        ("profile_phases", ctypes.c_int32),
        ("cluster", ctypes.c_int32),
        ("executor", ctypes.c_int32),
        ("async_sweeps", ctypes.c_int32),
        ("debug_async_slots", ctypes.c_int32),
        ("row_order", ctypes.c_int32),
        ("expand_mode", ctypes.c_int32),
        ("bottom_up_divisor", ctypes.c_int32),
        ("l2_persist", ctypes.c_int32),
        ("debug_order_bits", ctypes.c_int32),
        ("mid_cluster", ctypes.c_int32),
        ("mid_threshold", ctypes.c_int32),
        ("components_first", ctypes.c_int32),
    ]


class rcm_batch_options(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("row_sort_split", ctypes.c_int32),
                ("row_order", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class rcm_server_options(ctypes.Structure):
    _fields_ = [("cluster_min_vertices", ctypes.c_int64), ("cluster_blocks", ctypes.c_int32),
                ("debug_fail_after", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class rcm_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "components", "sweeps", "traversals", "levels", "max_ecc", "isolated", "narrow_levels", "grid_levels")] + [
        ("prep_ms", ctypes.c_double), ("traverse_ms", ctypes.c_double), ("phase_ns", ctypes.c_int64 * 8)]

    def as_dict(self):
        out = {}
        for f, t in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if f == "phase_ns" else (float if t is ctypes.c_double else int)(v)
        return out


class rcm_validate_report(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "bad_rows", "bad_columns", "duplicates", "asymmetric", "diagonal", "max_row", "first_bad_row", "reserved")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_ if f != "reserved"}


class rcm_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "completed", "failed", "cancelled", "waiting", "running", "max_running", "arena_bytes",
        "arena_peak_bytes")] + [(f, ctypes.c_double) for f in ("latency_p50_s", "latency_p99_s", "latency_max_s")]

    def as_dict(self):
        return {f: (float if t is ctypes.c_double else int)(getattr(self, f)) for f, t in self._fields_}


_lib = None


def library_path() -> str:
    return LIB_PATH


def load():
    """Load librcm_gb300.so. Raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1610_08128_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sigs = {
        "rcm_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "rcm_order": ([I32, P, P, P, P], ctypes.c_int),
        "rcm_order_ex": ([I32, P, P, P, ctypes.POINTER(rcm_options), ctypes.POINTER(rcm_stats), P], ctypes.c_int),
        "rcm_order_host": ([I32, P, P, P, P], ctypes.c_int),
        "rcm_order_noalloc": ([I32, P, P, P, P], ctypes.c_int),
        "rcm_order_batch": ([I32, I64, P, P, P, P, P], ctypes.c_int),
        "rcm_order_batch_ex": ([I32, I64, P, P, P, P, ctypes.POINTER(rcm_batch_options), P], ctypes.c_int),
        "rcm_batch_plan_create": ([I32, I64, I64, P, P, P, P, ctypes.POINTER(rcm_batch_options),
                                   ctypes.POINTER(P)], ctypes.c_int),
        "rcm_batch_plan_launch": ([P, P], ctypes.c_int),
        "rcm_batch_plan_status": ([P, P], ctypes.c_int),
        "rcm_batch_plan_destroy": ([P], ctypes.c_int),
        "rcm_stream_status": ([P], ctypes.c_int),
        "rcm_workspace_bytes": ([I32, I64], SZ),
        "rcm_bandwidth_profile": ([I32, P, P, P, ctypes.POINTER(I64), ctypes.POINTER(I64), P], ctypes.c_int),
        "rcm_validate": ([I32, P, P, ctypes.POINTER(rcm_validate_report), P], ctypes.c_int),
        "rcm_request_bytes": ([I32, I64, I32, I32], SZ),
        "rcm_server_create": ([SZ, I32, ctypes.POINTER(P)], ctypes.c_int),
        "rcm_server_create_ex": ([SZ, I32, ctypes.POINTER(rcm_server_options), ctypes.POINTER(P)], ctypes.c_int),
        "rcm_submit": ([P, I32, I64, P, P, P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "rcm_poll": ([P, ctypes.c_uint64], ctypes.c_int),
        "rcm_wait": ([P, ctypes.c_uint64], ctypes.c_int),
        "rcm_cancel": ([P, ctypes.c_uint64], ctypes.c_int),
        "rcm_server_info": ([P, ctypes.POINTER(rcm_server_stats)], ctypes.c_int),
        "rcm_server_destroy": ([P], ctypes.c_int),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(x, device: bool | None = None, dtype=None):
    """Raw pointer of a torch tensor (checked) or an int; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch

    if not isinstance(x, torch.Tensor):
        raise TypeError(f"expected a torch.Tensor or an int pointer, got {type(x)}")
    if dtype is not None and x.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {x.dtype}")
    if device is True and not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if device is False and x.is_cuda:
        raise ValueError("expected a host tensor")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def status_string(status: int) -> str:
    return load().rcm_status_string(int(status)).decode()


def _i32():
    import torch

    return torch.int32


def rcm_order(n, rowptr, colidx, perm_out, stream=None) -> int:
    return load().rcm_order(int(n), _ptr(rowptr, True, _i32()), _ptr(colidx, True, _i32()),
                            _ptr(perm_out, True, _i32()), _stream(stream))


def rcm_order_ex(n, rowptr, colidx, perm_out, options: rcm_options | None = None,
                 stats: rcm_stats | None = None, stream=None) -> int:
    return load().rcm_order_ex(int(n), _ptr(rowptr, True, _i32()), _ptr(colidx, True, _i32()),
                               _ptr(perm_out, True, _i32()),
                               ctypes.byref(options) if options is not None else None,
                               ctypes.byref(stats) if stats is not None else None, _stream(stream))


def rcm_order_host(n, rowptr, colidx, perm_out, stream=None) -> int:
    return load().rcm_order_host(int(n), _ptr(rowptr, False, _i32()), _ptr(colidx, False, _i32()),
                                 _ptr(perm_out, False, _i32()), _stream(stream))


def rcm_order_noalloc(n, rowptr, colidx, perm_out, stream=None) -> int:
    return load().rcm_order_noalloc(int(n), _ptr(rowptr, True, _i32()), _ptr(colidx, True, _i32()),
                                    _ptr(perm_out, True, _i32()), _stream(stream))


def rcm_order_batch(G, n_total, goff, rowptr, colidx, perm_out, stream=None) -> int:
    import torch

    return load().rcm_order_batch(int(G), int(n_total), _ptr(goff, True, torch.int64), _ptr(rowptr, True, _i32()),
                                  _ptr(colidx, True, _i32()), _ptr(perm_out, True, _i32()), _stream(stream))


def rcm_order_batch_ex(G, n_total, goff, rowptr, colidx, perm_out, options=None, stream=None) -> int:
    import torch

    return load().rcm_order_batch_ex(int(G), int(n_total), _ptr(goff, True, torch.int64), _ptr(rowptr, True, _i32()),
                                     _ptr(colidx, True, _i32()), _ptr(perm_out, True, _i32()),
                                     ctypes.byref(options) if options is not None else None, _stream(stream))


def rcm_batch_plan_create(G, n_total, nnz, goff, rowptr, colidx, perm_out, options=None):
    """Returns (status, plan handle)."""
    import torch

    h = ctypes.c_void_p()
    st = load().rcm_batch_plan_create(int(G), int(n_total), int(nnz), _ptr(goff, True, torch.int64),
                                      _ptr(rowptr, True, _i32()), _ptr(colidx, True, _i32()),
                                      _ptr(perm_out, True, _i32()),
                                      ctypes.byref(options) if options is not None else None, ctypes.byref(h))
    return st, h


def rcm_batch_plan_launch(plan, stream=None) -> int:
    return load().rcm_batch_plan_launch(plan, _stream(stream))


def rcm_batch_plan_status(plan, stream=None) -> int:
    return load().rcm_batch_plan_status(plan, _stream(stream))


def rcm_batch_plan_destroy(plan) -> int:
    return load().rcm_batch_plan_destroy(plan)


def rcm_stream_status(stream=None) -> int:
    return load().rcm_stream_status(_stream(stream))


def rcm_workspace_bytes(n, nnz) -> int:
    return int(load().rcm_workspace_bytes(int(n), int(nnz)))


def rcm_validate(n, rowptr, colidx, report: rcm_validate_report, stream=None) -> int:
    return load().rcm_validate(int(n), _ptr(rowptr, True, _i32()), _ptr(colidx, True, _i32()), ctypes.byref(report),
                               _stream(stream))


def rcm_bandwidth_profile(n, rowptr, colidx, perm, stream=None):
    """Returns (status, bandwidth, profile)."""
    bw, prof = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().rcm_bandwidth_profile(int(n), _ptr(rowptr, True, _i32()), _ptr(colidx, True, _i32()),
                                      _ptr(perm, True, _i32()), ctypes.byref(bw), ctypes.byref(prof),
                                      _stream(stream))
    return st, int(bw.value), int(prof.value)


def rcm_request_bytes(n, nnz, host_csr=True, host_out=True) -> int:
    return int(load().rcm_request_bytes(int(n), int(nnz), int(bool(host_csr)), int(bool(host_out))))


def rcm_server_create_ex(hbm_budget_bytes, max_inflight, options=None):
    """Returns (status, server handle); options: rcm_server_options or None."""
    h = ctypes.c_void_p()
    st = load().rcm_server_create_ex(int(hbm_budget_bytes), int(max_inflight),
                                     ctypes.byref(options) if options is not None else None, ctypes.byref(h))
    return st, h


def rcm_server_create(hbm_budget_bytes, max_inflight):
    """Returns (status, server handle)."""
    h = ctypes.c_void_p()
    st = load().rcm_server_create(int(hbm_budget_bytes), int(max_inflight), ctypes.byref(h))
    return st, h


def rcm_submit(srv, n, nnz, rowptr, colidx, perm_out):
    """Returns (status, ticket). Buffers: torch tensors (host or CUDA) or raw pointers."""
    t = ctypes.c_uint64(0)
    st = load().rcm_submit(srv, int(n), int(nnz), _ptr(rowptr, None, _i32()), _ptr(colidx, None, _i32()),
                           _ptr(perm_out, None, _i32()), ctypes.byref(t))
    return st, int(t.value)


def rcm_poll(srv, ticket) -> int:
    return load().rcm_poll(srv, int(ticket))


def rcm_wait(srv, ticket) -> int:
    return load().rcm_wait(srv, int(ticket))


def rcm_cancel(srv, ticket) -> int:
    return load().rcm_cancel(srv, int(ticket))


def rcm_server_info(srv):
    st = rcm_server_stats()
    s = load().rcm_server_info(srv, ctypes.byref(st))
    return s, st.as_dict()


def rcm_server_destroy(srv) -> int:
    return load().rcm_server_destroy(srv)


def check(status: int, what: str = "") -> None:
    if status != RCM_OK:
        raise RcmError(status, what)


# ---- conveniences on top of the ABI (allocation of outputs, error raising) ----


def order(rowptr, colidx, options: rcm_options | None = None, with_stats: bool = False, stream=None):
    """RCM permutation (new -> old) of a device CSR pattern as an int32 CUDA tensor."""
    import torch

    n = rowptr.numel() - 1
    perm = torch.empty(max(n, 0), dtype=torch.int32, device=rowptr.device)
    st = rcm_stats() if with_stats else None
    s = rcm_order_ex(n, rowptr, colidx, perm, options, st, stream)
    check(s, "rcm_order_ex")
    if not with_stats:
        check(rcm_stream_status(stream), "rcm_order")
    return (perm, st.as_dict()) if with_stats else perm


def order_batch(goff, rowptr, colidx, stream=None):
    import torch

    G = goff.numel() - 1
    n_total = int(goff[-1].item())
    perm = torch.empty(n_total, dtype=torch.int32, device=rowptr.device)
    check(rcm_order_batch(G, n_total, goff, rowptr, colidx, perm, stream), "rcm_order_batch")
    check(rcm_stream_status(stream), "rcm_order_batch")
    return perm


def validate(rowptr, colidx, stream=None):
    """(ok, report dict): the pattern checked against the library's contract (structure, columns,
    duplicates, symmetry) by rcm_validate."""
    rep = rcm_validate_report()
    st = rcm_validate(rowptr.numel() - 1, rowptr, colidx, rep, stream)
    if st not in (RCM_OK, RCM_ERR_BAD_CSR):
        check(st, "rcm_validate")
    return st == RCM_OK, rep.as_dict()


def bandwidth_profile(rowptr, colidx, perm, stream=None):
    st, bw, prof = rcm_bandwidth_profile(rowptr.numel() - 1, rowptr, colidx, perm, stream)
    check(st, "rcm_bandwidth_profile")
    return bw, prof
