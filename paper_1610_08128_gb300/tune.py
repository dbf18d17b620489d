"""Autotuner for the launch shapes of the ordering kernels.

Every tunable is a plain option of the C ABI and changes speed only: the batched executor's CTA
width and row-sort split (rcm_batch_options), and the one-graph executor, CTA width,
frontier-switch threshold, sweep mode (level by level or asynchronous), expansion mode (top-down
or chosen per level) and the top-down/bottom-up switch threshold (rcm_options). The tuner times each candidate on the caller's own data
through the C ABI (CUDA events, median of a few runs after one warm-up), checks that every
candidate returns the same permutation as the first one, and returns the fastest. Choices can be
cached per device and size class in a JSON file.
"""
from __future__ import annotations

import json
import os
import statistics

from . import rcm

BATCH_CANDIDATES = [
    {"block_threads": t, "row_sort_split": s} for t in (128, 256, 512) for s in (8, 32)
]

SINGLE_CANDIDATES = [
    {"executor": 1, "async_sweeps": a, "narrow_threshold": t}
    for a in (1, -1) for t in (128, 256, 512, 1024, 2048)
] + [
    {"executor": 1, "expand_mode": 1, "narrow_threshold": t, "l2_persist": l2} for t in (512, 1024) for l2 in (-1, 1)
] + [
    {"executor": 1, "narrow_threshold": t, "fused_sweeps": 1} for t in (128, 512)
] + [
    {"executor": 1, "narrow_threshold": 512, "fused_sweeps": 1, "components_first": 1}
] + [
    {"executor": 1, "expand_mode": 1, "narrow_threshold": 512, "l2_persist": 1, "mid_cluster": k} for k in (8, 16)
] + [
    {"executor": 1, "expand_mode": 3, "bottom_up_divisor": dv, "narrow_threshold": t}
    for dv in (4, 16, 64) for t in (512, 1024)
] + [
    {"executor": 2, "block_threads": 128},
    {"executor": 2, "block_threads": 256},
    {"executor": 2, "block_threads": 512},
]

CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune")


def _time_ms(fn, torch, repeats):
    stream = torch.cuda.current_stream()
    fn(stream)  # warm-up
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune_batch(G, n_total, goff, rowptr, colidx, perm_out, candidates=None, repeats=3):
    """Times rcm_order_batch_ex under each candidate on the given (device) batch. Returns
    (best options dict, [(options dict, ms), ...]). Raises if candidates disagree."""
    import torch

    ref, table = None, []
    for cand in candidates or BATCH_CANDIDATES:
        o = rcm.rcm_batch_options()
        for k, v in cand.items():
            setattr(o, k, v)

        def run(stream, o=o):
            rcm.check(rcm.rcm_order_batch_ex(G, n_total, goff, rowptr, colidx, perm_out, o, stream), "batch")
            rcm.check(rcm.rcm_stream_status(stream), "batch")

        ms = _time_ms(run, torch, repeats)
        got = perm_out.clone()
        if ref is None:
            ref = got
        elif not torch.equal(got, ref):
            raise RuntimeError(f"batch candidate {cand} changed the result")
        table.append((dict(cand), ms))
    best = min(table, key=lambda x: x[1])[0]
    return best, table


def tune_single(n, rowptr, colidx, perm_out, nnz=0, candidates=None, repeats=5):
    """Times rcm_order_ex under each candidate on one (device) graph; candidates the graph does not
    admit (the shared-memory executor above its size limit) are skipped. Returns (best, table)."""
    import torch

    ref, table = None, []
    for cand in candidates or SINGLE_CANDIDATES:
        o = rcm.rcm_options()
        o.nnz = nnz
        for k, v in cand.items():
            setattr(o, k, v)
        st = rcm.rcm_order_ex(n, rowptr, colidx, perm_out, o, None)
        if st == rcm.RCM_ERR_TOO_LARGE:
            continue
        rcm.check(st, "order")

        def run(stream, o=o):
            rcm.check(rcm.rcm_order_ex(n, rowptr, colidx, perm_out, o, None, stream), "order")
            rcm.check(rcm.rcm_stream_status(stream), "order")

        ms = _time_ms(run, torch, repeats)
        got = perm_out.clone()
        if ref is None:
            ref = got
        elif not torch.equal(got, ref):
            raise RuntimeError(f"candidate {cand} changed the result")
        table.append((dict(cand), ms))
    best = min(table, key=lambda x: x[1])[0]
    return best, table


def size_class(n: int) -> str:
    """Power-of-four bucket of a vertex count (choices transfer within a bucket)."""
    c = 0
    while (1 << (2 * (c + 1))) <= max(int(n), 1):
        c += 1
    return f"n<4^{c + 1}"


def _cache_path():
    import torch

    name = torch.cuda.get_device_name().replace(" ", "_").replace("/", "_")
    return os.path.join(CACHE_DIR, f"{name}.json")


def load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_choice(key: str, options: dict) -> None:
    data = load_cache()
    data[key] = options
    os.makedirs(CACHE_DIR, exist_ok=True)
    with open(_cache_path(), "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
