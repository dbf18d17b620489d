"""rcm_order_noalloc: the ordering entry point that allocates no device memory.

It serves callers that must not allocate while they run: an application whose memory framework
has already reserved the device memory for its own caching allocator, or a solver loop with a
memory budget fixed at start-up, where an allocation could fail or stall the device. Its output
must equal the oracle's and rcm_order's on the same input, exactly (orderings are integer
permutations), on two calls in a row, since the calls share one fixed workspace array that keeps
the previous call's contents. After the first call on a device (its one-time set-up), a call must
leave the device's free memory, the default memory pool and torch's caching allocator as they were.
This file is collected last, so a run that stops at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1610_08128_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_N = 1 << 16          # the documented limits of the fixed workspace
MAX_NNZ = 1 << 20


@pytest.fixture(scope="module")
def rcm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_08128_gb300 import build, rcm

    build.build()
    rcm.load()
    return rcm


def _dev(g):
    rp = torch.from_numpy(g.rowptr.copy()).cuda()
    ci = torch.from_numpy(g.colidx.copy() if g.nnz else np.zeros(1, np.int32)).cuda()
    return rp, ci


def _check_twice(rcm, g, with_rcm_order=True):
    rp, ci = _dev(g)
    want = oracle.rcm(g.n, g.rowptr, g.colidx)
    if with_rcm_order:
        ref = torch.empty(g.n, dtype=torch.int32, device="cuda")
        rcm.check(rcm.rcm_order(g.n, rp, ci, ref), "rcm_order")
        rcm.check(rcm.rcm_stream_status(), "rcm_order")
        assert np.array_equal(ref.cpu().numpy(), want)
    for _ in range(2):
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        rcm.check(rcm.rcm_order_noalloc(g.n, rp, ci, out), "rcm_order_noalloc")
        assert np.array_equal(out.cpu().numpy(), want)


def test_noalloc_matches_the_oracle_and_rcm_order_twice(rcm):
    graphs = [synth.c1_grid2d(), synth.random_graph(5000, 7000, 91), synth.grid((30, 40, 50), seed=92),
              synth.c3_mesh(20000), synth.csr_from_edges(4000, np.zeros(3999, np.int64), np.arange(1, 4000))]
    graphs += [synth.shuffle_rows(g, [94, i]) for i, g in enumerate(graphs)]   # rows stored in any order
    for g in graphs:
        _check_twice(rcm, g)


def test_noalloc_at_its_size_limits(rcm):
    """Patterns at the documented maximum: 65,536 vertices with exactly 1,048,576 stored entries
    (16 per row, rows shuffled), and a random pattern just below the entry limit."""
    g = synth.shuffle_rows(synth.circulant(MAX_N, range(1, 9), seed=95), 96)
    assert g.n == MAX_N and g.nnz == MAX_NNZ
    _check_twice(rcm, g, with_rcm_order=False)
    g = synth.random_graph(MAX_N, 520000, 97)
    assert g.n == MAX_N and MAX_NNZ - 16000 < g.nnz <= MAX_NNZ
    _check_twice(rcm, g, with_rcm_order=False)


def test_noalloc_rejects_sizes_beyond_its_array(rcm):
    for g in (synth.path(MAX_N + 1), synth.path(70000)):
        rp, ci = _dev(g)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        assert rcm.rcm_order_noalloc(g.n, rp, ci, out) == rcm.RCM_ERR_TOO_LARGE
    # within the vertex limit, one entry over the entry limit: a diagonal entry on one row
    g = synth.circulant(MAX_N, range(1, 9))
    g = synth.csr_from_edges(MAX_N, *_edges(g), diagonal=np.array([5]))
    assert g.n == MAX_N and g.nnz == MAX_NNZ + 1
    rp, ci = _dev(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_noalloc(g.n, rp, ci, out) == rcm.RCM_ERR_TOO_LARGE
    g = synth.random_graph(60000, 600000, 93)  # within the vertex limit, far over the entry limit
    rp, ci = _dev(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_noalloc(g.n, rp, ci, out) == rcm.RCM_ERR_TOO_LARGE


def _edges(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr.astype(np.int64)))
    return rows, g.colidx.astype(np.int64)


def _device_memory():
    """Free device memory, and the reserved / used bytes of the device's default memory pool (the
    pool the allocating entry points take their workspace from), through the CUDA driver."""
    cu = ctypes.CDLL("libcuda.so.1")
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    reserved, used = ctypes.c_uint64(), ctypes.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, 5, ctypes.byref(reserved)) == 0   # RESERVED_MEM_CURRENT
    assert cu.cuMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0       # USED_MEM_CURRENT
    return {"free": free.value, "pool_reserved": reserved.value, "pool_used": used.value,
            "torch_reserved": torch.cuda.memory_reserved()}


def test_noalloc_calls_after_the_first_allocate_nothing(rcm):
    """After one call (the per-device set-up, which may load device code), calls on both executors
    -- the shared-memory CTA for at most 4,608 vertices and the persistent grid above -- leave the
    device's memory as they found it."""
    small, large = synth.c1_grid2d(), synth.shuffle_rows(synth.grid((40, 40, 40), seed=98), 99)
    bufs = []
    for g in (small, large):
        rp, ci = _dev(g)
        bufs.append((g, rp, ci, torch.empty(g.n, dtype=torch.int32, device="cuda")))
    g, rp, ci, out = bufs[0]
    rcm.check(rcm.rcm_order_noalloc(g.n, rp, ci, out), "set-up call")
    torch.cuda.synchronize()
    before = _device_memory()
    for _ in range(2):
        for g, rp, ci, out in bufs:
            rcm.check(rcm.rcm_order_noalloc(g.n, rp, ci, out), "rcm_order_noalloc")
    torch.cuda.synchronize()
    after = _device_memory()
    assert after == before
    for g, _, _, out in bufs:
        assert np.array_equal(out.cpu().numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))
