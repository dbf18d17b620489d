"""rcm_order_noalloc: the ordering entry point that allocates no device memory.

It serves callers that must not allocate while they run (memory already handed to their own
allocator, or a memory budget fixed at start-up). Its output must equal rcm_order's on the same
input, exactly (orderings are integer permutations), on two calls in a row, since the calls share
one fixed workspace array that keeps the previous call's contents. This file is collected last.
"""
import numpy as np
import pytest

from paper_1610_08128_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_rcm_order_twice(rcm):
    graphs = [synth.c1_grid2d(), synth.random_graph(5000, 7000, 91), synth.grid((30, 40, 50), seed=92),
              synth.c3_mesh(20000)]
    for g in graphs:
        rp, ci = _dev(g)
        ref = torch.empty(g.n, dtype=torch.int32, device="cuda")
        rcm.check(rcm.rcm_order(g.n, rp, ci, ref), "rcm_order")
        rcm.check(rcm.rcm_stream_status(), "rcm_order")
        for _ in range(2):
            out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
            rcm.check(rcm.rcm_order_noalloc(g.n, rp, ci, out), "rcm_order_noalloc")
            assert torch.equal(out, ref)


def test_noalloc_rejects_sizes_beyond_its_array(rcm):
    g = synth.path(70000)
    rp, ci = _dev(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_noalloc(g.n, rp, ci, out) == rcm.RCM_ERR_TOO_LARGE
    g = synth.random_graph(60000, 600000, 93)  # within the vertex limit, over the entry limit
    rp, ci = _dev(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_noalloc(g.n, rp, ci, out) == rcm.RCM_ERR_TOO_LARGE
