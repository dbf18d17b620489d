"""Serving (continuous batching under an HBM budget): every request's result equals rcm_order on
the same pattern alone (and the oracle), while requests overlap on the GPU; admission, refusal,
cancellation and per-request errors behave as documented in include/rcm.h."""
import numpy as np
import pytest

import oracle
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


def region_bytes(g):
    """Arena bytes of one request with host-resident buffers (staged CSR and output)."""
    from paper_1610_08128_gb300 import rcm as r

    return r.rcm_request_bytes(g.n, g.nnz, True, True)


def mix(count, seed, lo=200, hi=60000):
    sizes, kinds = synth.mix_sizes(count, lo, hi, seed)
    return [synth.batch_graph(int(k), int(s), [seed, i]) for i, (k, s) in enumerate(zip(kinds, sizes))]


def alone(rcm, g):
    rp = torch.from_numpy(g.rowptr.copy()).cuda()
    ci = torch.from_numpy(g.colidx.copy() if g.nnz else np.zeros(1, np.int32)).cuda()
    return rcm.order(rp, ci).cpu().numpy()


def test_served_results_equal_single_calls(rcm):
    graphs = mix(48, 501) + [synth.c1_grid2d(), synth.csr_from_edges(9, [], []), synth.path(1)]
    st, srv = rcm.rcm_server_create(4 << 30, 64)
    rcm.check(st, "create")
    try:
        bufs, tickets = [], []
        for i, g in enumerate(graphs):
            pin = i % 3 != 0
            rp = torch.from_numpy(g.rowptr.copy())
            ci = torch.from_numpy(g.colidx.copy() if g.nnz else np.zeros(1, np.int32))
            out = torch.full((max(g.n, 1),), -1, dtype=torch.int32)
            if pin:
                rp, ci, out = rp.pin_memory(), ci.pin_memory(), out.pin_memory()
            if i % 5 == 0:  # device-resident inputs and output
                rp, ci, out = rp.cuda(), ci.cuda(), out.cuda()
            s, t = rcm.rcm_submit(srv, g.n, g.nnz, rp, ci, out)
            rcm.check(s, "submit")
            bufs.append((rp, ci, out))
            tickets.append(t)
        for g, t, (_, _, out) in zip(graphs, tickets, bufs):
            rcm.check(rcm.rcm_wait(srv, t), "wait")
            got = out.cpu().numpy()[:g.n]
            assert np.array_equal(got, oracle.rcm(g.n, g.rowptr, g.colidx))
        for g, (_, _, out) in list(zip(graphs, bufs))[::7]:
            assert np.array_equal(out.cpu().numpy()[:g.n], alone(rcm, g))
        s, info = rcm.rcm_server_info(srv)
        assert info["completed"] == len(graphs) and info["failed"] == 0
        assert info["max_running"] > 1          # requests really overlapped on the GPU
        assert rcm.rcm_poll(srv, tickets[0]) == rcm.RCM_ERR_UNKNOWN_TICKET  # consumed
    finally:
        rcm.check(rcm.rcm_server_destroy(srv), "destroy")


def test_large_requests_run_on_a_cluster(rcm):
    """Requests of 2^18 vertices or more run the persistent engine launched as one thread-block
    cluster, mixed with small requests on single CTAs; every result equals the oracle and
    rcm_order alone. The random graph (about 10 entries per row) runs the engine with per-level
    bottom-up expansion on its cluster."""
    big = [synth.grid((70, 70, 70), seed=11), synth.grid((600, 600), seed=12),
           synth.batch_graph(2, 300000, [503, 0]), synth.random_graph(280000, 1100000, 504, connected=True)]
    small = mix(12, 503)
    assert len(small[0::3]) == len(big)
    graphs = [g for pair in zip(big, small[0::3]) for g in pair] + small[1::3] + small[2::3]
    o = rcm.rcm_server_options()
    o.cluster_min_vertices = 1 << 18         # every large request here (280k-360k vertices) on a cluster
    st, srv = rcm.rcm_server_create_ex(8 << 30, 32, o)
    rcm.check(st, "create")
    try:
        outs, ins, tickets = [], [], []
        for g in graphs:
            o = torch.empty(g.n, dtype=torch.int32).pin_memory()
            rp, ci = torch.from_numpy(g.rowptr).pin_memory(), torch.from_numpy(g.colidx).pin_memory()
            s, t = rcm.rcm_submit(srv, g.n, g.nnz, rp, ci, o)
            rcm.check(s, "submit")
            ins.append((rp, ci))   # inputs stay valid until the request finishes
            outs.append(o)
            tickets.append(t)
        for g, t, o in zip(graphs, tickets, outs):
            rcm.check(rcm.rcm_wait(srv, t), "wait")
            assert np.array_equal(o.numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))
        for g, o in zip(big, outs[0::2][:len(big)]):
            assert np.array_equal(o.numpy(), alone(rcm, g))
        _, info = rcm.rcm_server_info(srv)
        assert info["failed"] == 0 and info["max_running"] > 1
    finally:
        rcm.check(rcm.rcm_server_destroy(srv), "destroy")


def test_served_rows_stored_in_any_order(rcm):
    """Requests whose rows are stored in shuffled order (the order inside a row is free): small
    requests on single CTAs, stars with rows longer than the per-thread sorters, and a request large
    enough for the cluster engine; each result equals the oracle."""
    star = synth.csr_from_edges(6001, np.zeros(6000, np.int64), np.arange(1, 6001))
    base = mix(16, 505) + [star, synth.csr_from_edges(41, np.full(40, 17, np.int64),
                                                       np.array([v for v in range(41) if v != 17])),
                           synth.grid((70, 70, 70), seed=13)]
    graphs = [synth.shuffle_rows(g, [506, i]) for i, g in enumerate(base)]
    st, srv = rcm.rcm_server_create(8 << 30, 32)
    rcm.check(st, "create")
    try:
        keep, tickets = [], []
        for g in graphs:
            o = torch.empty(g.n, dtype=torch.int32).pin_memory()
            rp, ci = torch.from_numpy(g.rowptr).pin_memory(), torch.from_numpy(g.colidx).pin_memory()
            s, t = rcm.rcm_submit(srv, g.n, g.nnz, rp, ci, o)
            rcm.check(s, "submit")
            keep.append((rp, ci, o))
            tickets.append(t)
        for g, t, (_, _, o) in zip(graphs, tickets, keep):
            rcm.check(rcm.rcm_wait(srv, t), "wait")
            assert np.array_equal(o.numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))
        _, info = rcm.rcm_server_info(srv)
        assert info["failed"] == 0
    finally:
        rcm.check(rcm.rcm_server_destroy(srv), "destroy")


def test_admission_under_a_small_budget(rcm):
    graphs = mix(12, 502, lo=20000, hi=40000)
    need = max(region_bytes(g) for g in graphs)
    st, srv = rcm.rcm_server_create(2 * need, 16)     # room for about two requests at a time
    rcm.check(st, "create")
    try:
        big = synth.grid((300, 300), seed=1)
        out = torch.empty(big.n, dtype=torch.int32)
        s, _ = rcm.rcm_submit(srv, big.n, big.nnz, torch.from_numpy(big.rowptr), torch.from_numpy(big.colidx), out)
        assert s == rcm.RCM_ERR_TOO_LARGE
        outs, tickets = [], []
        for g in graphs:
            o = torch.empty(g.n, dtype=torch.int32)
            s, t = rcm.rcm_submit(srv, g.n, g.nnz, torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx), o)
            rcm.check(s, "submit")
            outs.append(o)
            tickets.append(t)
        for g, t, o in zip(graphs, tickets, outs):
            rcm.check(rcm.rcm_wait(srv, t), "wait")
            assert np.array_equal(o.numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))
        _, info = rcm.rcm_server_info(srv)
        assert info["arena_peak_bytes"] <= info["arena_bytes"]
    finally:
        rcm.rcm_server_destroy(srv)


def test_cancel_and_failed_requests(rcm):
    g = synth.grid((150, 150), seed=3)
    st, srv = rcm.rcm_server_create(region_bytes(g), 1)  # one request at a time
    rcm.check(st, "create")
    try:
        rp, ci = torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx)
        outs = [torch.empty(g.n, dtype=torch.int32) for _ in range(4)]
        tickets = [rcm.rcm_submit(srv, g.n, g.nnz, rp, ci, o)[1] for o in outs]
        # the last one cannot have started yet: withdraw it
        assert rcm.rcm_cancel(srv, tickets[-1]) == rcm.RCM_OK
        assert rcm.rcm_poll(srv, tickets[-1]) == rcm.RCM_ERR_UNKNOWN_TICKET
        # a malformed request fails alone
        bad = g.colidx.copy()
        bad[5] = g.n + 3
        ob = torch.empty(g.n, dtype=torch.int32)
        s, tb = rcm.rcm_submit(srv, g.n, g.nnz, rp, torch.from_numpy(bad), ob)
        rcm.check(s, "submit")
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        for t, o in zip(tickets[:-1], outs[:-1]):
            rcm.check(rcm.rcm_wait(srv, t), "wait")
            assert np.array_equal(o.numpy(), want)
        assert rcm.rcm_wait(srv, tb) == rcm.RCM_ERR_BAD_CSR
        _, info = rcm.rcm_server_info(srv)
        assert info["failed"] == 1 and info["cancelled"] == 1 and info["max_running"] == 1
    finally:
        rcm.rcm_server_destroy(srv)


def test_stream_error_fails_outstanding_requests(rcm):
    """Failure handling without a device fault: a test hook makes the worker act as if a running
    request's stream reported an error once two requests have completed. Every outstanding request
    then finishes with RCM_ERR_CUDA (no waiter blocks), completed ones keep their correct results,
    later submissions are refused, and destroy returns."""
    graphs = [synth.grid((400, 400), seed=20 + i) for i in range(16)]
    o = rcm.rcm_server_options()
    o.debug_fail_after = 2
    st, srv = rcm.rcm_server_create_ex(4 << 30, 2, o)
    rcm.check(st, "create")
    try:
        outs, tickets = [], []
        for g in graphs:
            out = torch.empty(g.n, dtype=torch.int32)
            s, t = rcm.rcm_submit(srv, g.n, g.nnz, torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx), out)
            rcm.check(s, "submit")
            outs.append(out)
            tickets.append(t)
        statuses = [rcm.rcm_wait(srv, t) for t in tickets]
        assert set(statuses) <= {rcm.RCM_OK, rcm.RCM_ERR_CUDA}
        assert statuses.count(rcm.RCM_OK) >= 2 and rcm.RCM_ERR_CUDA in statuses
        for g, s_, out in zip(graphs, statuses, outs):
            if s_ == rcm.RCM_OK:
                assert np.array_equal(out.numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))
        g = graphs[0]
        s, _ = rcm.rcm_submit(srv, g.n, g.nnz, torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx),
                              torch.empty(g.n, dtype=torch.int32))
        assert s == rcm.RCM_ERR_CUDA
        _, info = rcm.rcm_server_info(srv)
        assert info["failed"] == statuses.count(rcm.RCM_ERR_CUDA)
    finally:
        assert rcm.rcm_server_destroy(srv) == rcm.RCM_OK


def test_destroy_with_waiting_requests(rcm):
    g = synth.grid((120, 120), seed=4)
    st, srv = rcm.rcm_server_create(region_bytes(g), 1)
    rcm.check(st, "create")
    outs = [torch.empty(g.n, dtype=torch.int32) for _ in range(5)]
    for o in outs:
        rcm.check(rcm.rcm_submit(srv, g.n, g.nnz, torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx), o)[0], "s")
    rcm.check(rcm.rcm_server_destroy(srv), "destroy")   # running ones finish, waiting ones are dropped
