"""GPU parity: the CUDA path (through the C ABI) against the serial CPU oracle, bit for bit.

Orderings are integer permutations, so the only tolerance is exact equality. Inputs are the seeded
generators' (shapes of the paper's workloads) plus random small graphs, special cases and the
variant/launch-shape invariance the library promises (no option changes the result).
"""
import numpy as np
import pytest

import oracle
from paper_1610_08128_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_08128_gb300 import build, rcm

    build.build()
    return rcm.load()


def rcm_mod():
    from paper_1610_08128_gb300 import rcm

    return rcm


def to_dev(g):
    rp = torch.from_numpy(np.ascontiguousarray(g.rowptr, dtype=np.int32)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.colidx if g.nnz else np.zeros(1, np.int32), dtype=np.int32)).cuda()
    return rp, ci


def gpu_perm(g, opts=None, with_stats=False):
    rcm = rcm_mod()
    rp, ci = to_dev(g)
    o = None
    if opts:
        o = rcm.rcm_options()
        for k, v in opts.items():
            setattr(o, k, v)
    out = rcm.order(rp, ci, options=o, with_stats=with_stats)
    if with_stats:
        return out[0].cpu().numpy(), out[1]
    return out.cpu().numpy()


def assert_parity(g, opts=None):
    want = oracle.rcm(g.n, g.rowptr, g.colidx)
    got = gpu_perm(g, opts)
    assert got.shape == want.shape
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"mismatch at {len(bad)} positions, first {bad[:8]}: got {got[bad[:8]]} want {want[bad[:8]]}")


def small_graphs(count, nmax, seed):
    rng = synth.rng_for(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(1, nmax + 1))
        m = int(rng.integers(0, 3 * n + 1))
        out.append(synth.random_graph(n, m, [seed, i], connected=bool(i % 2), diagonal=bool(i % 3 == 0)))
    return out


# ---------------------------------------------------------------------------------------------


def test_c1_grid64_parity():
    for off in range(4):
        assert_parity(synth.c1_grid2d(seed_offset=off))


def test_random_graphs_fuzz():
    for g in small_graphs(300, 400, 101):
        assert_parity(g)


def test_grids_2d_3d():
    for dims, seed in [((1, 1), 1), ((1, 7), 2), ((2, 2), 3), ((13, 29), 4), ((100, 37), 5), ((5, 6, 7), 6),
                       ((16, 16, 16), 7), ((40, 3, 22), 8), ((64, 64, 8), 9)]:
        assert_parity(synth.grid(dims, seed=seed))


def test_natural_ids_and_paths():
    for dims in [(10, 10), (3, 50), (4, 5, 6)]:
        assert_parity(synth.grid(dims))
    for n in (1, 2, 3, 50, 3000):
        assert_parity(synth.path(n))
        assert_parity(synth.path(n, seed=n))


def test_trees_and_stars():
    for i in range(20):
        assert_parity(synth.random_tree(1 + 37 * i, [5, i]))
    for leaves in (1, 2, 40, 5000, 20000):  # a row longer than the shared-memory sorter
        g = synth.csr_from_edges(leaves + 1, np.zeros(leaves, np.int64), np.arange(1, leaves + 1))
        assert_parity(g)


def test_special_cases():
    rcm = rcm_mod()
    # n = 0
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    pm = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order(0, rp, ci, pm) == rcm.RCM_OK
    # isolated vertices only, a self-loop only, many components, diagonal everywhere
    assert_parity(synth.csr_from_edges(1, [], []))
    assert_parity(synth.csr_from_edges(1, [], [], diagonal=True))
    assert_parity(synth.csr_from_edges(1000, [], []))
    assert_parity(synth.csr_from_edges(300, [], [], diagonal=True))
    assert_parity(synth.random_graph(2000, 700, 7))          # hundreds of components
    assert_parity(synth.random_graph(2000, 3000, 8, diagonal=np.arange(0, 2000, 7)))


def test_meshes():
    assert_parity(synth.c3_mesh(20000))
    assert_parity(synth.c3_mesh(20000, seed_offset=1))
    assert_parity(synth.c3_mesh(8000, stitch=False))          # raw kNN(2): thousands of components
    assert_parity(synth.knn_mesh(30000, 3, 11))


def test_components_concurrent_with_a_grid_sized_one():
    """One component large enough for the whole grid plus thousands of small ones (run one per
    CTA), and the same with isolated vertices: labels still follow the start rule exactly."""
    big = synth.grid((600, 520), seed=61)                       # 312,000 vertices, one component
    small = synth.random_graph(40000, 30000, 62)                # thousands of small components
    g = synth.concat([big, small])
    merged = synth.Csr(g.n, g.rowptr, g.colidx)
    p = synth.random_permutation(g.n, 63)
    assert_parity(synth.permute(merged, p))
    g2 = synth.concat([small, synth.csr_from_edges(500, [], []), big])
    assert_parity(synth.permute(synth.Csr(g2.n, g2.rowptr, g2.colidx), synth.random_permutation(g2.n, 64)))


def tiny_mix(seed, big=(60, 50), count=300):
    """One mid-sized grid plus a few hundred components of 2 to 40 vertices (paths, stars whose
    centre row is longer than the padded row, cycles, random connected graphs, small grids;
    sizes on both sides of the one-thread limit of 32) and isolated vertices; ids permuted and
    rows stored in shuffled order."""
    rng = synth.rng_for(seed)
    parts = [synth.grid(big, seed=[seed, 0])] if big else []
    for i in range(count):
        z = int(rng.integers(2, 41))
        kind = i % 5
        if kind == 0:
            g = synth.path(z, seed=[seed, i])
        elif kind == 1:
            g = synth.csr_from_edges(z, np.zeros(z - 1, np.int64), np.arange(1, z))
        elif kind == 2:
            g = synth.circulant(z, [1], seed=[seed, i]) if z >= 3 else synth.path(z)
        elif kind == 3:
            g = synth.random_graph(z, int(rng.integers(z - 1, 3 * z)), [seed, i], connected=True)
        else:
            a = max(1, int(np.sqrt(z)))
            g = synth.grid((a, max(1, z // a)), seed=[seed, i])
        parts.append(g)
    parts.append(synth.csr_from_edges(25, [], []))
    b = synth.concat(parts)
    g = synth.Csr(b.n, b.rowptr, b.colidx)
    return synth.shuffle_rows(synth.permute(g, synth.random_permutation(g.n, [seed, 1])), [seed, 2])


def test_tiny_components_one_per_thread():
    """Components of at most 32 vertices are ordered by one thread each (serial sweeps and
    numbering from the sorted rows); larger ones by the CTA or grid engines. Every executor and
    sweep mode gives the oracle's order, and the statistics count the same sweeps."""
    for seed in (171, 172):
        g = tiny_mix(seed)
        want, ost = oracle.rcm(g.n, g.rowptr, g.colidx, with_stats=True)
        for opts in ({}, {"executor": 1}, {"executor": 1, "fused_sweeps": -1}, {"executor": 1, "fused_sweeps": 2},
                     {"executor": 1, "narrow_threshold": -1}):
            got, st = gpu_perm(g, opts, with_stats=True)
            assert np.array_equal(got, want), opts
            # isolated vertices are numbered without sweeps; Alg. 2 on one vertex takes two
            sweeps = ost["sweeps"] - 2 * ost["isolated"]
            assert st["components"] == ost["components"] and st["sweeps"] == sweeps, opts
            assert st["max_ecc"] == ost["max_ecc"], opts
            if opts.get("fused_sweeps") == -1:
                assert st["traversals"] == sweeps + ost["components"] - ost["isolated"], opts
            else:
                assert st["traversals"] == sweeps, opts
    small = tiny_mix(173, big=None, count=150)       # small components only (the shared-memory CTA)
    assert small.n <= 4608
    assert_parity(small)
    assert_parity(small, {"executor": 2, "block_threads": 64})


def test_warp_levels_expanding_past_the_frontier_cache():
    """A one-vertex level whose hub expands to more vertices than the shared frontier cache holds
    (2,048): the warp-0 run hands over a level kept in global memory. On the shared-memory CTA (a
    star of 3,000 leaves alone) and in the component kernel (the same star beside a grid)."""
    star = synth.csr_from_edges(3001, np.zeros(3000, np.int64), np.arange(1, 3001))
    g = synth.permute(star, synth.random_permutation(star.n, 201))
    assert_parity(g, {"executor": 2, "block_threads": 64})
    assert_parity(g, {"executor": 2, "block_threads": 256})
    b = synth.concat([star, synth.grid((60, 60), seed=202)])
    mixed = synth.permute(synth.Csr(b.n, b.rowptr, b.colidx), synth.random_permutation(b.n, 203))
    assert_parity(mixed)
    assert_parity(mixed, {"executor": 1, "components_first": 1})
    assert_parity(mixed, {"executor": 1, "fused_sweeps": -1})


def test_tiny_components_in_the_batch():
    """The batched engine orders each graph's tiny components one per thread."""
    rcm = rcm_mod()
    graphs = [tiny_mix(181), tiny_mix(182, big=(9, 7)), tiny_mix(183, big=None), synth.knn_mesh(19000, 3, 184)]
    b = synth.concat(graphs)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    want = [oracle.rcm(g.n, g.rowptr, g.colidx) for g in graphs]
    for threads in (128, 256, 512):
        o = rcm.rcm_batch_options()
        o.block_threads = threads
        perm = torch.full((b.n,), -1, dtype=torch.int32, device="cuda")
        rcm.check(rcm.rcm_order_batch_ex(len(graphs), b.n, goff, rp, ci, perm, o), "batch_ex")
        rcm.check(rcm.rcm_stream_status(), "batch_ex")
        host = perm.cpu().numpy()
        for gi in range(len(graphs)):
            assert np.array_equal(host[b.goff[gi]:b.goff[gi + 1]], want[gi]), (threads, gi)


def golden(name):
    """A pattern from tests/golden (explicit stored rows, or an edge list) and its expected perm."""
    import os

    d = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split(":", 1)
                d.setdefault(k.strip(), []).extend(int(x) for x in v.split())
    n = d["n"][0]
    if "rowptr" in d:
        g = synth.Csr(n, np.array(d["rowptr"], np.int32), np.array(d["colidx"], np.int32))
    else:
        e = np.array(d["edges"], np.int64).reshape(-1, 2)
        g = synth.csr_from_edges(n, e[:, 0], e[:, 1])
    return g, np.array(d["perm"], np.int32)


def star(leaves, centre=0):
    others = np.array([v for v in range(leaves + 1) if v != centre], np.int64)
    return synth.csr_from_edges(leaves + 1, np.full(leaves, centre, np.int64), others)


def shuffled_graphs():
    """Patterns whose rows are stored in a seeded random order (the order inside a row is free):
    grids, meshes with and without components, random graphs, stars whose centre row is longer
    than the per-thread sorters (8 and 32 entries) and than the shared-memory sorter, a power-law
    graph with hubs of thousands of entries, and random small graphs."""
    base = [synth.c1_grid2d(), synth.grid((20, 30, 11), seed=3), synth.c3_mesh(20000),
            synth.c3_mesh(8000, stitch=False), synth.knn_mesh(30000, 3, 11), synth.random_graph(3000, 4000, 9),
            star(40, 17), star(5000, 2500), star(20000), synth.power_law(60000, 10, 2.5, 112),
            golden("broom78.txt")[0]]
    base += small_graphs(60, 400, 111)
    return [synth.shuffle_rows(g, [4242, i]) for i, g in enumerate(base)]


def test_rows_stored_in_any_order():
    """Exact mode on rows stored in shuffled order: the row sort (register network for rows of at
    most 8 entries, insertion sort up to 32, a whole CTA beyond) must recover the (degree, id) order
    of Alg. 1 from any stored order, on the persistent grid and the shared-memory CTA."""
    for g in shuffled_graphs():
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        assert_parity(g)
        assert np.array_equal(gpu_perm(g, {"executor": 1}), want)
        assert np.array_equal(gpu_perm(g, {"executor": 1, "narrow_threshold": -1}), want)
        if g.n <= 4608:
            assert np.array_equal(gpu_perm(g, {"executor": 2}), want)


def test_rows_stored_in_any_order_every_expansion():
    """The same on low-diameter shuffled graphs with every expansion mode and asynchronous sweeps."""
    graphs = [synth.shuffle_rows(g, [4243, i]) for i, g in
              enumerate([synth.random_graph(200000, 900000, 113, connected=True), synth.power_law(200000, 12, 2.3, 114)])]
    for g in graphs:
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        for opts in ({"expand_mode": 1}, {"expand_mode": 2}, {"expand_mode": 3}, {"async_sweeps": 1},
                     {"expand_mode": 2, "narrow_threshold": -1, "fused_sweeps": -1}):
            assert np.array_equal(gpu_perm(g, opts), want), opts


def test_power_law_hubs_on_every_executor():
    """Scale-free patterns whose hub rows hold hundreds to thousands of entries, read by whole warps
    in every expansion (top-down claims and ownership, bottom-up scans, levels-only sweeps, the
    union-find of the component pass): the persistent grid in every expansion mode, CTA 0 alone,
    the asynchronous sweeps, and the shared-memory CTA for a small one."""
    graphs = [synth.power_law(200000, 10, 2.5, 121), synth.power_law(300000, 6, 2.1, 122)]
    for g in graphs:
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        for opts in (None, {"executor": 1, "narrow_threshold": -1}, {"expand_mode": 1}, {"expand_mode": 2},
                     {"expand_mode": 3, "bottom_up_divisor": 64}, {"narrow_threshold": 1 << 30},
                     {"async_sweeps": 1}, {"fused_sweeps": -1}, {"fused_sweeps": 1}):
            assert np.array_equal(gpu_perm(g, opts), want), opts
    for i in range(6):
        g = synth.power_law(4000, 8, 2.2, [123, i])
        assert np.diff(g.rowptr).max() > 100
        assert_parity(g, {"executor": 2})
        assert_parity(g, {"executor": 1, "narrow_threshold": -1})


def test_power_law_batch():
    """Scale-free graphs in the batched engine (one CTA per graph, long rows read by warps)."""
    rcm = rcm_mod()
    graphs = [synth.power_law(int(n), 8, 2.3, [124, i]) for i, n in enumerate([300, 2000, 9000, 30000, 60000])]
    graphs += [synth.shuffle_rows(g, [125, i]) for i, g in enumerate(graphs)]
    b = synth.concat(graphs)
    perm = rcm.order_batch(torch.from_numpy(b.goff).cuda(), torch.from_numpy(b.rowptr).cuda(),
                           torch.from_numpy(b.colidx).cuda()).cpu().numpy()
    for gi, g in enumerate(graphs):
        assert np.array_equal(perm[b.goff[gi]:b.goff[gi + 1]], oracle.rcm(g.n, g.rowptr, g.colidx)), gi


@pytest.mark.slow
def test_power_law_1m_full_size():
    """A 1,000,000-vertex scale-free graph (hubs of about 7,000 entries), default launch."""
    g = synth.power_law(1_000_000, 10, 2.5, 5)
    assert np.diff(g.rowptr).max() > 5000
    assert_parity(g)


@pytest.mark.parametrize("name", ["star41_shuffled.txt", "star41_reversed.txt", "broom78.txt"])
def test_wide_row_fixtures(name):
    """The hand-worked wide-row fixtures (rows of more than 32 neighbours, stored out of order)."""
    g, perm = golden(name)
    for opts in (None, {"executor": 1}, {"executor": 2}, {"executor": 1, "narrow_threshold": -1}):
        assert np.array_equal(gpu_perm(g, opts), perm), opts


def test_batch_rows_stored_in_any_order():
    """The batched engine on shuffled rows, with every row-sort split and CTA width."""
    rcm = rcm_mod()
    graphs = [g for g in shuffled_graphs() if g.n <= 30000]
    b = synth.concat(graphs)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    want = [oracle.rcm(g.n, g.rowptr, g.colidx) for g in graphs]
    for threads in (128, 256, 512):
        for split in (4, 8, 32):
            o = rcm.rcm_batch_options()
            o.block_threads, o.row_sort_split = threads, split
            perm = torch.full((b.n,), -1, dtype=torch.int32, device="cuda")
            rcm.check(rcm.rcm_order_batch_ex(len(graphs), b.n, goff, rp, ci, perm, o), "batch_ex")
            rcm.check(rcm.rcm_stream_status(), "batch_ex")
            host = perm.cpu().numpy()
            for gi in range(len(graphs)):
                assert np.array_equal(host[b.goff[gi]:b.goff[gi + 1]], want[gi]), (threads, split, gi)


OPTION_SETS = [
    {"narrow_threshold": -1},            # whole grid for every level
    {"narrow_threshold": 1 << 30},       # CTA 0 for every level
    {"narrow_threshold": 7},
    {"grid_blocks": 1},
    {"grid_blocks": 3, "narrow_threshold": -1},
    {"block_threads": 256},
    {"block_threads": 512, "narrow_threshold": 100},
    {"fused_sweeps": -1},
    {"fused_sweeps": -1, "narrow_threshold": -1},
    {"cluster": 1},                      # one thread-block cluster, the largest the device allows
    {"cluster": 1, "grid_blocks": 8},
    {"cluster": 1, "grid_blocks": 2, "narrow_threshold": -1},
    {"executor": 1},                     # persistent grid even for graphs the shared-memory CTA takes
    {"executor": 1, "async_sweeps": 1},  # levels-only sweeps through the asynchronous work queue
    {"async_sweeps": 1, "grid_blocks": 3},
    {"async_sweeps": 1, "narrow_threshold": -1},
    {"async_sweeps": 1, "cluster": 1, "grid_blocks": 4},
    {"async_sweeps": -1, "executor": 1},
    {"executor": 1, "async_sweeps": 1, "debug_async_slots": 16},   # queue runs full: level-by-level fallback
    {"expand_mode": 2, "narrow_threshold": -1},                    # bottom-up on every level
    {"expand_mode": 2, "grid_blocks": 3, "narrow_threshold": -1, "fused_sweeps": -1},
    {"expand_mode": 2, "executor": 1},                             # bottom-up on the whole-grid levels
    {"expand_mode": 1, "narrow_threshold": -1},                    # top-down only
    {"expand_mode": 3, "narrow_threshold": -1},                    # chosen per level
    {"expand_mode": 3, "bottom_up_divisor": 1000000},              # per level, switching early
    {"l2_persist": 1, "executor": 1},                              # claims and stamps persisting in L2
    {"l2_persist": 1, "narrow_threshold": -1, "fused_sweeps": 1},
    {"fused_sweeps": 2, "executor": 1, "grid_blocks": 8},          # every sweep labelled on a small grid
    {"mid_cluster": 4, "executor": 1},                             # middle tier on a cluster of 4
    {"mid_cluster": 8, "executor": 1, "narrow_threshold": 32},     # ... of 8, entered early
    {"mid_cluster": 2, "executor": 1, "narrow_threshold": -1},     # no CTA-0 levels: grid and middle tier only
    {"mid_cluster": 8, "executor": 1, "l2_persist": 1},
    {"mid_cluster": 4, "expand_mode": 3, "bottom_up_divisor": 1000000},  # with bottom-up grid levels
    {"mid_cluster": 16, "executor": 1, "fused_sweeps": 1},
    {"mid_cluster": 8, "executor": 1, "mid_threshold": 8192},      # a tier far wider than the cluster
    {"mid_cluster": 4, "executor": 1, "mid_threshold": 600},       # a tier of one CTA-0 threshold's width
    {"mid_cluster": 4, "executor": 1, "mid_threshold": 100},       # bound below the CTA-0 threshold: tier unused
    {"components_first": 1, "executor": 1},                        # component table before any sweep
    {"components_first": 1, "executor": 1, "narrow_threshold": -1, "fused_sweeps": 2},
]


@pytest.mark.parametrize("opts", OPTION_SETS, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_options_do_not_change_the_result(opts):
    graphs = [synth.c1_grid2d(), synth.grid((20, 30, 11), seed=3), synth.c3_mesh(6000),
              synth.random_graph(3000, 4000, 9)] + small_graphs(25, 200, 102)
    for g in graphs:
        assert_parity(g, opts)


def test_async_sweeps_on_large_graphs():
    """Levels-only sweeps through the asynchronous work queue and level by level give the oracle's
    order and the same sweep counts on large graphs: a 3D grid, a high-diameter 2D grid, a mesh
    with components, a deep tree and a path. A queue that runs full falls back to level by level
    with the same result; the asynchronous engine exists for 512-thread CTAs only."""
    graphs = [synth.grid((80, 80, 80), seed=71), synth.grid((700, 700), seed=72), synth.c3_mesh(300000),
              synth.random_tree(200000, 73), synth.path(150000, seed=74)]
    keys = ("components", "sweeps", "traversals", "levels", "max_ecc", "isolated")
    for g in graphs:
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        a, sa = gpu_perm(g, {"async_sweeps": 1}, with_stats=True)
        b, sb = gpu_perm(g, {"async_sweeps": -1}, with_stats=True)
        assert np.array_equal(a, want)
        assert np.array_equal(b, want)
        assert {k: sa[k] for k in keys} == {k: sb[k] for k in keys}
    g = graphs[0]
    assert np.array_equal(gpu_perm(g, {"async_sweeps": 1, "debug_async_slots": 1000}), oracle.rcm(g.n, g.rowptr, g.colidx))
    rcm = rcm_mod()
    rp, ci = to_dev(g)
    o = rcm.rcm_options()
    o.async_sweeps, o.block_threads = 1, 256
    pm = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_ex(g.n, rp, ci, pm, o, None) == rcm.RCM_ERR_INVALID_ARG


def test_bottom_up_expansion_on_low_diameter_graphs():
    """Large random graphs of small diameter, where frontiers hold a large part of the graph and
    the automatic mode switches to bottom-up: top-down only, bottom-up everywhere and automatic
    all give the oracle's order (also with two large components ordered on the grid)."""
    rcm = rcm_mod()
    big = [synth.random_graph(300000, 1200000, 91, connected=True), synth.random_graph(200000, 300000, 92)]
    two = synth.concat([synth.random_graph(270000, 800000, 93, connected=True),
                        synth.random_graph(280000, 900000, 94, connected=True)])
    big.append(synth.permute(synth.Csr(two.n, two.rowptr, two.colidx), synth.random_permutation(two.n, 95)))
    for g in big:
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        for mode in (0, 1, 2, 3):
            assert np.array_equal(gpu_perm(g, {"expand_mode": mode}), want), mode
        assert np.array_equal(gpu_perm(g, {"expand_mode": 2, "narrow_threshold": -1, "fused_sweeps": -1}), want)
    rp, ci = to_dev(big[0])
    o = rcm.rcm_options()
    o.expand_mode = 4
    pm = torch.empty(big[0].n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_ex(big[0].n, rp, ci, pm, o, None) == rcm.RCM_ERR_INVALID_ARG
    o.expand_mode, o.block_threads = 3, 256
    assert rcm.rcm_order_ex(big[0].n, rp, ci, pm, o, None) == rcm.RCM_ERR_INVALID_ARG


def test_sort_free_variant_matches_the_oracle_variant():
    """rcm_options.row_order = 1 (children in stored row order) equals the oracle's sort-free
    variant on every executor: the persistent grid, the shared-memory CTA and the batched engine,
    including rows long enough for the whole-CTA sorter and rows stored in reverse."""
    rcm = rcm_mod()
    star = synth.csr_from_edges(20001, np.zeros(20000, np.int64), np.arange(1, 20001))
    rev = synth.Csr(star.n, star.rowptr, np.concatenate([star.colidx[:20000][::-1], star.colidx[20000:]]))
    graphs = [synth.c1_grid2d(), synth.grid((30, 20, 9), seed=81), synth.c3_mesh(20000), synth.knn_mesh(5000, 3, 82),
              synth.random_tree(3000, 83), rev, synth.random_graph(2000, 900, 84)] + small_graphs(40, 300, 85)
    for g in graphs:
        want = oracle.rcm(g.n, g.rowptr, g.colidx, row_order=1)
        assert np.array_equal(gpu_perm(g, {"row_order": 1}), want)
        assert np.array_equal(gpu_perm(g, {"row_order": 1, "executor": 1}), want)
        if g.n <= 4608:
            assert np.array_equal(gpu_perm(g, {"row_order": 1, "executor": 2}), want)
    batch = [g for g in graphs if g.n <= 30000]
    b = synth.concat(batch)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    o = rcm.rcm_batch_options()
    o.row_order = 1
    perm = torch.empty(b.n, dtype=torch.int32, device="cuda")
    rcm.check(rcm.rcm_order_batch_ex(len(batch), b.n, goff, rp, ci, perm, o), "batch_ex")
    rcm.check(rcm.rcm_stream_status(), "batch_ex")
    host = perm.cpu().numpy()
    for gi, g in enumerate(batch):
        assert np.array_equal(host[b.goff[gi]:b.goff[gi + 1]], oracle.rcm(g.n, g.rowptr, g.colidx, row_order=1))
    o.row_order = 2
    assert rcm.rcm_order_batch_ex(len(batch), b.n, goff, rp, ci, perm, o) == rcm.RCM_ERR_INVALID_ARG


def test_shared_memory_executor_matches_oracle():
    """One CTA with the graph's claims, stamps and padded rows in shared memory (graphs of at most
    4,608 vertices): the same orders as the oracle and the persistent grid, on grids, meshes with
    components, trees, stars with long rows, isolated vertices and random graphs."""
    graphs = [synth.c1_grid2d(), synth.grid((16, 16, 18), seed=5), synth.c3_mesh(4608, seed_offset=2),
              synth.path(4608), synth.random_tree(4000, 6), synth.csr_from_edges(300, [], []),
              synth.csr_from_edges(5, [0, 1], [1, 2])]
    star_src = np.zeros(999, np.int64)
    graphs.append(synth.csr_from_edges(1000, star_src, np.arange(1, 1000)))   # a 999-entry row
    graphs += small_graphs(40, 600, 108)
    for g in graphs:
        assert g.n <= 4608
        assert_parity(g, {"executor": 2})
        assert np.array_equal(gpu_perm(g, {"executor": 2}), gpu_perm(g, {"executor": 1}))


def test_shared_memory_executor_limits():
    rcm = rcm_mod()
    g = synth.grid((4609, 1), seed=1)
    rp, ci = to_dev(g)
    perm = torch.empty(g.n, dtype=torch.int32, device="cuda")
    o = rcm.rcm_options()
    o.executor = 2
    assert rcm.rcm_order_ex(g.n, rp, ci, perm, o, None) == rcm.RCM_ERR_TOO_LARGE
    o.executor = 3
    assert rcm.rcm_order_ex(g.n, rp, ci, perm, o, None) == rcm.RCM_ERR_INVALID_ARG


def test_stats_match_oracle():
    for g in [synth.c1_grid2d(), synth.grid((30, 20, 10), seed=1), synth.c3_mesh(20000)]:
        _, ost = oracle.rcm(g.n, g.rowptr, g.colidx, with_stats=True)
        _, st = gpu_perm(g, with_stats=True)
        assert st["components"] == ost["components"]
        assert st["sweeps"] == ost["sweeps"]
        assert st["max_ecc"] == ost["max_ecc"]
        assert st["traversals"] == ost["sweeps"]   # labelled sweep fused into the last sweep


def test_bad_csr_is_reported():
    rcm = rcm_mod()
    cases = [
        (np.array([0, 2, 1, 3], np.int32), np.array([1, 2, 0], np.int32)),   # rowptr decreases
        (np.array([0, 1, 2, 3], np.int32), np.array([1, 5, 0], np.int32)),   # column out of range
        (np.array([0, 1, 2, 3], np.int32), np.array([1, -1, 0], np.int32)),  # negative column
        (np.array([1, 1, 2, 3], np.int32), np.array([1, 0, 0], np.int32)),   # rowptr[0] != 0
    ]
    for rp_np, ci_np in cases:
        rp = torch.from_numpy(rp_np).cuda()
        ci = torch.from_numpy(ci_np).cuda()
        pm = torch.empty(3, dtype=torch.int32, device="cuda")
        st = rcm.rcm_order(3, rp, ci, pm)
        if st == rcm.RCM_OK:
            st = rcm.rcm_stream_status()
        assert st == rcm.RCM_ERR_BAD_CSR
    # the stream is usable afterwards
    assert_parity(synth.c1_grid2d())


def test_invalid_arguments():
    rcm = rcm_mod()
    pm = torch.empty(4, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order(-1, 0, 0, pm) == rcm.RCM_ERR_INVALID_ARG
    assert rcm.rcm_order(4, 0, 0, pm) == rcm.RCM_ERR_INVALID_ARG
    o = rcm.rcm_options()
    o.block_threads = 300
    g = synth.c1_grid2d()
    rp, ci = to_dev(g)
    perm = torch.empty(g.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_ex(g.n, rp, ci, perm, o, None) == rcm.RCM_ERR_INVALID_ARG
    o = rcm.rcm_options()
    o.grid_blocks = 100000
    assert rcm.rcm_order_ex(g.n, rp, ci, perm, o, None) == rcm.RCM_ERR_INVALID_ARG
    for cluster, blocks, threads in [(2, 0, 0), (1, 0, 256), (1, 17, 0)]:
        o = rcm.rcm_options()
        o.cluster, o.grid_blocks, o.block_threads = cluster, blocks, threads
        assert rcm.rcm_order_ex(g.n, rp, ci, perm, o, None) == rcm.RCM_ERR_INVALID_ARG


def test_bounded_wait_reports_timeout():
    """CTA 0 never arrives at the first grid barrier (test hook); the other CTAs' bounded waits run
    out, the kernel returns and the error is reported. Nothing faults or hangs; the context stays usable."""
    rcm = rcm_mod()
    g = synth.c1_grid2d()
    rp, ci = to_dev(g)
    perm = torch.empty(g.n, dtype=torch.int32, device="cuda")
    o = rcm.rcm_options()
    o.debug_stall_barrier = 1
    o.spin_limit_ns = 200_000_000
    o.grid_blocks = 4
    st = rcm.rcm_order_ex(g.n, rp, ci, perm, o, None)
    if st == rcm.RCM_OK:
        st = rcm.rcm_stream_status()
    assert st == rcm.RCM_ERR_TIMEOUT
    assert_parity(g)


def test_key_order_field_guard():
    """The labelled traversal's 64-bit claim keys hold the level above an in-level order field
    ord = b * slot + j; the host sizes the grid so that every CTA's share of a level fits its slot.
    With the field forced narrow (test hook) the kernel checks the slices itself: a level share that
    does not fit ends the call with RCM_ERR_TOO_LARGE, no fault, and the context stays usable; a
    forced width that still fits gives the oracle's order."""
    rcm = rcm_mod()
    g = synth.grid((30, 30, 30), seed=131)
    rp, ci = to_dev(g)
    perm = torch.empty(g.n, dtype=torch.int32, device="cuda")
    o = rcm.rcm_options()
    o.executor, o.narrow_threshold, o.debug_order_bits = 1, -1, 10   # slot = 1023 // CTAs: a few entries
    st = rcm.rcm_order_ex(g.n, rp, ci, perm, o, None)
    if st == rcm.RCM_OK:
        st = rcm.rcm_stream_status()
    assert st == rcm.RCM_ERR_TOO_LARGE
    assert_parity(g)
    o.debug_order_bits = 24                                           # roomy enough: same order
    rcm.check(rcm.rcm_order_ex(g.n, rp, ci, perm, o, None), "forced width")
    rcm.check(rcm.rcm_stream_status(), "forced width")
    assert np.array_equal(perm.cpu().numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))
    o.debug_order_bits = 63                                           # wider than the level leaves room for
    assert rcm.rcm_order_ex(g.n, rp, ci, perm, o, None) == rcm.RCM_ERR_INVALID_ARG


def test_latch_slots_are_freed_and_refused_when_all_are_held():
    """Every stream an ordering ran on holds one of 4,096 latch words until rcm_stream_status reads
    it. Ordering on new streams without reading their status ends with RCM_ERR_TOO_LARGE (before
    any work) once all are held, never with two streams sharing a word; reading one stream's status
    frees a word for the next stream. (Raw driver streams: torch hands out pooled streams.)"""
    import ctypes

    rcm = rcm_mod()
    cu = ctypes.CDLL("libcuda.so.1")
    g = synth.path(50, seed=3)
    rp, ci = to_dev(g)
    want = oracle.rcm(g.n, g.rowptr, g.colidx)
    o = rcm.rcm_options()
    o.executor, o.nnz = 2, g.nnz
    torch.cuda.synchronize()
    streams, outs, refused = [], [], None
    try:
        for _ in range(4097):
            h = ctypes.c_void_p()
            assert cu.cuStreamCreate(ctypes.byref(h), 1) == 0          # CU_STREAM_NON_BLOCKING
            out = torch.empty(g.n, dtype=torch.int32, device="cuda")
            status = rcm.rcm_order_ex(g.n, rp, ci, out, o, None, h.value)
            if status == rcm.RCM_ERR_TOO_LARGE:
                refused = h.value
                break
            assert status == rcm.RCM_OK
            streams.append(h.value)
            outs.append(out)
        assert refused is not None and len(streams) <= 4096
        assert rcm.rcm_stream_status(streams[0]) == rcm.RCM_OK          # frees its word
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        assert rcm.rcm_order_ex(g.n, rp, ci, out, o, None, refused) == rcm.RCM_OK
        assert rcm.rcm_stream_status(refused) == rcm.RCM_OK
        assert np.array_equal(out.cpu().numpy(), want)
        for st in streams[1:]:
            assert rcm.rcm_stream_status(st) == rcm.RCM_OK
        for out in outs[::512]:
            assert np.array_equal(out.cpu().numpy(), want)
    finally:
        for st in streams[1:]:
            rcm.rcm_stream_status(st)
        for st in streams + ([refused] if refused else []):
            cu.cuStreamDestroy_v2(ctypes.c_void_p(st))


def test_l2_window_restores_the_context_limit():
    """rcm_options.l2_persist raises the context's persisting-L2 limit for the traversal only: the
    call gives the oracle's order and leaves the limit as it found it (a raised limit slows later
    kernels of the context)."""
    import ctypes

    rcm = rcm_mod()
    cu = ctypes.CDLL("libcuda.so.1")

    def limit():
        v = ctypes.c_size_t()
        assert cu.cuCtxGetLimit(ctypes.byref(v), 6) == 0          # CU_LIMIT_PERSISTING_L2_CACHE_SIZE
        return v.value

    g = synth.grid((60, 60, 60), seed=141)
    rp, ci = to_dev(g)
    perm = torch.empty(g.n, dtype=torch.int32, device="cuda")
    o = rcm.rcm_options()
    o.executor, o.l2_persist = 1, 1
    before = limit()
    rcm.check(rcm.rcm_order_ex(g.n, rp, ci, perm, o, None), "l2 window")
    assert limit() == before
    rcm.check(rcm.rcm_stream_status(), "l2 window")
    assert np.array_equal(perm.cpu().numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))


def test_bandwidth_profile_matches_oracle():
    rcm = rcm_mod()
    for g in [synth.c1_grid2d(), synth.c3_mesh(5000), synth.random_graph(500, 900, 3)]:
        rp, ci = to_dev(g)
        for perm in [oracle.rcm(g.n, g.rowptr, g.colidx), np.arange(g.n, dtype=np.int32),
                     synth.rng_for(1).permutation(g.n).astype(np.int32)]:
            want = oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, perm)
            got = rcm.bandwidth_profile(rp, ci, torch.from_numpy(np.ascontiguousarray(perm)).cuda())
            assert got == want
        bad = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        st, _, _ = rcm.rcm_bandwidth_profile(g.n, rp, ci, bad)
        assert st == rcm.RCM_ERR_INVALID_ARG


def test_order_host_end_to_end():
    """Host buffers, pinned and pageable, including sizes that are not a multiple of 16 bytes and a
    pinned buffer at an odd 4-byte offset."""
    rcm = rcm_mod()
    for g in [synth.c1_grid2d(), synth.c3_mesh(10000), synth.csr_from_edges(5, [], []), synth.grid((7, 9), seed=4),
              synth.c3_mesh(300001)]:
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        ci_np = g.colidx.copy() if g.nnz else np.zeros(1, np.int32)
        for pinned in (True, False):
            rp = torch.from_numpy(g.rowptr.copy())
            ci = torch.from_numpy(ci_np.copy())
            pm = torch.empty(g.n, dtype=torch.int32)
            if pinned:
                rp, ci, pm = rp.pin_memory(), ci.pin_memory(), pm.pin_memory()
            rcm.check(rcm.rcm_order_host(g.n, rp, ci, pm), "rcm_order_host")
            assert np.array_equal(pm.numpy(), want), pinned
        # a pinned buffer whose data starts 4 bytes into its allocation
        big = torch.zeros(len(ci_np) + 1, dtype=torch.int32).pin_memory()
        big[1:] = torch.from_numpy(ci_np)
        pm = torch.empty(g.n, dtype=torch.int32).pin_memory()
        rcm.check(rcm.rcm_order_host(g.n, torch.from_numpy(g.rowptr.copy()).pin_memory(), big[1:], pm), "offset")
        assert np.array_equal(pm.numpy(), want)


def test_batch_matches_oracle_and_single():
    rcm = rcm_mod()
    graphs = [synth.batch_graph(int(k), int(s), [77, i]) for i, (k, s) in
              enumerate(zip(*synth.mix_sizes(60, 5, 4000, 77)[::-1]))]
    graphs += [synth.csr_from_edges(1, [], []), synth.csr_from_edges(7, [], []), synth.path(2)]
    b = synth.concat(graphs)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    perm = rcm.order_batch(goff, rp, ci).cpu().numpy()
    for gi, g in enumerate(graphs):
        seg = perm[b.goff[gi]:b.goff[gi + 1]]
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        assert np.array_equal(seg, want), gi
        if gi % 10 == 0:
            assert np.array_equal(seg, gpu_perm(g))


def test_batch_rejects_cross_block_entries():
    rcm = rcm_mod()
    a, c = synth.path(3), synth.path(3)
    b = synth.concat([a, c])
    colidx = b.colidx.copy()
    colidx[0] = 4  # row 0 of graph 0 points into graph 1
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(colidx).cuda()
    perm = torch.empty(b.n, dtype=torch.int32, device="cuda")
    st = rcm.rcm_order_batch(2, b.n, goff, rp, ci, perm)
    if st == rcm.RCM_OK:
        st = rcm.rcm_stream_status()
    assert st == rcm.RCM_ERR_BAD_CSR


def test_batch_validation_across_many_small_graphs():
    """Hundreds of graphs of 0 to 4 vertices, so one warp's 32 rows span many graphs (and empty
    ones): the valid batch orders as the oracle does, and an entry that leaves its graph's block,
    forward or backward, anywhere in the batch, is reported."""
    rcm = rcm_mod()
    rng = synth.rng_for(191)
    graphs = []
    for i in range(400):
        k = int(rng.integers(0, 5))
        graphs.append(synth.path(k, seed=[191, i]) if k > 0 else synth.csr_from_edges(0, [], []))
    b = synth.concat(graphs)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    perm = torch.empty(max(b.n, 1), dtype=torch.int32, device="cuda")
    rcm.check(rcm.rcm_order_batch(len(graphs), b.n, goff, rp, torch.from_numpy(b.colidx).cuda(), perm), "batch")
    rcm.check(rcm.rcm_stream_status(), "batch")
    host = perm.cpu().numpy()
    for gi, g in enumerate(graphs):
        assert np.array_equal(host[b.goff[gi]:b.goff[gi + 1]], oracle.rcm(g.n, g.rowptr, g.colidx)), gi
    big = [gi for gi, g in enumerate(graphs) if g.nnz > 0]
    for gi, step in ((big[-1], -1), (big[len(big) // 2], 1), (big[len(big) // 3], -1)):
        colidx = b.colidx.copy()
        e = int(b.rowptr[b.goff[gi]])
        colidx[e] = int(b.goff[gi] - 1) if step < 0 else int(b.goff[gi + 1])
        if not 0 <= colidx[e] < b.n:
            continue
        st = rcm.rcm_order_batch(len(graphs), b.n, goff, rp, torch.from_numpy(colidx).cuda(), perm)
        if st == rcm.RCM_OK:
            st = rcm.rcm_stream_status()
        assert st == rcm.RCM_ERR_BAD_CSR, (gi, step)


@pytest.mark.slow
def test_c2_grid192_full_size():
    """The full 192^3 workload in every launch configuration the benchmark's autotuner chooses from
    (frontier switches, sweep and expansion modes), and the sort-free variant against the oracle's."""
    from paper_1610_08128_gb300 import tune

    g = synth.c2_grid3d()
    want = oracle.rcm(g.n, g.rowptr, g.colidx)
    assert np.array_equal(gpu_perm(g), want)
    for opts in tune.SINGLE_CANDIDATES:
        if opts["executor"] == 2:
            continue  # the shared-memory CTA takes at most 4,608 vertices
        assert np.array_equal(gpu_perm(g, opts), want), opts
    assert np.array_equal(gpu_perm(g, {"row_order": 1}), oracle.rcm(g.n, g.rowptr, g.colidx, row_order=1))


@pytest.mark.slow
def test_middle_tier_on_high_diameter_grids():
    """The middle tier (levels of 512 to a few thousand vertices on one cluster) on grids whose
    levels mostly fall in that range: a 1000x1000 2D grid, a 3D grid, and a 2D grid with rows
    stored in shuffled order; every cluster size gives the oracle's order."""
    graphs = [synth.grid((1000, 1000), seed=151), synth.grid((96, 96, 96), seed=152),
              synth.shuffle_rows(synth.grid((700, 400), seed=153), 154)]
    for g in graphs:
        want = oracle.rcm(g.n, g.rowptr, g.colidx)
        for k in (2, 4, 8, 16):
            assert np.array_equal(gpu_perm(g, {"executor": 1, "mid_cluster": k}), want), k


@pytest.mark.slow
def test_c4_batch_full_size_sampled():
    """The full 10,000-graph batch, ordered as the benchmark does (tuned options, replay plan);
    a sample of graphs, including the largest, is checked against the oracle one by one."""
    from paper_1610_08128_gb300 import tune

    rcm = rcm_mod()
    b = synth.c4_batch(workers=synth.default_workers())
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    perm = torch.empty(b.n, dtype=torch.int32, device="cuda")
    best, _ = tune.tune_batch(b.G, b.n, goff, rp, ci, perm, repeats=1)
    o = rcm.rcm_batch_options()
    for k, v in best.items():
        setattr(o, k, v)
    st, plan = rcm.rcm_batch_plan_create(b.G, b.n, int(b.rowptr[-1]), goff, rp, ci, perm, o)
    rcm.check(st, "plan")
    try:
        rcm.check(rcm.rcm_batch_plan_launch(plan), "launch")
        rcm.check(rcm.rcm_batch_plan_status(plan), "status")
    finally:
        rcm.rcm_batch_plan_destroy(plan)
    host = perm.cpu().numpy()
    sizes = np.diff(b.goff)
    sample = list(synth.rng_for(81).choice(b.G, 60, replace=False)) + [int(np.argmax(sizes))]
    for gi in sample:
        g = b.graphs[gi]
        assert np.array_equal(host[b.goff[gi]:b.goff[gi + 1]], oracle.rcm(g.n, g.rowptr, g.colidx)), gi


@pytest.mark.slow
def test_c3_mesh_full_size():
    g = synth.c3_mesh()
    assert_parity(g)


def test_batch_options_and_replay_plan_match_oracle():
    """Every batched tuning (CTA width, row-sort split) and a CUDA-graph replay plan return the
    oracle's orders; the plan replays correctly after its inputs change."""
    rcm = rcm_mod()
    graphs = [synth.batch_graph(int(k), int(s), [78, i]) for i, (k, s) in
              enumerate(zip(*synth.mix_sizes(40, 5, 3000, 78)[::-1]))]
    graphs.append(synth.csr_from_edges(50, np.zeros(49, np.int64), np.arange(1, 50)))  # a 49-entry row
    b = synth.concat(graphs)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    want = [oracle.rcm(g.n, g.rowptr, g.colidx) for g in graphs]

    def check(perm):
        host = perm.cpu().numpy()
        for gi, g in enumerate(graphs):
            assert np.array_equal(host[b.goff[gi]:b.goff[gi + 1]], want[gi]), gi

    for threads in (128, 256, 512):
        for split in (4, 8, 32):
            o = rcm.rcm_batch_options()
            o.block_threads, o.row_sort_split = threads, split
            perm = torch.empty(b.n, dtype=torch.int32, device="cuda")
            rcm.check(rcm.rcm_order_batch_ex(len(graphs), b.n, goff, rp, ci, perm, o), "batch_ex")
            rcm.check(rcm.rcm_stream_status(), "batch_ex")
            check(perm)
    o = rcm.rcm_batch_options()
    o.block_threads = 100
    perm = torch.empty(b.n, dtype=torch.int32, device="cuda")
    assert rcm.rcm_order_batch_ex(len(graphs), b.n, goff, rp, ci, perm, o) == rcm.RCM_ERR_INVALID_ARG

    perm = torch.full((b.n,), -1, dtype=torch.int32, device="cuda")
    st, plan = rcm.rcm_batch_plan_create(len(graphs), b.n, int(b.rowptr[-1]), goff, rp, ci, perm)
    rcm.check(st, "plan")
    try:
        for _ in range(2):
            rcm.check(rcm.rcm_batch_plan_launch(plan), "launch")
            rcm.check(rcm.rcm_batch_plan_status(plan), "status")
            check(perm)
        # same structure, different ids inside each block: the replay orders the new pattern
        graphs2 = [synth.permute(g, synth.rng_for([79, i]).permutation(g.n)) for i, g in enumerate(graphs)]
        b2 = synth.concat(graphs2)
        assert np.array_equal(b2.goff, b.goff) and b2.rowptr[-1] == b.rowptr[-1]
        rp.copy_(torch.from_numpy(b2.rowptr))
        ci.copy_(torch.from_numpy(b2.colidx))
        rcm.check(rcm.rcm_batch_plan_launch(plan), "launch")
        rcm.check(rcm.rcm_batch_plan_status(plan), "status")
        host = perm.cpu().numpy()
        for gi, g in enumerate(graphs2):
            assert np.array_equal(host[b2.goff[gi]:b2.goff[gi + 1]], oracle.rcm(g.n, g.rowptr, g.colidx)), gi
    finally:
        rcm.check(rcm.rcm_batch_plan_destroy(plan), "destroy")


def test_autotuner_picks_a_candidate_with_identical_results():
    from paper_1610_08128_gb300 import tune

    rcm = rcm_mod()
    graphs = [synth.batch_graph(int(k), int(s), [80, i]) for i, (k, s) in
              enumerate(zip(*synth.mix_sizes(30, 50, 2000, 80)[::-1]))]
    b = synth.concat(graphs)
    goff = torch.from_numpy(b.goff).cuda()
    rp = torch.from_numpy(b.rowptr).cuda()
    ci = torch.from_numpy(b.colidx).cuda()
    perm = torch.empty(b.n, dtype=torch.int32, device="cuda")
    best, table = tune.tune_batch(len(graphs), b.n, goff, rp, ci, perm, repeats=1)
    assert best in tune.BATCH_CANDIDATES and len(table) == len(tune.BATCH_CANDIDATES)
    g = synth.c1_grid2d()
    rp1, ci1 = to_dev(g)
    perm1 = torch.empty(g.n, dtype=torch.int32, device="cuda")
    best1, table1 = tune.tune_single(g.n, rp1, ci1, perm1, nnz=g.nnz, repeats=1)
    assert best1 in tune.SINGLE_CANDIDATES and len(table1) == len(tune.SINGLE_CANDIDATES)
    assert np.array_equal(perm1.cpu().numpy(), oracle.rcm(g.n, g.rowptr, g.colidx))


def test_quality_report_permutes_the_matrix():
    """P A P^T built on the device equals the host permutation; SpMV on it equals the permuted
    product; the report's bandwidth and profile equal the oracle's."""
    from paper_1610_08128_gb300 import quality

    g = synth.c3_mesh(20000)
    want = oracle.rcm(g.n, g.rowptr, g.colidx)
    rp, ci = to_dev(g)
    perm = torch.from_numpy(np.asarray(want, dtype=np.int32)).cuda()
    prp, pci = quality.permute_csr(rp, ci, perm)
    pos = np.empty(g.n, np.int64)
    pos[want] = np.arange(g.n)
    h = synth.permute(g, pos)
    assert np.array_equal(prp.cpu().numpy(), h.rowptr) and np.array_equal(pci.cpu().numpy(), h.colidx)
    vals = torch.ones(ci.numel(), dtype=torch.float32, device="cuda")
    a = torch.sparse_csr_tensor(rp, ci, vals, size=(g.n, g.n))
    b = torch.sparse_csr_tensor(prp, pci, vals, size=(g.n, g.n))
    x = torch.rand(g.n, 1, device="cuda")
    assert torch.allclose((a @ x)[perm.long()], b @ x[perm.long()], rtol=1e-5, atol=1e-5)
    r = quality.report(rp, ci, perm, repeats=2)
    assert (r["bandwidth_rcm"], r["profile_rcm"]) == oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, want)
    assert r["bandwidth_rcm"] < r["bandwidth_original"]
