"""The seeded generators: determinism, symmetry, sizes of the workloads, component counts."""
import numpy as np
import pytest

from paper_1610_08128_gb300 import synth


def _sym_ok(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    a = set(zip(rows.tolist(), g.colidx.tolist()))
    return all((c, r) in a for r, c in a)


def test_grid_sizes_and_symmetry():
    g = synth.c1_grid2d()
    assert (g.n, g.nnz) == (4096, 16128)
    assert _sym_ok(g)
    g3 = synth.grid((7, 6, 5), seed=1)
    assert g3.nnz == 2 * (6 * 6 * 5 + 7 * 5 * 5 + 7 * 6 * 4)
    assert np.array_equal(synth.grid_fast((7, 6, 5), seed=1).colidx, g3.colidx)
    assert _sym_ok(g3)


def test_c2_counts_formula():
    # 192^3 7-point grid: 3 * 191 * 192^2 undirected edges
    side = 192
    assert 2 * 3 * (side - 1) * side * side == 42_246_144


def test_deterministic_in_seed():
    a, b = synth.c3_mesh(5000), synth.c3_mesh(5000)
    assert np.array_equal(a.colidx, b.colidx) and np.array_equal(a.rowptr, b.rowptr)
    c = synth.c3_mesh(5000, seed_offset=1)
    assert not (c.n == a.n and np.array_equal(c.colidx, a.colidx))


def test_mesh_components_equal_regions():
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import connected_components
    for off in range(3):
        g = synth.c3_mesh(20000, seed_offset=off)
        A = sp.csr_matrix((np.ones(g.nnz), g.colidx, g.rowptr), shape=(g.n, g.n))
        assert connected_components(A)[0] == g.meta["regions"]
        assert _sym_ok(g)
        # diagonal stored on every row
        rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        assert np.count_nonzero(rows == g.colidx) == g.n


def test_batch_concat_offsets():
    b = synth.c4_batch(G=12, nmin=50, nmax=500)
    assert b.G == 12 and b.n == sum(g.n for g in b.graphs)
    for gi, g in enumerate(b.graphs):
        a0, a1 = int(b.goff[gi]), int(b.goff[gi + 1])
        seg = b.colidx[b.rowptr[a0]:b.rowptr[a1]]
        assert seg.min(initial=a0) >= a0 and seg.max(initial=a0) < max(a1, a0 + 1)
        assert np.array_equal(b.rowptr[a0:a1 + 1] - b.rowptr[a0], g.rowptr)


def test_trace_shape():
    arr, which, pool = synth.c5_trace(requests=50, pool=4, nmin=100, nmax=2000)
    assert len(arr) == 50 and np.all(np.diff(arr) >= 0) and arr[0] == 0
    assert which.max() < 4 and len(pool) == 4


def test_shuffle_rows_keeps_each_row_set_and_is_seeded():
    g = synth.grid((9, 11), seed=3)
    a, b, c = synth.shuffle_rows(g, 1), synth.shuffle_rows(g, 1), synth.shuffle_rows(g, 2)
    assert np.array_equal(a.rowptr, g.rowptr) and np.array_equal(a.colidx, b.colidx)
    assert not np.array_equal(a.colidx, c.colidx)
    for v in range(g.n):
        lo, hi = g.rowptr[v], g.rowptr[v + 1]
        assert sorted(a.colidx[lo:hi]) == list(g.colidx[lo:hi])


def test_power_law_and_circulant_patterns():
    g = synth.power_law(20000, 10, 2.5, 3)
    lens = np.diff(g.rowptr)
    assert lens.max() > 200 and np.median(lens) < 20          # hubs and a light tail
    rows = np.repeat(np.arange(g.n), lens)
    keys = set(zip(rows.tolist(), g.colidx.tolist()))
    assert all((c, r) in keys for r, c in keys) and all(r != c for r, c in keys)
    assert len(keys) == g.nnz                                 # no duplicates
    c = synth.circulant(1000, range(1, 4), seed=2)
    assert c.nnz == 6000 and set(np.diff(c.rowptr).tolist()) == {6}
