"""rcm_validate (the pattern contract checked on the GPU) against the plain definitions, computed on
the host with Python sets: structure, columns, diagonal entries, duplicates and symmetry."""
import numpy as np
import pytest

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


def reference(n, rowptr, colidx):
    """The report by definition: faults per row, first faulty row; duplicates and asymmetric
    entries only when every row and column is well formed (else -1)."""
    rp = np.asarray(rowptr, np.int64)
    ci = np.asarray(colidx, np.int64)
    nnz = int(rp[n])
    bad_rows = bad_cols = diag = maxrow = 0
    faulty = set()
    if rp[0] != 0:
        bad_rows += 1
        faulty.add(0)
    for v in range(n):
        a, b = int(rp[v]), int(rp[v + 1])
        if a < 0 or b < a or b > nnz:
            bad_rows += 1
            faulty.add(v)
            continue
        row = ci[a:b]
        out = int(((row < 0) | (row >= n)).sum())
        diag += int((row == v).sum())
        if out:
            bad_cols += out
            faulty.add(v)
            continue
        maxrow = max(maxrow, b - a)
    dup = asym = -1
    if bad_rows == 0 and bad_cols == 0:
        sets = [set(ci[rp[v]:rp[v + 1]].tolist()) for v in range(n)]
        dup = asym = 0
        for v in range(n):
            d = int(rp[v + 1] - rp[v]) - len(sets[v])
            dup += d
            miss = sum(1 for w in sets[v] if w != v and v not in sets[w])
            asym += miss
            if d or miss:
                faulty.add(v)
    return {"bad_rows": bad_rows, "bad_columns": bad_cols, "duplicates": dup, "asymmetric": asym, "diagonal": diag,
            "max_row": maxrow, "first_bad_row": min(faulty) if faulty else -1}


def run(n, rowptr, colidx):
    from paper_1610_08128_gb300 import rcm

    rp = torch.from_numpy(np.ascontiguousarray(rowptr, np.int32)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(colidx if len(colidx) else np.zeros(1), np.int32)).cuda()
    assert rp.numel() == n + 1
    return rcm.validate(rp, ci)


def check(n, rowptr, colidx):
    ok, rep = run(n, rowptr, colidx)
    want = reference(n, rowptr, colidx)
    assert rep == want
    clean = want["bad_rows"] == 0 and want["bad_columns"] == 0 and want["duplicates"] == 0 and want["asymmetric"] == 0
    assert ok == clean
    return rep


def test_valid_patterns():
    star = synth.csr_from_edges(20001, np.zeros(20000, np.int64), np.arange(1, 20001))      # a row beyond shared memory
    star5 = synth.csr_from_edges(5001, np.zeros(5000, np.int64), np.arange(1, 5001))        # a whole-CTA row
    graphs = [synth.c1_grid2d(), synth.c3_mesh(20000), synth.random_graph(3000, 9000, 3, diagonal=True), star, star5,
              synth.path(100), synth.csr_from_edges(1, [], []), synth.csr_from_edges(6, [0], [1])]
    for g in graphs:
        rep = check(g.n, g.rowptr, g.colidx)
        assert rep["asymmetric"] == 0 and rep["duplicates"] == 0
    rep = check(star.n, star.rowptr, star.colidx)
    assert rep["max_row"] == 20000
    assert run(0, np.zeros(1, np.int32), np.zeros(0, np.int32))[0]


def drop_entries(g, frac, seed):
    rng = synth.rng_for(seed)
    keep = rng.random(g.nnz) >= frac
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    rp = np.zeros(g.n + 1, np.int64)
    np.add.at(rp, rows[keep] + 1, 1)
    return np.cumsum(rp).astype(np.int32), g.colidx[keep]


def test_asymmetric_entries_are_counted():
    g = synth.random_graph(2000, 6000, 11)
    rp, ci = drop_entries(g, 0.01, 12)
    rep = check(g.n, rp, ci)
    assert rep["asymmetric"] > 0
    # a long row whose partners lack the back entries, and the other way round
    star = synth.csr_from_edges(12001, np.zeros(12000, np.int64), np.arange(1, 12001))
    rp, ci = drop_entries(star, 0.001, 13)
    check(star.n, rp, ci)


def test_duplicates_are_counted():
    g = synth.random_graph(1500, 4000, 14)
    rng = synth.rng_for(15)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    extra = rng.choice(g.nnz, 40, replace=False)
    r2 = np.concatenate([rows, rows[extra]])
    c2 = np.concatenate([g.colidx, g.colidx[extra]])
    order = np.argsort(r2, kind="stable")
    rp = np.zeros(g.n + 1, np.int64)
    np.add.at(rp, r2 + 1, 1)
    rep = check(g.n, np.cumsum(rp).astype(np.int32), c2[order].astype(np.int32))
    assert rep["duplicates"] == 40
    # a long row with a repeated entry (sorted by the whole CTA)
    star = synth.csr_from_edges(9001, np.zeros(9000, np.int64), np.arange(1, 9001))
    ci = star.colidx.copy()
    ci[5] = ci[6]
    check(star.n, star.rowptr, ci)


def test_malformed_rows_and_columns():
    g = synth.random_graph(500, 1500, 16)
    ci = g.colidx.copy()
    ci[[3, 100, 700]] = [g.n, -1, g.n + 7]
    rep = check(g.n, g.rowptr, ci)
    assert rep["bad_columns"] == 3 and rep["duplicates"] == -1
    rp = g.rowptr.copy()
    rp[10], rp[11] = rp[11], rp[10]                  # a descending pair: two malformed rows at most
    check(g.n, rp, g.colidx)
    rp = g.rowptr.copy()
    rp[0] = 1
    check(g.n, rp, g.colidx)
    rp = g.rowptr.copy()
    rp[-1] = -5                                      # negative entry count: every row is malformed
    check(g.n, rp, g.colidx)
