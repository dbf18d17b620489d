"""Pins that tie the serial oracle to the paper and to mathematics, not to itself.

Each test names the passage it follows. Every check here is computed independently of the
oracle's C code: closed forms (path, square grid), theorems (tree diameter), a brute-force search
over all orderings that satisfy the Cuthill-McKee definition, an independent level-synchronous
restatement of Alg. 3/Alg. 4 in numpy, hand-worked fixtures under tests/golden/, and mutants of
the oracle source that the pins must reject.
"""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import tempfile
from collections import deque

import numpy as np
import pytest

import oracle
from paper_1610_08128_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------
# independent helpers (plain Python, written from the definitions of Sec. II-A)


def adjacency(g):
    adj = [set() for _ in range(g.n)]
    for v in range(g.n):
        for w in g.colidx[g.rowptr[v]:g.rowptr[v + 1]]:
            if w != v:
                adj[v].add(int(w))
    return adj


def bfs_dist(adj, s):
    d = {s: 0}
    q = deque([s])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if w not in d:
                d[w] = d[u] + 1
                q.append(w)
    return d


def bandwidth_profile_py(adj, perm):
    """beta_i = i - f_i with f_i the smallest new index among row i's entries (diagonal included)."""
    pos = {int(v): i for i, v in enumerate(perm)}
    bw = prof = 0
    for i, v in enumerate(perm):
        f = min([i] + [pos[w] for w in adj[int(v)]])
        bw = max(bw, i - f)
        prof += i - f
    return bw, prof


def is_permutation(p, n):
    return len(p) == n and np.array_equal(np.sort(np.asarray(p)), np.arange(n))


def components(adj):
    seen, comps = {}, []
    for s in range(len(adj)):
        if s in seen:
            continue
        d = bfs_dist(adj, s)
        for v in d:
            seen[v] = len(comps)
        comps.append(sorted(d))
    return comps


def key(deg, v):
    return (deg[v], v)


def george_liu_roots(adj, deg):
    """Alg. 2 restated over an all-pairs distance table (tiny graphs only): for each component in
    start-rule order (lowest (degree, id) unnumbered vertex first), the sweep sequence and root."""
    n = len(adj)
    dist = [bfs_dist(adj, s) for s in range(n)]
    ecc = [max(d.values()) for d in dist]
    comps = components(adj)
    comps.sort(key=lambda c: min(key(deg, v) for v in c))
    out = []
    for c in comps:
        r = min(c, key=lambda v: key(deg, v))
        seq = [r]
        nlvl = ecc[r] - 1
        while ecc[r] > nlvl:
            nlvl = ecc[r]
            last = [v for v, dv in dist[r].items() if dv == ecc[r]]
            r = min(last, key=lambda v: key(deg, v))
            seq.append(r)
        out.append((c, r, seq))
    return out


def enumerate_cm_sequences(adj, deg, comp_roots, limit=3):
    """All vertex sequences that satisfy the Cuthill-McKee definition (Alg. 1 / Sec. III-B):
    components appear in start-rule order, each beginning at its root; every later vertex of a
    component has an earlier neighbour; the position of a vertex's earliest neighbour (its parent)
    never decreases along the sequence; children of one parent appear in increasing (degree, id).
    Backtracking over valid prefixes; stops after ``limit`` solutions."""
    n = len(adj)
    comp_of = {}
    for ci, (c, _, _) in enumerate(comp_roots):
        for v in c:
            comp_of[v] = ci
    sols = []
    seq, pos = [], {}

    def parent_pos(v):
        ps = [pos[w] for w in adj[v] if w in pos]
        return min(ps) if ps else None

    def rec(ci, last_parent, last_key):
        if len(sols) >= limit:
            return
        if len(seq) == n:
            sols.append(list(seq))
            return
        comp_done = all(v in pos for v in comp_roots[ci][0]) if ci >= 0 else True
        if comp_done:
            nci = ci + 1
            root = comp_roots[nci][1]
            seq.append(root)
            pos[root] = len(seq) - 1
            rec(nci, -1, None)
            seq.pop()
            del pos[root]
            return
        for v in range(n):
            if v in pos or comp_of[v] != ci:
                continue
            p = parent_pos(v)
            if p is None or p < last_parent:
                continue
            if p == last_parent and last_key is not None and key(deg, v) <= last_key:
                continue
            seq.append(v)
            pos[v] = len(seq) - 1
            rec(ci, p, key(deg, v))
            seq.pop()
            del pos[v]

    rec(-1, -1, None)
    return sols


def alg3_level_synchronous(g, deg, root, nv0, R, stored_order=False):
    """Alg. 3 restated with dense numpy vectors: SpMSpV over (select2nd, min) gives each discovered
    vertex the smallest label among its frontier neighbours; SELECT keeps unlabelled vertices;
    SORTPERM orders them by (parent label, degree, id); labels continue from nv.
    stored_order=True: the sort-free variant, (parent label, position in the parent's row)."""
    rp, ci = g.rowptr.astype(np.int64), g.colidx.astype(np.int64)
    R[root] = nv0
    nv = nv0 + 1
    cur = np.array([root], dtype=np.int64)
    while len(cur):
        lens = rp[cur + 1] - rp[cur]
        starts = np.repeat(rp[cur], lens)
        offs = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens)
        w = ci[starts + offs]
        lab = np.repeat(R[cur], lens)
        sel = R[w] == -1                       # SELECT(R = -1)
        w, lab, offs = w[sel], lab[sel], offs[sel]
        if len(w) == 0:
            break
        parent = np.full(g.n, np.iinfo(np.int64).max)
        np.minimum.at(parent, w, lab)          # (select2nd, min)
        nxt = np.unique(w)
        if stored_order:
            at = np.full(g.n, np.iinfo(np.int64).max)
            mine = lab == parent[w]            # the entry of w in its parent's row
            np.minimum.at(at, w[mine], offs[mine])
            order = np.lexsort((at[nxt], parent[nxt]))
        else:
            order = np.lexsort((nxt, deg[nxt], parent[nxt]))   # SORTPERM by (parent, degree, id)
        nxt = nxt[order]
        R[nxt] = nv + np.arange(len(nxt))
        nv += len(nxt)
        cur = nxt
    return nv


def alg4_level_synchronous(g, deg, r):
    """Alg. 4 with the reading that compares the eccentricities of successive sweeps: repeated
    level-synchronous BFS, REDUCE(min (degree, id)) over the last non-empty level."""
    rp, ci = g.rowptr.astype(np.int64), g.colidx.astype(np.int64)
    prev = -1
    sweeps = 0
    while True:
        L = np.full(g.n, -1)
        L[r] = 0
        cur = np.array([r])
        lev = 0
        while True:
            lens = rp[cur + 1] - rp[cur]
            starts = np.repeat(rp[cur], lens)
            offs = np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens)
            w = np.unique(ci[starts + offs])
            w = w[L[w] == -1]
            if len(w) == 0:
                break
            lev += 1
            L[w] = lev
            cur = w
        sweeps += 1
        nxt = cur[np.lexsort((cur, deg[cur]))][0]
        if prev >= 0 and lev <= prev:
            return r, sweeps, lev
        prev = lev
        r = int(nxt)


def small_graphs(count, nmax, seed, connected=None):
    rng = synth.rng_for(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(1, nmax + 1))
        m = int(rng.integers(0, 2 * n + 1))
        conn = bool(rng.integers(0, 2)) if connected is None else connected
        out.append(synth.random_graph(n, m, [seed, i], connected=conn, diagonal=bool(i % 3 == 0)))
    return out


def rcm_of(g, lib=None):
    return oracle.rcm(g.n, g.rowptr, g.colidx, lib=lib)


# ------------------------------------------------------------------------------------------
# closed forms


def test_path_natural_ids_is_identity_bandwidth_one():
    """Path 0-1-...-(n-1): start at 0 (degree 1, lowest id), sweep to n-1, stop (ecc equal),
    label from n-1 downwards, reverse: the identity; bandwidth 1 (Sec. II-A definitions)."""
    for n in range(2, 40):
        g = synth.path(n)
        p = rcm_of(g)
        assert np.array_equal(p, np.arange(n))
        assert oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, p) == (1, n - 1)


def test_path_any_ids_bandwidth_one():
    for n in range(2, 60, 3):
        for s in range(4):
            g = synth.path(n, seed=[n, s])
            p = rcm_of(g)
            assert is_permutation(p, n)
            assert bandwidth_profile_py(adjacency(g), p) == (1, n - 1)


def test_square_grid_bandwidth_equals_side():
    """A k x k 5-point grid ordered by RCM from a corner has bandwidth exactly k, for any ids."""
    for k in range(2, 21):
        for s in range(5):
            g = synth.grid((k, k), seed=[k, s])
            p = rcm_of(g)
            bw, _ = bandwidth_profile_py(adjacency(g), p)
            assert bw == k, (k, s, bw)


def test_rect_grid_bandwidth_min_or_min_plus_one():
    for r, c in [(3, 7), (5, 2), (8, 13), (12, 4), (2, 9), (17, 6)]:
        for s in range(4):
            g = synth.grid((r, c), seed=[r, c, s])
            bw, _ = bandwidth_profile_py(adjacency(g), rcm_of(g))
            assert bw in (min(r, c), min(r, c) + 1), (r, c, s, bw)


def test_cube_grid_root_is_corner():
    """On a 3D grid the pseudo-peripheral root is a corner: ecc = sum of (side - 1)."""
    for dims in [(3, 4, 5), (6, 6, 6), (2, 7, 3)]:
        g = synth.grid(dims, seed=list(dims))
        deg = oracle.degrees(g.n, g.rowptr, g.colidx)
        r0 = int(np.lexsort((np.arange(g.n), deg))[0])
        root, sweeps, ecc = oracle.pseudo_peripheral(g.n, g.rowptr, g.colidx, r0)
        assert ecc == sum(d - 1 for d in dims)
        assert deg[root] == 3
        assert sweeps == 2


def test_tree_root_is_diameter_endpoint():
    """For a tree, the farthest vertex from any vertex is an end of a longest path, so the George-
    Liu search (Alg. 2) returns a vertex whose eccentricity equals the diameter."""
    for i in range(60):
        n = 2 + (i * 7) % 40
        g = synth.random_tree(n, [11, i])
        adj = adjacency(g)
        diam = max(max(bfs_dist(adj, s).values()) for s in range(n))
        deg = oracle.degrees(g.n, g.rowptr, g.colidx)
        r0 = int(np.lexsort((np.arange(n), deg))[0])
        root, _, ecc = oracle.pseudo_peripheral(g.n, g.rowptr, g.colidx, r0)
        assert ecc == diam == max(bfs_dist(adj, root).values())


# ------------------------------------------------------------------------------------------
# the definition, by brute force


def test_bruteforce_unique_cm_sequence_small_graphs():
    """On graphs of at most 12 vertices, exactly one vertex sequence satisfies the Cuthill-McKee
    definition from the George-Liu roots, and the oracle's output is that sequence reversed."""
    checked = 0
    for g in small_graphs(250, 12, 21):
        adj = adjacency(g)
        deg = np.array([len(a) for a in adj], dtype=np.int64)
        roots = george_liu_roots(adj, deg)
        sols = enumerate_cm_sequences(adj, deg, roots)
        assert len(sols) == 1
        p = rcm_of(g)
        assert list(p[::-1]) == sols[0]
        checked += 1
    assert checked == 250


def test_roots_and_sweep_counts_match_bruteforce():
    for g in small_graphs(200, 14, 22, connected=True):
        adj = adjacency(g)
        deg = np.array([len(a) for a in adj], dtype=np.int64)
        (c, root, seq), = george_liu_roots(adj, deg)
        r0 = seq[0]
        got = oracle.pseudo_peripheral(g.n, g.rowptr, g.colidx, r0)
        dist = bfs_dist(adj, root)
        assert got == (root, len(seq), max(dist.values()))


def test_structural_invariants_in_cm_order():
    """In Cuthill-McKee order: BFS levels from the root are contiguous and increasing; the label of
    the earliest neighbour (parent) is non-decreasing; equal parents appear in (degree, id) order;
    ecc(root) >= ecc(start vertex)."""
    for g in small_graphs(40, 300, 23, connected=True) + [synth.c1_grid2d()]:
        adj = adjacency(g)
        deg = [len(a) for a in adj]
        seq = list(rcm_of(g)[::-1])
        pos = {v: i for i, v in enumerate(seq)}
        root = seq[0]
        dist = bfs_dist(adj, root)
        levels = [dist[v] for v in seq]
        assert levels == sorted(levels)
        parents = [min(pos[w] for w in adj[v]) for v in seq[1:]]
        assert parents == sorted(parents)
        for i in range(1, len(seq) - 1):
            if parents[i - 1] == parents[i]:
                assert (deg[seq[i]], seq[i]) < (deg[seq[i + 1]], seq[i + 1])
        r0 = min(range(g.n), key=lambda v: (deg[v], v))
        assert max(dist.values()) >= max(bfs_dist(adj, r0).values())


def test_fig2_child_attaches_to_min_label_parent():
    """Fig. 2: with frontier {e, b} where e has the smaller label, a child c adjacent to both takes
    e as its parent, so c is numbered before b's other children."""
    data = read_golden("fig2_min_parent.txt")
    n = int(data["n"][0])
    e = np.array(data["edges"], dtype=np.int64).reshape(-1, 2)
    g = synth.csr_from_edges(n, e[:, 0], e[:, 1])
    label = oracle.cm_from_root(g.n, g.rowptr, g.colidx, int(data["root"][0]))
    assert list(label) == [int(x) for x in data["labels"]]


# ------------------------------------------------------------------------------------------
# independent level-synchronous restatement (Alg. 3 / Alg. 4) against the queue form (Alg. 1/2)


def test_alg3_level_form_equals_queue_form():
    for g in small_graphs(120, 400, 24) + [synth.c1_grid2d(), synth.c3_mesh(3000)]:
        deg = oracle.degrees(g.n, g.rowptr, g.colidx).astype(np.int64)
        R = np.full(g.n, -1, dtype=np.int64)
        nv = 0
        order = np.lexsort((np.arange(g.n), deg))
        for r0 in order:
            if R[r0] != -1:
                continue
            root, _, _ = alg4_level_synchronous(g, deg, int(r0))
            nv = alg3_level_synchronous(g, deg, root, nv, R)
        assert nv == g.n
        perm = np.empty(g.n, dtype=np.int64)
        perm[g.n - 1 - R] = np.arange(g.n)
        assert np.array_equal(perm, rcm_of(g))


def test_fifo_traversal_over_sorted_rows_is_the_ordering_of_each_component():
    """The one-thread ordering of tiny components rests on this: with every row stored in (degree,
    id) order, a plain FIFO traversal that appends each dequeued vertex's unvisited neighbours in
    row order numbers a component as Alg. 1 does, and its level boundaries give Alg. 2 the
    eccentricity and the last level's least (degree, id) vertex. Restated per component (sweeps
    from the component's start vertex while the eccentricity grows strictly, the last root's
    traversal as its numbering; components in start order; one reversal) and compared with the
    oracle, sweep counts included, on small graphs of many components."""
    graphs = small_graphs(150, 60, 31) + small_graphs(40, 300, 32)
    for g in graphs:
        deg = oracle.degrees(g.n, g.rowptr, g.colidx).astype(np.int64)
        rows = []
        for v in range(g.n):
            nb = [int(w) for w in g.colidx[g.rowptr[v]:g.rowptr[v + 1]] if w != v]
            rows.append(sorted(nb, key=lambda w: (deg[w], w)))

        def fifo(root):
            seen = {root}
            q = [root]
            head, lend, ecc, lmin = 0, 1, 0, None
            while True:
                u = q[head]
                head += 1
                key = (int(deg[u]), u)
                lmin = key if lmin is None or key < lmin else lmin
                for w in rows[u]:
                    if w not in seen:
                        seen.add(w)
                        q.append(w)
                if head == lend:
                    if len(q) == lend:
                        return ecc, lmin[1], q
                    ecc, lend, lmin = ecc + 1, len(q), None

        labelled, seq, sweeps = set(), [], 0
        for r0 in sorted(range(g.n), key=lambda v: (deg[v], v)):
            if r0 in labelled:
                continue
            ecc_prev, r, q = fifo(r0)
            sweeps += 1
            while True:
                ecc, nxt, q = fifo(r)
                sweeps += 1
                if ecc <= ecc_prev:
                    break
                ecc_prev, r = ecc, nxt
            seq += q
            labelled.update(q)
        want, st = oracle.rcm(g.n, g.rowptr, g.colidx, with_stats=True)
        assert np.array_equal(np.array(seq[::-1], dtype=np.int64), want.astype(np.int64))
        assert sweeps == st["sweeps"]


def test_sort_free_variant_level_form_equals_queue_form():
    """The sort-free variant (children in stored row order) against the level form with the key
    (parent label, position in the parent's row)."""
    for g in small_graphs(120, 400, 31) + [synth.c1_grid2d(), synth.c3_mesh(3000), synth.knn_mesh(2000, 3, 5)]:
        deg = oracle.degrees(g.n, g.rowptr, g.colidx).astype(np.int64)
        R = np.full(g.n, -1, dtype=np.int64)
        nv = 0
        for r0 in np.lexsort((np.arange(g.n), deg)):
            if R[r0] != -1:
                continue
            root, _, _ = alg4_level_synchronous(g, deg, int(r0))
            nv = alg3_level_synchronous(g, deg, root, nv, R, stored_order=True)
        perm = np.empty(g.n, dtype=np.int64)
        perm[g.n - 1 - R] = np.arange(g.n)
        assert np.array_equal(perm, oracle.rcm(g.n, g.rowptr, g.colidx, row_order=1))


def _rows_sorted_by_degree(g):
    deg = oracle.degrees(g.n, g.rowptr, g.colidx).astype(np.int64)
    ci = g.colidx.copy()
    for v in range(g.n):
        a, b = g.rowptr[v], g.rowptr[v + 1]
        row = ci[a:b]
        ci[a:b] = row[np.lexsort((row, deg[row]))]
    return synth.Csr(g.n, g.rowptr, ci)


def test_sort_free_variant_is_the_ordering_when_rows_are_stored_sorted():
    """With every row stored in (degree, id) order the variant coincides with the ordering itself,
    and the ordering does not depend on how rows are stored; on a star whose leaves are stored
    in reverse id order it numbers the leaves in that stored order."""
    for g in small_graphs(60, 300, 32) + [synth.c3_mesh(2000)]:
        gs = _rows_sorted_by_degree(g)
        exact = oracle.rcm(g.n, g.rowptr, g.colidx)
        assert np.array_equal(oracle.rcm(gs.n, gs.rowptr, gs.colidx), exact)
        assert np.array_equal(oracle.rcm(gs.n, gs.rowptr, gs.colidx, row_order=1), exact)
    # star: centre 0, leaves 1..5 stored as 5, 4, 3, 2, 1 in the centre's row
    rp = np.array([0, 5, 6, 7, 8, 9, 10], np.int32)
    ci = np.array([5, 4, 3, 2, 1, 0, 0, 0, 0, 0], np.int32)
    # start = leaf 1 (degree 1, lowest id); its sweep ends at leaf 2 (min (degree, id) of the last
    # level), which the second sweep does not beat: root 2, then the centre, then the other
    # leaves in the centre's stored order 5, 4, 3, 1; reversed.
    assert list(oracle.rcm(6, rp, ci, row_order=1)) == [1, 3, 4, 5, 0, 2]
    assert list(oracle.rcm(6, rp, ci)) == [5, 4, 3, 1, 0, 2]


def test_alg4_level_form_matches_alg2():
    for g in small_graphs(120, 300, 25, connected=True) + [synth.grid((9, 14), seed=3)]:
        deg = oracle.degrees(g.n, g.rowptr, g.colidx).astype(np.int64)
        r0 = int(np.lexsort((np.arange(g.n), deg))[0])
        assert alg4_level_synchronous(g, deg, r0) == oracle.pseudo_peripheral(g.n, g.rowptr, g.colidx, r0)


# ------------------------------------------------------------------------------------------
# special cases and reported quantities


def test_special_cases():
    # n = 0, n = 1, all isolated, a self-loop only
    assert len(oracle.rcm(0, np.zeros(1, np.int32), np.zeros(0, np.int32))) == 0
    assert list(oracle.rcm(1, np.array([0, 0], np.int32), np.zeros(0, np.int32))) == [0]
    assert list(oracle.rcm(1, np.array([0, 1], np.int32), np.array([0], np.int32))) == [0]
    g = synth.csr_from_edges(5, [], [])
    # isolated vertices are components of their own, numbered first in id order, so placed last
    assert list(rcm_of(g)) == [4, 3, 2, 1, 0]


def test_diagonal_entries_do_not_change_the_order():
    """Diagonal entries carry no edge and do not count in the degree (on all rows or on some)."""
    for i in range(30):
        g = synth.random_graph(80, 150, [26, i])
        some = synth.rng_for([26, i, 1]).choice(80, 30, replace=False)
        for diag in (True, some):
            gd = synth.csr_from_edges(80, *_edges(g), diagonal=diag)
            assert np.array_equal(rcm_of(g), rcm_of(gd))


def _edges(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    return rows, g.colidx


def test_components_numbered_in_start_order_and_reversed_once():
    """Components are processed in start-rule order (lowest (degree, id) vertex first) with labels
    continuing, then the whole sequence is reversed, so the first component ends up last."""
    for g in small_graphs(60, 200, 27, connected=False):
        adj = adjacency(g)
        deg = [len(a) for a in adj]
        seq = list(rcm_of(g)[::-1])
        comps = components(adj)
        comp_of = {v: i for i, c in enumerate(comps) for v in c}
        blocks = []
        for v in seq:
            if not blocks or comp_of[v] != blocks[-1]:
                blocks.append(comp_of[v])
        assert len(blocks) == len(comps)  # each component contiguous
        keys = [min((deg[v], v) for v in comps[b]) for b in blocks]
        assert keys == sorted(keys)


def test_bandwidth_profile_matches_definition():
    for g in small_graphs(50, 150, 28):
        p = rcm_of(g)
        assert oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, p) == bandwidth_profile_py(adjacency(g), p)
        ident = np.arange(g.n, dtype=np.int32)
        assert oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, ident) == bandwidth_profile_py(adjacency(g), ident)


def test_bad_csr_is_rejected():
    assert oracle.check_csr(2, np.array([0, 2, 1], np.int32), np.array([1, 0], np.int32)) == -2
    assert oracle.check_csr(2, np.array([0, 1, 2], np.int32), np.array([1, 2], np.int32)) == -2
    assert oracle.check_csr(2, np.array([1, 1, 2], np.int32), np.array([1, 0], np.int32)) == -2
    with pytest.raises(ValueError):
        oracle.rcm(2, np.array([0, 1, 2], np.int32), np.array([1, -1], np.int32))


def test_quality_no_worse_than_scipy_by_a_wide_margin():
    """Quality sanity only (scipy's start and tie rules differ, so there is no parity)."""
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import reverse_cuthill_mckee

    for g in [synth.c1_grid2d(), synth.grid((20, 20, 20), seed=5), synth.c3_mesh(20000)]:
        A = sp.csr_matrix((np.ones(g.nnz), g.colidx, g.rowptr), shape=(g.n, g.n))
        ps = reverse_cuthill_mckee(A, symmetric_mode=True)
        adj = adjacency(g)
        bw_s, _ = bandwidth_profile_py(adj, ps)
        bw_o, _ = oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, rcm_of(g))
        assert bw_o <= 1.5 * bw_s + 4


# ------------------------------------------------------------------------------------------
# golden fixtures


def read_golden(name):
    data = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split(":", 1)
            data.setdefault(k.strip(), []).extend(v.split())
    return data


def golden_graph(d):
    """The fixture's pattern: an undirected edge list (rows sorted by id), or explicit stored rows
    (rowptr / colidx, kept in the order the fixture gives them)."""
    n = int(d["n"][0])
    if "rowptr" in d:
        return synth.Csr(n, np.array(d["rowptr"], dtype=np.int32), np.array(d["colidx"], dtype=np.int32))
    e = np.array(d.get("edges", []), dtype=np.int64).reshape(-1, 2)
    return synth.csr_from_edges(n, e[:, 0], e[:, 1])


HAND_WORKED = ["star6.txt", "grid3x3.txt", "path6.txt", "two_components.txt"]
# rows with more than 32 neighbours to number, stored out of id order
WIDE_ROWS = ["star41_shuffled.txt", "star41_reversed.txt", "broom78.txt"]


@pytest.mark.parametrize("name", HAND_WORKED + WIDE_ROWS)
def test_hand_worked_fixtures(name):
    d = read_golden(name)
    g = golden_graph(d)
    p = rcm_of(g)
    assert list(p) == [int(x) for x in d["perm"]]
    if "bandwidth" in d:
        assert oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, p) == (int(d["bandwidth"][0]), int(d["profile"][0]))


@pytest.mark.parametrize("name", WIDE_ROWS)
def test_wide_row_fixtures_are_symmetric_stored_out_of_order(name):
    """The wide-row fixtures are valid patterns (symmetric, no duplicates or diagonal), have a row
    with more than 32 entries, and store at least one row out of ascending id order, so that they
    reach the oracle's branch for long neighbour lists with unsorted input."""
    g = golden_graph(read_golden(name))
    pairs = set()
    unsorted = False
    for v in range(g.n):
        row = [int(w) for w in g.colidx[g.rowptr[v]:g.rowptr[v + 1]]]
        assert len(set(row)) == len(row) and v not in row
        unsorted |= row != sorted(row)
        pairs |= {(v, w) for w in row}
    assert all((w, v) in pairs for v, w in pairs)
    assert np.diff(g.rowptr).max() > 33 and unsorted


@pytest.mark.parametrize("name", WIDE_ROWS)
def test_wide_row_fixtures_match_level_form(name):
    """The same fixtures through the independent level-synchronous restatement of Alg. 3/Alg. 4
    (numpy lexsort, not the oracle's sort)."""
    g = golden_graph(read_golden(name))
    deg = oracle.degrees(g.n, g.rowptr, g.colidx).astype(np.int64)
    r0 = int(np.lexsort((np.arange(g.n), deg))[0])
    root, _, _ = alg4_level_synchronous(g, deg, r0)
    R = np.full(g.n, -1, dtype=np.int64)
    assert alg3_level_synchronous(g, deg, root, 0, R) == g.n
    seq = np.empty(g.n, dtype=np.int64)
    seq[R] = np.arange(g.n)
    assert list(seq[::-1]) == [int(x) for x in read_golden(name)["perm"]]


def test_regression_fixture_written_from_oracle():
    """tests/golden/oracle_regression.txt is written by tests/golden/make_golden.py (oracle only)."""
    import hashlib
    d = read_golden("oracle_regression.txt")
    for name, digest, bw, prof in zip(d["case"][0::4], d["case"][1::4], d["case"][2::4], d["case"][3::4]):
        g = _golden_case(name)
        p = rcm_of(g)
        assert hashlib.sha256(p.astype("<i4").tobytes()).hexdigest()[:16] == digest
        assert oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, p) == (int(bw), int(prof))


def _golden_case(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.CASES[name]()


# ------------------------------------------------------------------------------------------
# mutants: a plausible mistake planted in the oracle must fail at least one pin

MUTANTS = {
    "tie_break_highest_id": ("    return a < b;\n}", "    return a > b;\n}"),
    "no_reversal": ("perm[n - 1 - i] = seq[i];", "perm[i] = seq[i];"),
    "degree_counts_diagonal": ("if (colidx[k] != v) d++;", "d++;"),
    "children_by_descending_degree": ("while (j >= 0 && before(deg, x, a[j]))", "while (j >= 0 && before(deg, a[j], x))"),
    "last_level_off_by_one": ("*last = i;\n    return tail;", "*last = i > 0 ? i - 1 : 0;\n    return tail;"),
    "one_sweep_only": ("    while (ecc_r > nlvl) {", "    while (0) {"),
    "bandwidth_f_starts_at_zero": ("int32_t v = perm[i], f = i;", "int32_t v = perm[i], f = 0;"),
    "sort_free_still_sorts": ("        if (!by_degree) {", "        if (0) {"),
    # the branch that sorts more than 32 neighbours at once (packed (degree, id) keys)
    "wide_rows_tie_break_highest_id": (
        "                keys[i] = ((uint64_t)(uint32_t)deg[scratch[i]] << 32) | (uint32_t)scratch[i];\n"
        "            qsort(keys, (size_t)found, sizeof(uint64_t), cmp_key);\n"
        "            for (int32_t i = 0; i < found; ++i) scratch[i] = (int32_t)(keys[i] & 0xffffffffu);",
        "                keys[i] = ((uint64_t)(uint32_t)deg[scratch[i]] << 32) | (uint32_t)(0x7fffffff - scratch[i]);\n"
        "            qsort(keys, (size_t)found, sizeof(uint64_t), cmp_key);\n"
        "            for (int32_t i = 0; i < found; ++i) scratch[i] = 0x7fffffff - (int32_t)(keys[i] & 0xffffffffu);"),
    "wide_rows_by_id_only": ("keys[i] = ((uint64_t)(uint32_t)deg[scratch[i]] << 32) | (uint32_t)scratch[i];",
                             "keys[i] = (uint64_t)(uint32_t)scratch[i];"),
    "start_at_highest_degree": ("while (label[start_order[cursor]] >= 0) cursor++;\n        int32_t r0 = start_order[cursor];",
                                "int32_t r0 = -1;\n        for (int32_t c = n - 1; c >= 0; --c) if (label[start_order[c]] < 0) { r0 = start_order[c]; break; }"),
}


def _pins_with(lib):
    """A compact set of the pins above, run against a given oracle build. Returns True if all pass."""
    try:
        for n in range(2, 12):
            g = synth.path(n)
            p = oracle.rcm(g.n, g.rowptr, g.colidx, lib=lib)
            if not np.array_equal(p, np.arange(n)):
                return False
        for k in range(3, 9):
            g = synth.grid((k, k), seed=[k, 0])
            p = oracle.rcm(g.n, g.rowptr, g.colidx, lib=lib)
            if oracle.bandwidth_profile(g.n, g.rowptr, g.colidx, p, lib=lib) != bandwidth_profile_py(adjacency(g), p):
                return False
            if bandwidth_profile_py(adjacency(g), p)[0] != k:
                return False
        for g in small_graphs(60, 10, 29):
            adj = adjacency(g)
            deg = np.array([len(a) for a in adj], dtype=np.int64)
            sols = enumerate_cm_sequences(adj, deg, george_liu_roots(adj, deg))
            p = oracle.rcm(g.n, g.rowptr, g.colidx, lib=lib)
            if len(sols) != 1 or list(p[::-1]) != sols[0]:
                return False
        for name in HAND_WORKED + WIDE_ROWS:
            d = read_golden(name)
            g = golden_graph(d)
            if list(oracle.rcm(g.n, g.rowptr, g.colidx, lib=lib)) != [int(x) for x in d["perm"]]:
                return False
        rp = np.array([0, 5, 6, 7, 8, 9, 10], np.int32)          # the stored-order star above
        ci = np.array([5, 4, 3, 2, 1, 0, 0, 0, 0, 0], np.int32)
        if list(oracle.rcm(6, rp, ci, lib=lib, row_order=1)) != [1, 3, 4, 5, 0, 2]:
            return False
        for i in range(10):
            g = synth.random_graph(40, 70, [30, i])
            gd = synth.csr_from_edges(40, *_edges(g), diagonal=np.arange(0, 40, 3))
            if not np.array_equal(oracle.rcm(g.n, g.rowptr, g.colidx, lib=lib),
                                  oracle.rcm(gd.n, gd.rowptr, gd.colidx, lib=lib)):
                return False
    except Exception:
        return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(mutant, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "rcm_oracle.c")).read()
    old, new = MUTANTS[mutant]
    assert src.count(old) == 1, f"mutation site for {mutant} not found exactly once"
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = oracle.load(oracle.build(str(msrc), str(tmp_path / "libmutant.so")))
    assert not _pins_with(lib), f"mutant {mutant} passed the pins"


def test_unmutated_oracle_passes_compact_pins():
    assert _pins_with(oracle.load())
