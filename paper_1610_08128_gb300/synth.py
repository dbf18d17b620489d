"""Seeded synthetic sparsity patterns shaped like the paper's workloads.

This module only builds inputs: symmetric int32 CSR patterns (rowptr, colidx) and batches of them.
It holds none of the ordering method's arithmetic, and both the CUDA path and the serial CPU oracle
take their inputs from here.

The paper evaluates SuiteSparse matrices (Fig. 3, Table II) that are not available offline; these
generators stand in for their shapes (2D/3D meshes, the 1.2 M-row thermal2-like 2D mesh of Fig. 1,
high-diameter structural grids). Every generator is deterministic in its seed: numpy's PCG64 seeded
through ``SeedSequence``.

Conventions (Sec. III, graph of A): vertex v is row/column v; an undirected edge {i, j} appears as
both (i, j) and (j, i); there are no duplicate entries; diagonal entries appear only when asked for
(they carry no edge). Column indices inside a row are sorted ascending, except after
:func:`shuffle_rows` and in :func:`csr_from_rows`, which keep a given stored order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1610081280


def rng_for(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))


@dataclass
class Csr:
    """A symmetric sparsity pattern in int32 CSR (pattern only, no values)."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    colidx: np.ndarray  # int32[nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def offdiag_nnz(self) -> int:
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr.astype(np.int64)))
        return int(np.count_nonzero(rows != self.colidx))


def csr_from_edges(n: int, src, dst, diagonal: bool = False) -> Csr:
    """Symmetric CSR from an undirected edge list; duplicates and self pairs are dropped.

    With ``diagonal`` every row also stores its diagonal entry (a self-loop that carries no edge);
    an array of vertex ids stores the diagonal of those rows only.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    a = np.concatenate([src, dst])
    b = np.concatenate([dst, src])
    if diagonal is not False and diagonal is not None:
        d = np.arange(n, dtype=np.int64) if diagonal is True else np.unique(np.asarray(diagonal, np.int64))
        a = np.concatenate([a, d])
        b = np.concatenate([b, d])
    key = np.unique(a * n + b) if len(a) else np.zeros(0, dtype=np.int64)
    rows = key // n if n else key
    cols = key - rows * n if n else key
    rowptr = np.zeros(n + 1, dtype=np.int64)
    if n:
        rowptr[1:] = np.bincount(rows, minlength=n)
    rowptr = np.cumsum(rowptr)
    return Csr(n, rowptr.astype(np.int32), cols.astype(np.int32))


def permute(g: Csr, p: np.ndarray) -> Csr:
    """Relabel vertices: old vertex i becomes new vertex p[i]; rows and columns move together."""
    n = g.n
    p = np.asarray(p, dtype=np.int64)
    q = np.empty(n, dtype=np.int64)
    q[p] = np.arange(n, dtype=np.int64)  # q[new] = old
    lens = np.diff(g.rowptr.astype(np.int64))
    new_lens = lens[q]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(new_lens)
    # gather old rows in new-row order
    starts = g.rowptr[:-1].astype(np.int64)[q]
    total = int(rowptr[-1])
    seg = np.repeat(starts - rowptr[:-1], new_lens)
    src_pos = np.arange(total, dtype=np.int64) + seg
    cols = p[g.colidx.astype(np.int64)[src_pos]]
    # sort columns within each row
    rows = np.repeat(np.arange(n, dtype=np.int64), new_lens)
    order = np.lexsort((cols, rows))
    cols = cols[order]
    out = Csr(n, rowptr.astype(np.int32), cols.astype(np.int32), dict(g.meta))
    return out


def random_permutation(n: int, seed) -> np.ndarray:
    return rng_for(seed).permutation(n).astype(np.int64)


def shuffle_rows(g: Csr, seed) -> Csr:
    """The same pattern with the entries of every row stored in a seeded random order.

    A CSR pattern is a set of nonzeros per row (Sec. III-A); the order inside a row is free. The
    other generators store rows sorted by column id, which this undoes."""
    rng = rng_for(seed)
    lens = np.diff(g.rowptr.astype(np.int64))
    rows = np.repeat(np.arange(g.n, dtype=np.int64), lens)
    order = np.lexsort((rng.random(g.nnz), rows))
    meta = dict(g.meta)
    meta["row_shuffle"] = seed
    return Csr(g.n, g.rowptr.copy(), g.colidx[order].astype(np.int32), meta)


def csr_from_rows(rows) -> Csr:
    """CSR from explicit stored rows (a list of column lists), keeping each row's order as given."""
    lens = np.array([len(r) for r in rows], dtype=np.int64)
    rowptr = np.zeros(len(rows) + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lens)
    colidx = np.array([c for r in rows for c in r], dtype=np.int32)
    return Csr(len(rows), rowptr.astype(np.int32), colidx)


def power_law(n: int, avg_degree: float, gamma: float, seed) -> Csr:
    """Chung-Lu random graph with a power-law expected degree sequence.

    Vertex i (before the id permutation) gets weight w_i proportional to (i + i0)^(-1/(gamma-1)),
    scaled so the weights average ``avg_degree``; n * avg_degree / 2 edges are drawn with both
    endpoints chosen with probability proportional to weight (duplicates and self pairs dropped).
    A few hub rows hold thousands of entries, as in the scale-free matrices of circuit and network
    problems. Ids are permuted uniformly from the seed."""
    rng = rng_for(seed)
    i0 = 10.0  # keeps the largest weight finite and the top hubs a few thousand strong at n = 10^6
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))
    w *= avg_degree * n / w.sum()
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(n * avg_degree / 2))
    src = np.minimum(np.searchsorted(cdf, rng.random(m), side="right"), n - 1)
    dst = np.minimum(np.searchsorted(cdf, rng.random(m), side="right"), n - 1)
    g = csr_from_edges(n, src, dst)
    g = permute(g, rng.permutation(n))
    g.meta = {"kind": "power_law", "n": n, "avg_degree": avg_degree, "gamma": gamma, "seed": seed}
    return g


def _grid_natural(dims) -> Csr:
    """5-point (2D) / 7-point (3D) stencil pattern on a regular grid, natural C-order ids."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims)) if dims else 0
    ids = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(ids, dims)
    strides = [int(np.prod(dims[a + 1:])) for a in range(len(dims))]
    cols = []
    for ax in range(len(dims)):
        c = coords[ax]
        s = strides[ax]
        cols.append(np.where(c > 0, ids - s, -1))
        cols.append(np.where(c < dims[ax] - 1, ids + s, -1))
    nb = np.stack(cols, axis=1) if cols else np.zeros((n, 0), dtype=np.int64)
    return _csr_from_padded(n, nb)


def _csr_from_padded(n: int, nb: np.ndarray) -> Csr:
    """Rows given as a padded (n, w) array of neighbour ids with -1 holes."""
    big = np.iinfo(np.int64).max
    nbs = np.where(nb < 0, big, nb)
    nbs.sort(axis=1)
    valid = nbs != big
    lens = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lens)
    colidx = nbs[valid]
    return Csr(n, rowptr.astype(np.int32), colidx.astype(np.int32))


def grid(dims, seed=None) -> Csr:
    """Regular grid (2D 5-point or 3D 7-point stencil). With a seed, vertex ids are permuted uniformly."""
    g = _grid_natural(dims)
    g.meta = {"kind": f"grid{len(dims)}d", "dims": list(map(int, dims)), "seed": seed}
    if seed is not None:
        g = permute(g, random_permutation(g.n, seed))
    return g


def _padded_permute(nb: np.ndarray, p: np.ndarray) -> np.ndarray:
    q = np.empty(len(p), dtype=np.int64)
    q[p] = np.arange(len(p), dtype=np.int64)
    rows = nb[q]
    return np.where(rows >= 0, p[np.maximum(rows, 0)], -1)


def grid_fast(dims, seed=None) -> Csr:
    """Same pattern as :func:`grid`, built directly in permuted order (lower peak memory for 192^3)."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    ids = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(ids, dims)
    strides = [int(np.prod(dims[a + 1:])) for a in range(len(dims))]
    cols = []
    for ax in range(len(dims)):
        c = coords[ax]
        s = strides[ax]
        cols.append(np.where(c > 0, ids - s, -1))
        cols.append(np.where(c < dims[ax] - 1, ids + s, -1))
    del coords
    nb = np.stack(cols, axis=1)
    del cols
    if seed is not None:
        nb = _padded_permute(nb, random_permutation(n, seed))
    g = _csr_from_padded(n, nb)
    g.meta = {"kind": f"grid{len(dims)}d", "dims": list(dims), "seed": seed}
    return g


def path(n: int, seed=None) -> Csr:
    g = csr_from_edges(n, np.arange(n - 1), np.arange(1, n)) if n > 1 else csr_from_edges(n, [], [])
    g.meta = {"kind": "path", "seed": seed}
    if seed is not None:
        g = permute(g, random_permutation(n, seed))
    return g


def circulant(n: int, offsets, seed=None) -> Csr:
    """Circulant pattern: vertex v joined to v + k and v - k (mod n) for every k in ``offsets``, so
    each row holds exactly 2 * len(offsets) entries when n > 2 * max(offsets). With a seed, ids are
    permuted uniformly."""
    src = np.repeat(np.arange(n, dtype=np.int64), len(offsets))
    dst = (src + np.tile(np.asarray(offsets, dtype=np.int64), n)) % n
    g = csr_from_edges(n, src, dst)
    g.meta = {"kind": "circulant", "offsets": list(map(int, offsets)), "seed": seed}
    if seed is not None:
        g = permute(g, random_permutation(n, seed))
    return g


def random_graph(n: int, m: int, seed, connected: bool = False, diagonal: bool = False) -> Csr:
    """Erdos-Renyi-like pattern with m undirected edges (duplicates dropped); optionally a random
    spanning tree is added first so the graph is connected."""
    rng = rng_for(seed)
    src, dst = [], []
    if connected and n > 1:
        order = rng.permutation(n)
        parents = np.array([order[rng.integers(0, i)] for i in range(1, n)], dtype=np.int64)
        src.append(order[1:])
        dst.append(parents)
    if m > 0 and n > 1:
        src.append(rng.integers(0, n, m))
        dst.append(rng.integers(0, n, m))
    s = np.concatenate(src) if src else np.zeros(0, np.int64)
    d = np.concatenate(dst) if dst else np.zeros(0, np.int64)
    g = csr_from_edges(n, s, d, diagonal=diagonal)
    g.meta = {"kind": "random", "n": n, "m": m, "seed": seed}
    return g


def random_tree(n: int, seed) -> Csr:
    rng = rng_for(seed)
    if n <= 1:
        return csr_from_edges(n, [], [])
    order = rng.permutation(n)
    parents = np.array([order[rng.integers(0, i)] for i in range(1, n)], dtype=np.int64)
    g = csr_from_edges(n, order[1:], parents)
    g.meta = {"kind": "tree", "seed": seed}
    return g


def _strip_regions(pts: np.ndarray, regions: int, width: float, rng) -> tuple[np.ndarray, np.ndarray]:
    """Cut the unit square into ``regions`` slabs by removing regions-1 parallel strips of the given
    width (all vertical or all horizontal, chosen by the seed). Returns (keep mask, region id)."""
    axis = int(rng.integers(0, 2))
    x = pts[:, axis]
    if regions <= 1:
        return np.ones(len(pts), bool), np.zeros(len(pts), np.int64)
    # strip centres: sorted, separated so every slab is non-empty with margin
    while True:
        centres = np.sort(rng.uniform(width, 1.0 - width, regions - 1))
        gaps = np.diff(np.concatenate([[0.0], centres, [1.0]]))
        if gaps.min() > 4 * width:
            break
    keep = np.ones(len(pts), bool)
    for c in centres:
        keep &= np.abs(x - c) > width / 2
    region = np.searchsorted(centres, x)
    return keep, region


def knn_mesh(npts: int, k: int, seed, regions: int = 1, strip_width: float = 0.002,
             stitch: bool = False, diagonal: bool = False) -> Csr:
    """2D random geometric mesh: ``npts`` points uniform in the unit square, each joined to its k
    nearest neighbours, symmetrised. With ``regions`` > 1, points inside regions-1 random strips are
    removed and edges across strips are dropped. With ``stitch``, each region's Euclidean minimum
    spanning tree (from its Delaunay triangulation) is added, so the graph has exactly ``regions``
    connected components. Vertex ids are permuted uniformly from the seed."""
    from scipy.spatial import cKDTree

    rng = rng_for(seed)
    pts = rng.random((npts, 2))
    keep, region = _strip_regions(pts, regions, strip_width, rng)
    pts = pts[keep]
    region = region[keep]
    n = len(pts)
    src_l, dst_l = [], []
    if n > 1:
        kk = min(k, n - 1)
        tree = cKDTree(pts)
        _, nbr = tree.query(pts, kk + 1)
        nbr = np.asarray(nbr).reshape(n, kk + 1)[:, 1:]
        s = np.repeat(np.arange(n, dtype=np.int64), kk)
        d = nbr.reshape(-1).astype(np.int64)
        same = region[s] == region[d]
        src_l.append(s[same])
        dst_l.append(d[same])
    if stitch and n > 1:
        for rid in np.unique(region):
            members = np.nonzero(region == rid)[0]
            if len(members) < 2:
                continue
            s, d = _emst_edges(pts[members])
            src_l.append(members[s])
            dst_l.append(members[d])
    src = np.concatenate(src_l) if src_l else np.zeros(0, np.int64)
    dst = np.concatenate(dst_l) if dst_l else np.zeros(0, np.int64)
    g = csr_from_edges(n, src, dst, diagonal=diagonal)
    g = permute(g, rng.permutation(n))
    g.meta = {"kind": "knn", "k": k, "npts": npts, "regions": regions, "stitch": stitch,
              "diagonal": diagonal, "seed": seed}
    return g


def _emst_edges(p: np.ndarray):
    """Euclidean minimum spanning tree edges of a point set (Delaunay graph + MST)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    m = len(p)
    if m == 2:
        return np.array([0]), np.array([1])
    if m == 3:
        return np.array([0, 1]), np.array([1, 2])
    try:
        from scipy.spatial import Delaunay

        tri = Delaunay(p).simplices
        e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [0, 2]]]).astype(np.int64)
    except Exception:  # degenerate (collinear) sets: chain sorted points
        o = np.argsort(p[:, 0] + 1e-9 * p[:, 1])
        return o[:-1], o[1:]
    e = np.unique(np.sort(e, axis=1), axis=0)
    w = np.sqrt(((p[e[:, 0]] - p[e[:, 1]]) ** 2).sum(1)) + 1e-300
    t = minimum_spanning_tree(coo_matrix((w, (e[:, 0], e[:, 1])), shape=(m, m))).tocoo()
    return t.row.astype(np.int64), t.col.astype(np.int64)


# ----------------------------------------------------------------------------------------------
# The five workloads


def c1_grid2d(seed_offset: int = 0) -> Csr:
    """64x64 2D 5-point grid, ids permuted (4,096 vertices, 16,128 off-diagonal entries)."""
    return grid((64, 64), seed=SEED_BASE + 1 + 1000 * seed_offset)


def c2_grid3d(side: int = 192, seed_offset: int = 0) -> Csr:
    """side^3 3D 7-point grid, ids permuted (192^3: 7,077,888 vertices, 42,246,144 entries)."""
    return grid_fast((side, side, side), seed=SEED_BASE + 2 + 1000 * seed_offset)


def c3_mesh(npts: int = 1_200_000, seed_offset: int = 0, stitch: bool = True) -> Csr:
    """1.2 M-point 2D kNN(2) mesh with the diagonal stored, cut into 1-20 regions by strips.
    ``stitch`` adds each region's Euclidean MST so there is exactly one component per region;
    without it the raw symmetrised kNN(2) graph has tens of thousands of components."""
    seed = SEED_BASE + 3 + 1000 * seed_offset
    regions = int(rng_for([seed, 7]).integers(1, 21))
    return knn_mesh(npts, 2, seed, regions=regions, stitch=stitch, diagonal=True)


@dataclass
class Batch:
    """G graphs concatenated block-diagonally: vertex offsets goff[G+1] (int64), one global CSR whose
    column ids are global; graph g owns rows goff[g]..goff[g+1]-1."""

    goff: np.ndarray
    rowptr: np.ndarray
    colidx: np.ndarray
    graphs: list

    @property
    def G(self) -> int:
        return len(self.goff) - 1

    @property
    def n(self) -> int:
        return int(self.goff[-1])


def batch_graph(kind: int, n: int, seed) -> Csr:
    """One member of the batched/served mix: 0 = 2D grid (r = round(sqrt n), c = round(n/r)),
    1 = 3D grid (a = round(cbrt n), a x a x round(n/a^2)), 2 = 2D kNN(k=3) mesh of n points."""
    if kind == 0:
        r = max(1, int(round(math.sqrt(n))))
        c = max(1, int(round(n / r)))
        return grid((r, c), seed=seed)
    if kind == 1:
        a = max(1, int(round(n ** (1.0 / 3.0))))
        c = max(1, int(round(n / (a * a))))
        return grid((a, a, c), seed=seed)
    return knn_mesh(n, 3, seed)


def concat(graphs) -> Batch:
    sizes = np.array([g.n for g in graphs], dtype=np.int64)
    goff = np.zeros(len(graphs) + 1, dtype=np.int64)
    goff[1:] = np.cumsum(sizes)
    nnzs = np.array([g.nnz for g in graphs], dtype=np.int64)
    eoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    eoff[1:] = np.cumsum(nnzs)
    if eoff[-1] >= 2**31:
        raise ValueError("batch has 2^31 or more entries; int32 rowptr cannot index it")
    rowptr = np.empty(int(goff[-1]) + 1, dtype=np.int32)
    colidx = np.empty(int(eoff[-1]), dtype=np.int32)
    for g, gr in enumerate(graphs):
        a, b = int(goff[g]), int(goff[g + 1])
        rowptr[a:b] = gr.rowptr[:-1] + eoff[g]
        colidx[eoff[g]:eoff[g + 1]] = gr.colidx + goff[g]
    rowptr[-1] = eoff[-1]
    return Batch(goff, rowptr, colidx, list(graphs))


def mix_sizes(count: int, lo: float, hi: float, seed) -> tuple[np.ndarray, np.ndarray]:
    """Log-uniform vertex counts in [lo, hi] and generator kinds uniform over {0, 1, 2}."""
    rng = rng_for(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), count)).round().astype(np.int64)
    kinds = rng.integers(0, 3, count)
    return sizes, kinds


def _make_graphs(specs):
    return [batch_graph(k, s, seed) for k, s, seed in specs]


def make_graphs(specs, workers: int = 0):
    """batch_graph for every (kind, n, seed) spec; with workers > 1 the specs are split over a
    process pool started with 'spawn' (safe in processes that already use the GPU)."""
    specs = list(specs)
    if workers <= 1 or len(specs) < 64:
        return _make_graphs(specs)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    chunks = [specs[i::workers] for i in range(workers)]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_make_graphs, chunks))
    out = [None] * len(specs)
    for w, part in enumerate(parts):
        out[w::workers] = part
    return out


def default_workers() -> int:
    import os

    return max(1, min(32, len(os.sched_getaffinity(0))))


def c4_specs(G: int = 10_000, nmin: int = 100, nmax: int = 50_000, seed_offset: int = 0):
    """The (kind, n, seed) of every graph of the batched workload, without building any."""
    base = SEED_BASE + 4 + 1000 * seed_offset
    sizes, kinds = mix_sizes(G, nmin, nmax, base)
    return [(int(k), int(s), [base, i]) for i, (k, s) in enumerate(zip(kinds, sizes))]


def c4_batch(G: int = 10_000, nmin: int = 100, nmax: int = 50_000, seed_offset: int = 0, workers: int = 1,
             indices=None) -> Batch:
    """G independent graphs, vertex counts log-uniform in [nmin, nmax], kind uniform over
    {2D grid, 3D grid, kNN(3) mesh}, ids permuted per graph, concatenated block-diagonally.
    With ``indices``, only those graphs of the G (in that order): one rank's share of the batch."""
    specs = c4_specs(G, nmin, nmax, seed_offset)
    if indices is not None:
        specs = [specs[i] for i in indices]
    return concat(make_graphs(specs, workers))


def c5_trace(requests: int = 4000, rate_per_s: float = 2000.0, pool: int = 256,
             nmin: float = 1e3, nmax: float = 4e6, seed_offset: int = 0, workers: int = 1):
    """Serving workload: Poisson arrival times (mean gap 1/rate) over ``requests`` requests, each
    naming one graph of a pool of ``pool`` pre-generated graphs with log-uniform sizes in
    [nmin, nmax] from the three batch generators. Returns (arrival_s, pool_index, pool graphs)."""
    base = SEED_BASE + 5 + 1000 * seed_offset
    sizes, kinds = mix_sizes(pool, nmin, nmax, [base, 1])
    specs = [(int(k), int(s), [base, 2, i]) for i, (k, s) in enumerate(zip(kinds, sizes))]
    graphs = make_graphs(specs, workers)
    rng = rng_for([base, 3])
    gaps = rng.exponential(1.0 / rate_per_s, requests)
    arrival = np.cumsum(gaps) - gaps[0]
    which = rng.integers(0, pool, requests)
    return arrival, which, graphs
