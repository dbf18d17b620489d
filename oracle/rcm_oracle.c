/*
 * rcm_oracle.c -- plain serial CPU reference for the Reverse Cuthill-McKee ordering of
 * Azad, Jacquelin, Buluc and Ng, "The Reverse Cuthill-McKee Algorithm in Distributed-Memory".
 *
 * TEST INFRASTRUCTURE ONLY. This file is the oracle that the GPU library is checked against.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never calls it and shares no code, header or table with it.
 *
 * It follows the serial algorithms of Sec. II-A step by step, with fixed tie rules:
 *   - degree D[v] = number of off-diagonal entries in row v (diagonal entries carry no edge);
 *   - components are processed one after another (Sec. III-B: Alg. 3 is invoked once per
 *     connected component); each starts from the lowest-id vertex of minimum degree among the
 *     vertices not yet numbered (the "arbitrary vertex" of Alg. 2, fixed);
 *   - pseudo-peripheral search = Alg. 2 (George-Liu): BFS from r, move to the lowest-id
 *     minimum-degree vertex of the last level, repeat while the eccentricity grows strictly;
 *     the root is the last vertex swept;
 *   - Cuthill-McKee labelling = Alg. 1: vertices are taken in label order, and the unnumbered
 *     neighbours of each get the next labels in increasing (degree, id);
 *   - labels continue across components, and the whole sequence is reversed once at the end
 *     (Alg. 1 last line, Alg. 3 "return R in the reverse order").
 * Output: perm[k] = original vertex placed at new position k, so (P A P^T)_{ij} = A_{perm[i],perm[j]}.
 *
 * oracle_rcm_ex(..., row_order = 1) is the sort-free variant of the paper's conclusion (no sort of
 * a level beyond its parent order): the same steps, but each vertex's unnumbered neighbours are
 * numbered in the order its row stores them instead of by (degree, id).
 *
 * All arithmetic is integer. Functions are reentrant (no globals), so callers may run one graph
 * per thread.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_ARG (-1)
#define ORACLE_BAD_CSR (-2)
#define ORACLE_NO_MEM (-3)

/* Structural checks of the input pattern: rowptr[0] = 0, rowptr non-decreasing, 0 <= colidx < n. */
int oracle_check_csr(int32_t n, const int32_t *rowptr, const int32_t *colidx)
{
    if (n < 0) return ORACLE_BAD_ARG;
    if (n == 0) return ORACLE_OK;
    if (!rowptr) return ORACLE_BAD_ARG;
    if (rowptr[0] != 0) return ORACLE_BAD_CSR;
    for (int32_t v = 0; v < n; ++v)
        if (rowptr[v + 1] < rowptr[v]) return ORACLE_BAD_CSR;
    if (rowptr[n] > 0 && !colidx) return ORACLE_BAD_ARG;
    for (int64_t k = 0; k < rowptr[n]; ++k)
        if (colidx[k] < 0 || colidx[k] >= n) return ORACLE_BAD_CSR;
    return ORACLE_OK;
}

/* D[v]: off-diagonal entries of row v (the degree vector that Alg. 3 and Alg. 4 take as input). */
void oracle_degrees(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *deg)
{
    for (int32_t v = 0; v < n; ++v) {
        int32_t d = 0;
        for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k)
            if (colidx[k] != v) d++;
        deg[v] = d;
    }
}

/* The (degree, id) order used for every tie: a before b iff (deg a, a) < (deg b, b). */
static int before(const int32_t *deg, int32_t a, int32_t b)
{
    if (deg[a] != deg[b]) return deg[a] < deg[b];
    return a < b;
}

/*
 * Rooted level structure L(r) = {L_0, ..., L_ecc} (Sec. II-A) by breadth-first search.
 * lvl[] must be -1 on entry for every vertex of r's component; on return it holds the level of
 * each reached vertex. queue receives the reached vertices level by level. Returns the number of
 * reached vertices; *ecc = index of the last level; *last = queue index where the last level starts.
 */
static int32_t level_structure(const int32_t *rowptr, const int32_t *colidx, int32_t r,
                               int32_t *lvl, int32_t *queue, int32_t *ecc, int32_t *last)
{
    int32_t head = 0, tail = 0;
    lvl[r] = 0;
    queue[tail++] = r;
    *last = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            int32_t w = colidx[k];
            if (lvl[w] < 0) {
                lvl[w] = lvl[u] + 1;
                queue[tail++] = w;
            }
        }
    }
    *ecc = lvl[queue[tail - 1]];
    int32_t i = tail - 1;
    while (i > 0 && lvl[queue[i - 1]] == *ecc) --i;
    *last = i;
    return tail;
}

static void clear_levels(int32_t *lvl, const int32_t *queue, int32_t count)
{
    for (int32_t i = 0; i < count; ++i) lvl[queue[i]] = -1;
}

/*
 * Alg. 2 (George-Liu pseudo-peripheral vertex), starting at r0:
 *   L(r) <- level structure of r;  nlvl <- ecc(r) - 1
 *   while ecc(r) > nlvl:  nlvl <- ecc(r); v <- minimum-degree vertex of the last level
 *                         (lowest id among equal degrees); L(v) <- level structure; r <- v
 * Returns the final r. *sweeps = number of level structures computed, *ecc_out = ecc of the root.
 * lvl must be all -1 on r0's component on entry and is restored to -1 on return.
 */
static int32_t pseudo_peripheral(const int32_t *rowptr, const int32_t *colidx, const int32_t *deg,
                                 int32_t r0, int32_t *lvl, int32_t *queue,
                                 int32_t *sweeps, int32_t *ecc_out)
{
    int32_t r = r0, ecc_r, last;
    int32_t reached = level_structure(rowptr, colidx, r, lvl, queue, &ecc_r, &last);
    int32_t nlvl = ecc_r - 1;
    int32_t count = 1;
    while (ecc_r > nlvl) {
        nlvl = ecc_r;
        int32_t v = queue[last];
        for (int32_t i = last + 1; i < reached; ++i)
            if (before(deg, queue[i], v)) v = queue[i];
        clear_levels(lvl, queue, reached);
        reached = level_structure(rowptr, colidx, v, lvl, queue, &ecc_r, &last);
        count++;
        r = v;
    }
    clear_levels(lvl, queue, reached);
    *sweeps = count;
    *ecc_out = ecc_r;
    return r;
}

/* Exported for tests: the pseudo-peripheral root found from r0, the number of sweeps and ecc(root). */
int oracle_pseudo_peripheral(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t r0,
                             int32_t *out3)
{
    int rc = oracle_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (r0 < 0 || r0 >= n) return ORACLE_BAD_ARG;
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *lvl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!deg || !lvl || !queue) { free(deg); free(lvl); free(queue); return ORACLE_NO_MEM; }
    oracle_degrees(n, rowptr, colidx, deg);
    for (int32_t v = 0; v < n; ++v) lvl[v] = -1;
    int32_t sweeps, ecc;
    out3[0] = pseudo_peripheral(rowptr, colidx, deg, r0, lvl, queue, &sweeps, &ecc);
    out3[1] = sweeps;
    out3[2] = ecc;
    free(deg); free(lvl); free(queue);
    return ORACLE_OK;
}

/* Insertion sort of a short list of vertices by (degree, id). */
static void sort_by_degree(int32_t *a, int32_t len, const int32_t *deg)
{
    for (int32_t i = 1; i < len; ++i) {
        int32_t x = a[i], j = i - 1;
        while (j >= 0 && before(deg, x, a[j])) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

static int cmp_key(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return (a > b) - (a < b);
}

/*
 * Alg. 1 (Cuthill-McKee labelling) from root, labels starting at nv:
 *   v_1 <- root; for i = 1, 2, ...: find the unnumbered neighbours of v_i and number them in
 *   increasing order of degree (ties by lowest id).
 * With by_degree = 0 (the sort-free variant the paper's conclusion proposes: the level is not
 * sorted beyond its parent order) the neighbours are numbered in the order the row stores them.
 * label[] is -1 for unnumbered vertices. seq[] receives the vertices in label order from index nv.
 * Returns the new nv.
 */
static int32_t cuthill_mckee(const int32_t *rowptr, const int32_t *colidx, const int32_t *deg,
                             int32_t root, int32_t nv, int32_t *label, int32_t *seq,
                             int32_t *scratch, uint64_t *keys, int by_degree)
{
    int32_t head = nv;
    label[root] = nv;
    seq[nv++] = root;
    while (head < nv) {
        int32_t u = seq[head++];
        int32_t found = 0;
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            int32_t w = colidx[k];
            if (w != u && label[w] < 0) {
                label[w] = -2; /* found in this row: exclude duplicates within the row */
                scratch[found++] = w;
            }
        }
        if (!by_degree) {
            /* stored order: nothing to sort */
        } else if (found <= 32) {
            sort_by_degree(scratch, found, deg);
        } else {
            for (int32_t i = 0; i < found; ++i)
                keys[i] = ((uint64_t)(uint32_t)deg[scratch[i]] << 32) | (uint32_t)scratch[i];
            qsort(keys, (size_t)found, sizeof(uint64_t), cmp_key);
            for (int32_t i = 0; i < found; ++i) scratch[i] = (int32_t)(keys[i] & 0xffffffffu);
        }
        for (int32_t i = 0; i < found; ++i) {
            label[scratch[i]] = nv;
            seq[nv++] = scratch[i];
        }
    }
    return nv;
}

/*
 * The full ordering. stats (may be NULL) receives int64[8]:
 *   [0] connected components, [1] BFS level structures computed (all sweeps of Alg. 2),
 *   [2] sum over components of ecc(root)+1 (levels of the labelled traversals),
 *   [3] largest ecc(root), [4] vertices of degree zero.
 */
int oracle_rcm_ex(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *perm, int64_t *stats,
                  int row_order)
{
    int rc = oracle_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    if (stats) memset(stats, 0, 8 * sizeof(int64_t));
    if (n == 0) return ORACLE_OK;
    if (!perm) return ORACLE_BAD_ARG;
    size_t sz = sizeof(int32_t) * (size_t)n;
    int32_t *deg = (int32_t *)malloc(sz), *label = (int32_t *)malloc(sz), *lvl = (int32_t *)malloc(sz);
    int32_t *queue = (int32_t *)malloc(sz), *seq = (int32_t *)malloc(sz), *scratch = (int32_t *)malloc(sz);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *start_order = (int32_t *)malloc(sz);
    if (!deg || !label || !lvl || !queue || !seq || !scratch || !keys || !start_order) {
        rc = ORACLE_NO_MEM;
        goto done;
    }
    oracle_degrees(n, rowptr, colidx, deg);
    /* All vertices in (degree, id) order: the start of each component is the first vertex of this
       list that is still unnumbered. */
    for (int32_t v = 0; v < n; ++v) keys[v] = ((uint64_t)(uint32_t)deg[v] << 32) | (uint32_t)v;
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_key);
    for (int32_t i = 0; i < n; ++i) start_order[i] = (int32_t)(keys[i] & 0xffffffffu);
    for (int32_t v = 0; v < n; ++v) { label[v] = -1; lvl[v] = -1; if (deg[v] == 0 && stats) stats[4]++; }

    int32_t nv = 0, cursor = 0;
    while (nv < n) {
        while (label[start_order[cursor]] >= 0) cursor++;
        int32_t r0 = start_order[cursor];
        int32_t sweeps, ecc;
        int32_t root = pseudo_peripheral(rowptr, colidx, deg, r0, lvl, queue, &sweeps, &ecc);
        nv = cuthill_mckee(rowptr, colidx, deg, root, nv, label, seq, scratch, keys, row_order == 0);
        if (stats) {
            stats[0] += 1;
            stats[1] += sweeps;
            stats[2] += (int64_t)ecc + 1;
            if (ecc > stats[3]) stats[3] = ecc;
        }
    }
    /* Reverse the Cuthill-McKee sequence once: w_i = v_{n-i+1}. */
    for (int32_t i = 0; i < n; ++i) perm[n - 1 - i] = seq[i];
    rc = ORACLE_OK;
done:
    free(deg); free(label); free(lvl); free(queue); free(seq); free(scratch); free(keys); free(start_order);
    return rc;
}

/* The ordering of Sec. II-A / III: children in (degree, id) order. */
int oracle_rcm(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *perm, int64_t *stats)
{
    return oracle_rcm_ex(n, rowptr, colidx, perm, stats, 0);
}

/*
 * Bandwidth and profile of P A P^T (Sec. II-A). For new row i with original vertex perm[i],
 * f_i = min(i, min{ pos[w] : w adjacent to perm[i] }) where pos is the inverse permutation;
 * beta_i = i - f_i; bandwidth = max beta_i; profile |Env| = sum beta_i.
 */
int oracle_bandwidth_profile(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *perm,
                             int64_t *bw, int64_t *profile)
{
    int rc = oracle_check_csr(n, rowptr, colidx);
    if (rc) return rc;
    *bw = 0;
    *profile = 0;
    if (n == 0) return ORACLE_OK;
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!pos) return ORACLE_NO_MEM;
    for (int32_t v = 0; v < n; ++v) pos[v] = -1;
    for (int32_t i = 0; i < n; ++i) {
        if (perm[i] < 0 || perm[i] >= n || pos[perm[i]] >= 0) { free(pos); return ORACLE_BAD_ARG; }
        pos[perm[i]] = i;
    }
    for (int32_t i = 0; i < n; ++i) {
        int32_t v = perm[i], f = i;
        for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k)
            if (pos[colidx[k]] < f) f = pos[colidx[k]];
        int64_t beta = (int64_t)i - f;
        if (beta > *bw) *bw = beta;
        *profile += beta;
    }
    free(pos);
    return ORACLE_OK;
}

/* Exported for tests: Alg. 1 labelling of root's component from a given root (labels from 0);
   vertices outside the component keep label -1. Returns the number of vertices labelled. */
int32_t oracle_cm_from_root(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t root,
                            int32_t *label)
{
    if (oracle_check_csr(n, rowptr, colidx) || root < 0 || root >= n) return -1;
    size_t sz = sizeof(int32_t) * (size_t)n;
    int32_t *deg = (int32_t *)malloc(sz), *seq = (int32_t *)malloc(sz), *scratch = (int32_t *)malloc(sz);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t count = -1;
    if (deg && seq && scratch && keys) {
        oracle_degrees(n, rowptr, colidx, deg);
        for (int32_t v = 0; v < n; ++v) label[v] = -1;
        count = cuthill_mckee(rowptr, colidx, deg, root, 0, label, seq, scratch, keys, 1);
    }
    free(deg); free(seq); free(scratch); free(keys);
    return count;
}
