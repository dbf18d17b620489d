// rcm_engine.cuh -- the device-side RCM engine: start vertex, pseudo-peripheral sweeps and the
// labelled level loop, generic over the executor that runs it.
//
//   kCtaOnly = false : one graph, all CTAs of a cooperative persistent grid. Levels whose frontier
//                      is small run on CTA 0 alone (CTA barriers, frontier in shared memory) while
//                      the other CTAs wait at the next exchange; wide levels use the whole grid.
//   kCtaOnly = true  : one graph per CTA (batched engine); every level uses CTA barriers only.
//
// Per component (Sec. III-B: Alg. 3 once per connected component, in start-rule order):
//   1. start r0 = lowest-id vertex of minimum degree not yet numbered (min of packed
//      (degree, id) keys);
//   2. sweep 1: levels-only BFS from r0 (the level structure of Alg. 2 / the do-while of Alg. 4);
//      the next root is the min (degree, id) vertex of the last level (REDUCE in Alg. 4), taken
//      while that level is expanded;
//   3. sweeps 2.. (fused mode): labelled BFS (Alg. 3) from the current root. If its eccentricity
//      does not exceed the previous sweep's, the search stops (loop test of Alg. 2) and the labels
//      just computed are final, because the root is the last vertex swept. Otherwise the labels
//      are discarded and the next sweep starts from the last level's min (degree, id) vertex.
//      (Separate mode: all sweeps levels-only, then one labelled traversal from the root.)
//
// Labelled level d (body of Alg. 3). Every frontier vertex u carries a 64-bit key
//   key(u) = ((d + 1) << obits) | ord(u),
// where ord(u) increases with u's label inside the level. Keys therefore increase with the level
// and, inside a level, follow label order.
//   phase A  SpMSpV over (select2nd, min): claim[w] = min(claim[w], key(u)) for every neighbour w.
//            No read of w is needed: a vertex numbered earlier already holds a smaller claim (its
//            parent's key from an earlier level, or 0 for a root), so the min leaves it unchanged.
//   phase B  SELECT + SortPerm (Alg. 3): u owns w iff claim[w] == key(u). Rows are pre-sorted by
//            (degree, id), so scanning the frontier in key order and each row in order lists the
//            next level in (parent label, degree, id) order; an exclusive prefix sum of
//            owned-children counts ranks it.
// On the whole grid, CTA b keeps the children it found as its next slice and numbers them
// ord = b * slot + j (j = rank inside the CTA), which is already in label order because CTA
// slices are contiguous in label order. Their final labels ("+nv" of Alg. 3) need the prefix of
// all CTAs' counts, which the next level's exchange delivers, so a grid level costs one exchange.
// When slices drift out of balance, or the level becomes small, the level is written to perm at
// its final labels and redistributed (one more exchange).
// The reversal of Alg. 1 is fused: the vertex with label L is written to perm[n-1-L].
//
// Grid synchronisation is an "exchange": each CTA writes (count, key) into its slot, arrives on a
// monotone counter with a release reduction, and one thread polls the counter with acquire
// loads; warp 0 then reads all slots, giving the barrier plus the total, this CTA's prefix, the
// largest count and the min key. Every wait is bounded by a %globaltimer limit.
#pragma once

#include "rcm_cc.cuh"
#include "rcm_internal.cuh"

namespace rcm {

constexpr int kEllNb = 7;       // neighbours stored in a vertex's 32-byte row; slot 7 = degree
constexpr int kCache = 2048;    // frontier ids cached in shared memory per buffer
constexpr int kTinyMax = 32;    // components of at most this many vertices are ordered by one thread
constexpr int kWarpLevel = 32;  // narrow levels of at most this many vertices run on warp 0 alone
// A level of a few hundred vertices that holds a hub is far more work than one CTA does quickly,
// and a labelled first sweep over hubs costs more than a levels-only one: graphs with a vertex of
// more than kHubDegree neighbours take a lower frontier switch and levels-only first sweeps by
// default (the 1M-vertex power-law graph with hubs of 7,000: 24.3 ms with the grid defaults,
// 8.8 ms with these).
constexpr int kHubDegree = 512;
constexpr int kHubNarrow = 128;
constexpr unsigned long long kClaimNone = ~0ull;

struct EngineArgs {
    int n;                       // vertices of this graph
    int v0;                      // global id of its first vertex (rows hold global ids)
    const int* rowptr;           // global rows (overflow neighbours of rows with degree > 7)
    const int4* ell;             // 2 x int4 per vertex: 7 sorted neighbours (-1 padded) + degree
    const int* adj;              // full sorted rows, valid for rows with degree > 7
    const int* deg;              // global
    unsigned long long* claim;   // global, 64-bit keys (kClaimNone = not reached)
    int* vis;                    // global sweep stamps
    int* qa;                     // this graph's queue / staging buffer (n ints)
    int* qb;                     // this graph's queue / staging buffer (n ints)
    int* boff;                   // this graph's per-frontier offsets (n ints)
    int* perm;                   // this graph's output segment (n ints); global ids while running
    Ctl* ctl;                    // grid control block (whole-grid executor only)
    int* status;                 // where device-detected error bits are ORed
    int* diag;                   // optional (may be null): first failed guard's site and value
    int narrow_thr;
    int fused;
    int cc_first;                // persistent grid: build the component table before the first sweep
    int hub_auto;                // default launch of the persistent grid: a graph with a vertex of more
                                 // than kHubDegree neighbours takes the frontier switch kHubNarrow and
                                 // levels-only first sweeps (decided on the device from ctl->maxdeg)
    int obits;                   // low bits of a key holding the in-level order
    int profile;                 // accumulate per-phase time (CTA 0, thread 0)
    long long limit_ns;
    // concurrent components (whole-grid executor only)
    int* cc_parent;              // n ints
    int* cc_size;                // n ints (indexed by root)
    unsigned long long* cc_key;  // n keys (indexed by root)
    int* cc_roots;               // cc_cap ints
    unsigned long long* cc_gkey; // next_pow2(cc_cap) keys (sort scratch beyond shared memory)
    int* cc_gidx;                // next_pow2(cc_cap) ints
    int4* cc_tab;                // cc_cap entries: (start vertex, first label, size, root)
    int cc_cap;                  // most components ordered concurrently (else one by one)
    int cc_big;                  // components at least this large run on the whole grid
    // bottom-up expansion (whole-grid executor only; fkey == null: top-down only)
    unsigned long long* fkey;    // n words: a labelled frontier vertex's key, published for bottom-up claims
    int expand_mode;             // 2 = bottom-up on every grid level, 1 = top-down, else per level by frontier size
    int bu_divisor;              // per level: bottom-up once the frontier holds n / bu_divisor vertices
    // asynchronous levels-only sweeps (whole-grid executor only; adist == null: level by level)
    unsigned long long* adist;   // n words: (~sweep stamp) << 32 | breadth-first distance
    unsigned long long* aq;      // work queue of aq_cap (distance << 32 | vertex) items
    AsyncCtl* actl;
    unsigned aq_cap;
    // middle tier (whole-grid executor launched in clusters of mid_k CTAs; 0 = off): labelled
    // levels of narrow_thr <= size < mid_thr run on cluster 0 alone, exchanging through
    // distributed shared memory, while the other CTAs wait at the next grid barrier
    int mid_k;
    int mid_thr;
};

enum { kPhExpand = 0, kPhClaim, kPhOwn, kPhLabels, kPhExchange, kPhRedist, kPhWaitNarrow, kPhOther };

// Shared memory of one engine CTA.
struct EngineSmem {
    EngineArgs args;
    long long st[8];             // statistics (rcm_stats order), updated by thread 0
    long long prof[8];           // per-phase ns (profile), updated by thread 0 of CTA 0
    unsigned long long prof_t;   // timestamp of the last phase boundary
    int scan[64];
    int acc_cnt;                 // CTA count accumulator feeding the exchange
    unsigned long long wkey[32]; // per-warp min keys of the last accumulate()
    int ex[4];                   // exchange results: total, pre, maxcnt
    unsigned long long ex_key;
    int bc[8];
    unsigned long long bck;
    int tail;
    int ntail[3];                // narrow levels-only loop: new-vertex counters, by level mod 3
    struct {                     // state after a run of warp-0 levels, read by the whole CTA
        int F, d, lstart, cb, lastF, bad, qb;
        long long reached;
        unsigned long long lk;
    } wr;
    int aflag;                   // async sweep: stop flag relayed to the CTA's warps
    // middle tier: this CTA's part of each cluster exchange, read by the cluster's CTAs through
    // distributed shared memory; double-buffered by epoch parity
    unsigned long long xc_flag[2];  // (epoch << 32) | count, released at cluster scope
    unsigned long long xc_key[2];   // min (degree, id) key of the CTA's slice
    int cache[2][kCache];
};

enum { kStComponents = 0, kStSweeps, kStTraversals, kStLevels, kStMaxEcc, kStIsolated, kStNarrow, kStGrid };

struct ExResult {
    int total;                // sum of the CTAs' counts
    int pre;                  // sum over CTAs before this one
    int maxcnt;               // largest CTA count
    unsigned long long key;   // min of the CTAs' keys
};

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// kWarp (CTA engines only; on by default with kSmem): narrow levels of at most kWarpLevel vertices
// run on warp 0 alone. Off in the engines it slowed through register allocation.
// kSmem (CTA engines only): the claims, visit stamps and padded rows of the graph live in shared
// memory, indexed from the graph's first vertex v0; otherwise they are global arrays indexed by
// vertex id.
// kAsync (whole-grid engine only): levels-only sweeps through the asynchronous work queue when
// the arguments provide it. kBottomUp (whole-grid engine only): each whole-grid level may run
// bottom-up, chosen per level. Separate instantiations, so the plain top-down kernels carry none
// of their code or registers.
template <bool kCtaOnly, bool kSmem, bool kAsync, bool kBottomUp, bool kWarp>
struct Engine;

// The warp-0 runs of narrow levels, kept out of line: they are entered once per run of levels, and
// inlined they would raise every engine kernel's register pressure.
template <bool kCtaOnly, bool kSmem, bool kAsync, bool kBottomUp, bool kWarp>
__device__ __noinline__ void run_warp_levels(const EngineArgs* a, EngineSmem* sm, int s, int F, int cb, int* cur,
                                             int* nxt, int ecc, long long reached);
template <bool kCtaOnly, bool kSmem, bool kAsync, bool kBottomUp, bool kWarp>
__device__ __noinline__ void run_warp_labelled(const EngineArgs* a, EngineSmem* sm, int d, int lstart, int F, int cb,
                                               const int* sh, const int* g, int step);

template <bool kCtaOnly, bool kSmem = false, bool kAsync = false, bool kBottomUp = false, bool kWarp = kSmem>
struct Engine {
    static_assert(kCtaOnly || !kSmem, "shared-memory state needs a CTA engine");
    static_assert(kCtaOnly || !kWarp, "warp-0 levels need a CTA engine");
    static_assert(!kAsync || !kCtaOnly, "asynchronous sweeps need the whole grid");
    static_assert(!kBottomUp || !kCtaOnly, "bottom-up levels need the whole grid");
    const EngineArgs* a;   // in shared memory (keeps the per-thread register footprint small)
    unsigned epoch;
    unsigned cepoch;       // middle-tier exchanges so far
    int sweep_id;
    int scan_par;          // alternates between consecutive CTA scans (see block_excl_scan)
    bool async_ok;         // asynchronous levels-only sweeps still enabled (off once the queue ran full)
    EngineSmem* sm;
    unsigned long long* sm_sort = nullptr;  // component-table sort buffer (shared), if any
    int sm_sort_cap = 0;

    // All threads call; args are copied to shared memory by thread 0.
    __device__ void init(const EngineArgs& args, EngineSmem* smem) {
        sm = smem;
        if (threadIdx.x == 0) {
            smem->args = args;
            for (int i = 0; i < 8; ++i) smem->st[i] = 0;
            for (int i = 0; i < 8; ++i) smem->prof[i] = 0;
            smem->prof_t = globaltimer_ns();
            smem->acc_cnt = 0;
            for (int i = 0; i < 32; ++i) smem->wkey[i] = kKeyMax;
        }
        __syncthreads();
        a = &smem->args;
        epoch = 0;
        cepoch = 0;
        sweep_id = 0;
        scan_par = 0;
        async_ok = true;
    }

    // Phase boundary: the time since the previous boundary is charged to phase `ph`.
    __device__ void tick(int ph) {
        if (a->profile && threadIdx.x == 0 && cta_rank() == 0) {
            const unsigned long long t = globaltimer_ns();
            sm->prof[ph] += (long long)(t - sm->prof_t);
            sm->prof_t = t;
        }
    }

    __device__ int cta_scan(int x, int* total) {
        const int r = block_excl_scan(x, total, sm->scan, scan_par);
        scan_par ^= 1;
        return r;
    }

    __device__ void stat_add(int i, long long v) {
        if (threadIdx.x == 0) sm->st[i] += v;
    }
    __device__ void stat_max(int i, long long v) {
        if (threadIdx.x == 0 && v > sm->st[i]) sm->st[i] = v;
    }
    __device__ bool in_graph(int v) const { return (unsigned)(v - a->v0) < (unsigned)a->n; }
    __device__ void fail(int bits) { atomicOr(a->status, bits); }
    // An index guard tripped: the run fails with kErrInternal; the first site and its offending
    // value go to diag[0], diag[1] when a diagnostic word is given.
    __device__ void fail_at(int site, int value) {
        atomicOr(a->status, kErrInternal);
        if (a->diag && atomicCAS(a->diag, 0, site) == 0) atomicExch(a->diag + 1, value);
    }
    // A component-table entry (start vertex, first label, size, root) that can be ordered with
    // labels from at least nv.
    __device__ bool tab_ok(const int4& t, int nv) const {
        return in_graph(t.x) && t.y >= nv && t.z > 0 && (long long)t.y + t.z <= a->n;
    }
    __device__ int cta_rank() const { return kCtaOnly ? 0 : (int)blockIdx.x; }
    __device__ int cta_count() const { return kCtaOnly ? 1 : (int)gridDim.x; }

    // Bring a vertex's padded row into L2 ahead of the level that will read it.
    __device__ void prefetch_row(int u) const {
        if constexpr (!kSmem) asm volatile("prefetch.global.L2 [%0];" ::"l"(a->ell + 2 * (size_t)u));
    }

    __device__ unsigned long long* claim_p(int v) const { return a->claim + (kSmem ? v - a->v0 : v); }
    __device__ int* vis_p(int v) const { return a->vis + (kSmem ? v - a->v0 : v); }
    // Claims are updated by atomics: global ones are read from L2 (other CTAs' atomics, and no
    // stale L1 line); shared-memory ones with plain loads.
    __device__ unsigned long long ld_claim(int v) const {
        if constexpr (kSmem) return *claim_p(v);
        else return __ldcg(claim_p(v));
    }

    __device__ void load_row(int u, int (&r)[8]) const {
        int4 x, y;
        if constexpr (kSmem) {
            const int4* p = a->ell + 2 * (size_t)(u - a->v0);
            x = p[0];
            y = p[1];
        } else {
            const int4* p = a->ell + 2 * (size_t)u;
            x = __ldg(p);
            y = __ldg(p + 1);
        }
        r[0] = x.x; r[1] = x.y; r[2] = x.z; r[3] = x.w;
        r[4] = y.x; r[5] = y.y; r[6] = y.z; r[7] = y.w;
    }

    // ---- long rows, read by the whole warp ----
    // A row keeps its first kEllNb neighbours in the padded row; the rest (degree > kEllNb) are
    // read from adj. The lanes holding such a row hand it to the whole warp one row at a time, and
    // the warp reads it 32 entries per round, coalesced: a hub of a scale-free graph costs its
    // degree / 32 rounds instead of its degree serial steps in one thread. The entries of
    // kLongRounds rounds are loaded before the first of them is used, so a hub's rounds do not
    // each wait for their own row read.
    // fn(src, w) runs on all 32 lanes for one round of lane src's row, w = the lane's entry or -1
    // past the row's end; it may use warp-collective operations, and returns true (warp-uniform)
    // to stop reading that row. Must be called by all 32 lanes of the warp.
    static constexpr int kLongRounds = 4;

    template <class Fn>
    __device__ void for_long_rows(bool has, int u, int dg, Fn fn) const {
        unsigned pend = __ballot_sync(0xffffffffu, has && dg > kEllNb);
        const int lane = threadIdx.x & 31;
        while (pend) {
            const int src = __ffs(pend) - 1;
            pend &= pend - 1;
            const int uu = __shfl_sync(0xffffffffu, u, src);
            const int dd = __shfl_sync(0xffffffffu, dg, src);
            const int* row = a->adj + __ldg(a->rowptr + uu);
            for (int k0 = kEllNb; k0 < dd; k0 += 32 * kLongRounds) {
                int w[kLongRounds];
#pragma unroll
                for (int r = 0; r < kLongRounds; ++r) {
                    const int k = k0 + 32 * r + lane;
                    w[r] = k < dd ? __ldg(row + k) : -1;
                }
                bool stop = false;
#pragma unroll
                for (int r = 0; r < kLongRounds; ++r)
                    if (!stop && k0 + 32 * r < dd) stop = fn(src, w[r]);
                if (stop) break;
            }
        }
    }

    // The same for the ownership tests of phase B: each round's entries come with their claims,
    // fn(src, w, claim) (claim = kClaimNone past the row's end), and the entries of kLongRounds
    // rounds, then their claims, are loaded before any is used: a hub costs two dependent round
    // trips per kLongRounds rounds, not per round.
    template <class Fn>
    __device__ void for_long_rows_claims(bool has, int u, int dg, Fn fn) const {
        unsigned pend = __ballot_sync(0xffffffffu, has && dg > kEllNb);
        const int lane = threadIdx.x & 31;
        while (pend) {
            const int src = __ffs(pend) - 1;
            pend &= pend - 1;
            const int uu = __shfl_sync(0xffffffffu, u, src);
            const int dd = __shfl_sync(0xffffffffu, dg, src);
            const int* row = a->adj + __ldg(a->rowptr + uu);
            for (int k0 = kEllNb; k0 < dd; k0 += 32 * kLongRounds) {
                int w[kLongRounds];
                unsigned long long c[kLongRounds];
#pragma unroll
                for (int r = 0; r < kLongRounds; ++r) {
                    const int k = k0 + 32 * r + lane;
                    w[r] = k < dd ? __ldg(row + k) : -1;
                }
#pragma unroll
                for (int r = 0; r < kLongRounds; ++r) c[r] = w[r] >= 0 ? ld_claim(w[r]) : kClaimNone;
#pragma unroll
                for (int r = 0; r < kLongRounds; ++r)
                    if (k0 + 32 * r < dd) fn(src, w[r], c[r]);
            }
        }
    }

    // Per-thread (count, key) partials: counts go to a shared counter, keys to one slot per warp
    // (a 64-bit shared-memory min would need a compare-and-swap loop). Consumers read the CTA
    // min with cta_key() after a barrier.
    __device__ void accumulate(int cnt, unsigned long long key) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            const unsigned long long k = __shfl_xor_sync(0xffffffffu, key, o);
            key = k < key ? k : key;
        }
        if ((threadIdx.x & 31) == 0) {
            if (cnt) atomicAdd(&sm->acc_cnt, cnt);
            sm->wkey[threadIdx.x >> 5] = key;
        }
    }

    // Min over the per-warp keys of the last accumulate(); call after a barrier.
    __device__ unsigned long long cta_key() const {
        unsigned long long k = kKeyMax;
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; ++w) k = sm->wkey[w] < k ? sm->wkey[w] : k;
        return k;
    }

    // ---- the exchange: grid barrier carrying the accumulated (count, key) of every CTA ----
    // Callers accumulate() first; the accumulators are consumed and reset. Returns false if a wait
    // ran out or another CTA failed.
    __device__ bool exchange(ExResult& r, bool payload = true) {
        __syncthreads();
        if (kCtaOnly) {
            r.total = sm->acc_cnt;
            r.pre = 0;
            r.maxcnt = r.total;
            r.key = cta_key();
            __syncthreads();
            if (threadIdx.x == 0) sm->acc_cnt = 0;
            return true;
        }
        const unsigned e = ++epoch;
        const int B = gridDim.x, b = blockIdx.x;
        Ctl* c = a->ctl;
        if (threadIdx.x < 32) {
            int bad = 0;
            if (threadIdx.x == 0) {
                ExSlot* sl = &c->slots[e & 1][b];
                sl->flag = ((unsigned long long)e << 32) | (unsigned)sm->acc_cnt;
                sl->key = cta_key();
                sm->acc_cnt = 0;
                red_release_add(&c->arrive, 1u);
                const unsigned target = e * (unsigned)B;
                if ((int)(ld_acquire(&c->arrive) - target) < 0) {
                    const unsigned long long t0 = globaltimer_ns();
                    unsigned spins = 0;
                    while ((int)(ld_acquire(&c->arrive) - target) < 0) {
                        if ((++spins & 31u) == 0) {
                            if (ld_volatile(&c->status) & (kErrTimeout | kErrInternal | kErrTooLarge)) { bad = 1; break; }
                            if ((long long)(globaltimer_ns() - t0) > a->limit_ns) {
                                atomicOr(&c->status, kErrTimeout);
                                bad = 1;
                                break;
                            }
                        }
                    }
                }
            }
            bad = __shfl_sync(0xffffffffu, bad, 0);
            __syncwarp();
            int x = 0, y = 0, mx = 0;
            unsigned long long k = kKeyMax;
            if (payload && !bad) {
                // slots in batches of 8 per lane: all loads of a batch are issued before use
                for (int i0 = threadIdx.x; i0 < B; i0 += 32 * 8) {
                    unsigned long long f[8], kk[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int i = i0 + 32 * t;
                        f[t] = i < B ? __ldcg(&c->slots[e & 1][i].flag) : 0ull;
                        kk[t] = i < B ? __ldcg(&c->slots[e & 1][i].key) : kKeyMax;
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int i = i0 + 32 * t;
                        const int v = (int)(unsigned)(f[t] & 0xffffffffu);
                        if (i < b) x += v;
                        y += v;
                        mx = max(mx, v);
                        k = kk[t] < k ? kk[t] : k;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    const unsigned long long kk = __shfl_xor_sync(0xffffffffu, k, o);
                    k = kk < k ? kk : k;
                }
            }
            if (threadIdx.x == 0) {
                sm->ex[0] = y;
                sm->ex[1] = x;
                sm->ex[2] = mx;
                sm->ex[3] = bad;
                sm->ex_key = k;
            }
        }
        __syncthreads();
        r.total = sm->ex[0];
        r.pre = sm->ex[1];
        r.maxcnt = sm->ex[2];
        r.key = sm->ex_key;
        const bool ok = sm->ex[3] == 0;
        __syncthreads();
        return ok;
    }

    __device__ bool barrier() {
        ExResult r;
        return exchange(r, false);
    }

    // ---- the middle tier's exchange: the mid_k CTAs of cluster 0 ----
    // Each CTA publishes (epoch << 32) | count in its own shared memory with a cluster-scope release
    // (after a CTA barrier, so its claims are released with it); warp 0's lanes poll the peers' words
    // with cluster-scope acquire loads through distributed shared memory. The words are double-
    // buffered by epoch parity: a CTA rewrites a slot two epochs later, only after every peer has
    // published the epoch in between, i.e. finished reading this one. Every wait is bounded by
    // limit_ns. r receives the total, this CTA's prefix and the largest count (not the key: see
    // mid_min_key). Returns false if a wait ran out or another CTA failed.
    __device__ bool exchange_mid(ExResult& r) {
        __syncthreads();
        const unsigned e = ++cepoch;
        const int K = a->mid_k;
        const int me = (int)cluster_rank();
        if (threadIdx.x == 0) {
            sm->xc_key[e & 1] = cta_key();
            const unsigned cnt = (unsigned)sm->acc_cnt;
            sm->acc_cnt = 0;
            st_release_cluster_u64(&sm->xc_flag[e & 1], ((unsigned long long)e << 32) | cnt);
        }
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int bad = 0, x = 0, y = 0, mx = 0;
            if (lane < K) {
                const unsigned fr = dsmem_addr(&sm->xc_flag[e & 1], (unsigned)lane);
                unsigned long long f = ld_acquire_cluster_u64(fr);
                if ((unsigned)(f >> 32) != e) {
                    const unsigned long long t0 = globaltimer_ns();
                    unsigned spins = 0;
                    while ((unsigned)((f = ld_acquire_cluster_u64(fr)) >> 32) != e) {
                        if ((++spins & 31u) == 0) {
                            if (ld_volatile(a->status) & (kErrTimeout | kErrInternal | kErrTooLarge)) {
                                bad = 1;
                                break;
                            }
                            if ((long long)(globaltimer_ns() - t0) > a->limit_ns) {
                                atomicOr(a->status, kErrTimeout);
                                bad = 1;
                                break;
                            }
                        }
                    }
                }
                if (!bad) {
                    const int v = (int)(unsigned)(f & 0xffffffffu);
                    y = v;
                    x = lane < me ? v : 0;
                    mx = v;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                y += __shfl_xor_sync(0xffffffffu, y, o);
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                bad |= __shfl_xor_sync(0xffffffffu, bad, o);
            }
            if (lane == 0) {
                // a member that failed set the status before publishing: every member sees it here
                if (ld_volatile(a->status) & (kErrTimeout | kErrInternal | kErrTooLarge)) bad = 1;
                sm->ex[0] = y;
                sm->ex[1] = x;
                sm->ex[2] = mx;
                sm->ex[3] = bad;
            }
        }
        __syncthreads();
        r.total = sm->ex[0];
        r.pre = sm->ex[1];
        r.maxcnt = sm->ex[2];
        r.key = kKeyMax;
        const bool ok = sm->ex[3] == 0;
        __syncthreads();
        return ok;
    }

    // Min over the cluster-0 CTAs of the keys published at middle-tier exchange e. Valid after
    // exchange e + 1 as long as no CTA has started exchange e + 2 (true where it is used: the
    // run's end, before the grid barrier every CTA must reach).
    __device__ unsigned long long mid_min_key(unsigned e) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            unsigned long long k = kKeyMax;
            if (lane < a->mid_k) k = ld_dsmem_u64(dsmem_addr(&sm->xc_key[e & 1], (unsigned)lane));
            k = warp_min_u64(k);
            if (lane == 0) sm->ex_key = k;
        }
        __syncthreads();
        const unsigned long long k = sm->ex_key;
        __syncthreads();
        return k;
    }

    // ---------------- levels-only level ----------------
    // Frontier f[i], i in [lo, hi): the shared cache when `cache` is set, else the global queue
    // cur. Newly reached vertices get stamp s in vis[] and are appended to nxt (positions reserved
    // once per CTA and round through *tail) and, for positions below kCache, to `ncache`.
    // Accumulates this CTA's count of new vertices and its min (degree, id) over the slice.
    __device__ void expand_levels(int s, const int* cur, const int* cache, int lo, int hi, int* nxt,
                                  int* ncache, int* tail) {
        const int T = blockDim.x;
        unsigned long long key = kKeyMax;
        int cnt = 0;
        for (int i0 = lo; i0 < hi; i0 += T) {
            const int i = i0 + (int)threadIdx.x;
            unsigned mask = 0;
            int r[8];
            int d = 0, u = -1;
            if (i < hi) {
                u = cache ? cache[i] : ldcg(cur + i);
                if (!in_graph(u)) {
                    fail(kErrInternal);
                    u = -1;
                } else {
                    load_row(u, r);
                    d = r[7];
                    key = min(key, pack_key(d, u));
                    // issue every exchange before looking at any result, so they overlap
                    int old[kEllNb];
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k) old[k] = k < d ? atomicExch(vis_p(r[k]), s) : s;
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k) mask |= (old[k] != s ? 1u : 0u) << k;
                }
            }
            // neighbours beyond the padded row (degree > 7), a warp round at a time; the new ones of
            // a round take consecutive positions reserved by one atomic
            for_long_rows(u >= 0, u, d, [&](int, int w) {
                const bool fresh = w >= 0 && atomicExch(vis_p(w), s) != s;
                const unsigned bal = __ballot_sync(0xffffffffu, fresh);
                if (bal) {
                    const int lane = threadIdx.x & 31;
                    int base = 0;
                    if (lane == 0) base = atomicAdd(tail, __popc(bal));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (fresh) {
                        const int pos = base + __popc(bal & ((1u << lane) - 1u));
                        prefetch_row(w);
                        nxt[pos] = w;
                        if (ncache && pos < kCache) ncache[pos] = w;
                    }
                    if (lane == 0) cnt += __popc(bal);
                }
                return false;
            });
            const int c = __popc(mask);
            int tot;
            const int ex = cta_scan(c, &tot);
            if (tot) {
                if (threadIdx.x == 0) sm->bc[0] = atomicAdd(tail, tot);
                __syncthreads();
                int pos = sm->bc[0] + ex;
                __syncthreads();
#pragma unroll
                for (int k = 0; k < kEllNb; ++k)
                    if (mask & (1u << k)) {
                        prefetch_row(r[k]);
                        nxt[pos] = r[k];
                        if (ncache && pos < kCache) ncache[pos] = r[k];
                        ++pos;
                    }
            }
            cnt += c;
        }
        accumulate(cnt, key);
    }

    // Levels-only levels of at most kWarpLevel vertices, run by warp 0 alone (one vertex per lane,
    // the frontier in the shared cache): positions come from a warp scan, the only synchronisation
    // is __syncwarp, and the rows held in registers give the (degree, id) minimum of the last level.
    // Runs while the levels stay that narrow (and, on the grid, below the narrow threshold); lane 0
    // leaves the state in sm->wr. Called by the 32 threads of warp 0 only.
    __device__ void warp_levels(int s, int F, int cb, int* cur, int* nxt, int ecc, long long reached) {
        const int lane = threadIdx.x & 31;
        unsigned long long lk = kKeyMax;
        int bad = 0;
        while (true) {
            int* nc = sm->cache[cb ^ 1];
            int cnt = 0;
            unsigned long long m = kKeyMax;
            unsigned mask = 0;
            int r[8];
            int d = 0, u = -1;
            if (lane < F) {
                u = sm->cache[cb][lane];
                if (!in_graph(u)) {
                    bad = 1;
                    u = -1;
                } else {
                    load_row(u, r);
                    d = r[7];
                    m = pack_key(d, u);
                    int old[kEllNb];
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k) old[k] = k < d ? atomicExch(vis_p(r[k]), s) : s;
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k) mask |= (old[k] != s ? 1u : 0u) << k;
                }
            }
            for_long_rows(u >= 0, u, d, [&](int, int w) {
                const bool fresh = w >= 0 && atomicExch(vis_p(w), s) != s;
                const unsigned bal = __ballot_sync(0xffffffffu, fresh);
                if (fresh) {
                    const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                    prefetch_row(w);
                    nxt[pos] = w;
                    if (pos < kCache) nc[pos] = w;
                }
                cnt += __popc(bal);
                return false;
            });
            const int cc = __popc(mask);
            const int incl = warp_incl_scan(cc);
            int pos = cnt + incl - cc;
#pragma unroll
            for (int k = 0; k < kEllNb; ++k)
                if (mask & (1u << k)) {
                    prefetch_row(r[k]);
                    nxt[pos] = r[k];
                    if (pos < kCache) nc[pos] = r[k];
                    ++pos;
                }
            cnt += __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            tick(kPhExpand);
            stat_add(kStNarrow, 1);
            if (cnt == 0) {
                lk = warp_min_u64(m);
                F = 0;
                break;
            }
            int* t = cur; cur = nxt; nxt = t;
            cb ^= 1;
            F = cnt;
            reached += cnt;
            if (++ecc > a->n) {
                if (lane == 0) fail_at(kSiteLevels, ecc);
                bad = 1;
                break;
            }
            if (F > kWarpLevel || (!kCtaOnly && F >= a->narrow_thr)) break;
        }
        bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
        if (lane == 0) {
            if (bad) fail(kErrInternal);
            sm->wr.F = F;
            sm->wr.cb = cb;
            sm->wr.d = ecc;
            sm->wr.reached = reached;
            sm->wr.lk = lk;
            sm->wr.bad = bad;
            sm->wr.qb = cur == a->qb ? 1 : 0;
        }
    }

    // Levels-only level run by one CTA alone (CTA 0 of the grid, or a CTA engine): the order of a
    // levels-only frontier does not matter, so each warp reserves its new vertices' positions with
    // one shared-memory atomic on *tail, which ends as the level's count. No CTA barrier and no
    // (degree, id) minimum: the caller takes the minimum over the last level only.
    __device__ void expand_narrow(int s, const int* cur, const int* cache, int F, int* nxt, int* ncache, int* tail) {
        const int T = blockDim.x, lane = threadIdx.x & 31;
        for (int i0 = 0; i0 < F; i0 += T) {
            const int i = i0 + (int)threadIdx.x;
            unsigned mask = 0;
            int r[8];
            int d = 0, u = -1;
            if (i < F) {
                u = cache ? cache[i] : ldcg(cur + i);
                if (!in_graph(u)) {
                    fail(kErrInternal);
                    u = -1;
                } else {
                    load_row(u, r);
                    d = r[7];
                    int old[kEllNb];
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k) old[k] = k < d ? atomicExch(vis_p(r[k]), s) : s;
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k) mask |= (old[k] != s ? 1u : 0u) << k;
                }
            }
            for_long_rows(u >= 0, u, d, [&](int, int w) {
                const bool fresh = w >= 0 && atomicExch(vis_p(w), s) != s;
                const unsigned bal = __ballot_sync(0xffffffffu, fresh);
                if (bal) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(tail, __popc(bal));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (fresh) {
                        const int pos = base + __popc(bal & ((1u << lane) - 1u));
                        prefetch_row(w);
                        nxt[pos] = w;
                        if (ncache && pos < kCache) ncache[pos] = w;
                    }
                }
                return false;
            });
            const int c = __popc(mask);
            const int incl = warp_incl_scan(c);
            const int wtot = __shfl_sync(0xffffffffu, incl, 31);
            if (wtot) {
                int base = 0;
                if (lane == 0) base = atomicAdd(tail, wtot);
                int pos = __shfl_sync(0xffffffffu, base, 0) + incl - c;
#pragma unroll
                for (int k = 0; k < kEllNb; ++k)
                    if (mask & (1u << k)) {
                        prefetch_row(r[k]);
                        nxt[pos] = r[k];
                        if (ncache && pos < kCache) ncache[pos] = r[k];
                        ++pos;
                    }
            }
        }
    }

    // Min (degree, id) key over a level of F vertices held in cache (shared) or cur (global), for
    // every thread of the CTA: Alg. 2's next root is the least such vertex of the last level.
    __device__ unsigned long long level_min_key(const int* cur, const int* cache, int F) {
        unsigned long long key = kKeyMax;
        for (int i = threadIdx.x; i < F; i += blockDim.x) {
            const int u = cache ? cache[i] : ldcg(cur + i);
            if (!in_graph(u)) {
                fail(kErrInternal);
                continue;
            }
            int r[8];
            load_row(u, r);
            key = min(key, pack_key(r[7], u));
        }
        return block_min_u64(key, sm->wkey);
    }

    // ---------------- bottom-up expansion (whole grid) ----------------
    // Top-down, a level's frontier pushes to its neighbours. Bottom-up, every vertex not yet reached
    // looks at its own neighbours instead. An unvisited vertex has no neighbour in a level below
    // the current one (its neighbours there would have reached it), so "some neighbour visited" means
    // "some neighbour in the current level", and the smallest frontier key among its neighbours is
    // what the top-down atomicMin would leave in its claim. Both give the same levels and labels;
    // bottom-up reads every vertex once per level and pays off only when the frontier is a large
    // part of the graph.

    // Whether whole-grid level work of frontier size F, with `seen` vertices already reached, runs
    // bottom-up. Uniform over the grid (every CTA holds the same F and seen).
    __device__ bool bottom_up(long long F, long long seen) const {
        if constexpr (!kBottomUp) return false;
        if (!a->fkey || a->expand_mode == 1) return false;
        if (a->expand_mode == 2) return true;
        return F * a->bu_divisor >= a->n && F * 4 >= (long long)a->n - seen;
    }

    // Levels-only, bottom-up: every vertex not stamped s with a stamped neighbour is appended to
    // nxt, unstamped (the caller stamps the new level after the exchange, so that this pass never
    // sees it). Accumulates their count and the min (degree, id) over the frontier slice [lo, hi).
    __device__ void expand_levels_bottom_up(int s, const int* cur, int lo, int hi, int* nxt, int* tail) {
        const int T = blockDim.x, n = a->n;
        unsigned long long key = kKeyMax;
        for (int i = lo + (int)threadIdx.x; i < hi; i += T) {
            const int u = ldcg(cur + i);
            if (in_graph(u)) key = min(key, pack_key(__ldg(a->deg + u), u));
        }
        int cnt = 0;
        const int stride = cta_count() * T;
        for (int i0 = cta_rank() * T; i0 < n; i0 += stride) {
            const int i = i0 + (int)threadIdx.x;
            const int w = a->v0 + i;
            bool found = false;
            int dgl = 0;  // degree of an unvisited vertex whose padded row showed no stamped neighbour
            if (i < n && ldcg(vis_p(w)) != s) {
                int r[8];
                load_row(w, r);
                const int dg = r[7];
                int st[kEllNb];
#pragma unroll
                for (int k = 0; k < kEllNb; ++k) st[k] = k < dg ? ldcg(vis_p(r[k])) : 0;
#pragma unroll
                for (int k = 0; k < kEllNb; ++k) found |= k < dg && st[k] == s;
                dgl = found ? 0 : dg;
            }
            // rows beyond the padded part, by the warp until a stamped neighbour turns up
            for_long_rows(dgl > kEllNb, w, dgl, [&](int src, int x) {
                const unsigned bal = __ballot_sync(0xffffffffu, x >= 0 && ldcg(vis_p(x)) == s);
                if ((int)(threadIdx.x & 31) == src && bal) found = true;
                return bal != 0;
            });
            int tot;
            const int ex = cta_scan(found ? 1 : 0, &tot);
            if (tot) {
                if (threadIdx.x == 0) sm->bc[0] = atomicAdd(tail, tot);
                __syncthreads();
                if (found) nxt[sm->bc[0] + ex] = w;
                __syncthreads();
            }
            cnt += found ? 1 : 0;
        }
        accumulate(cnt, key);
    }

    // Stamps the F vertices of nxt with s (balanced slices), then a grid barrier.
    __device__ bool stamp_level(int s, const int* nxt, int F) {
        const int b = cta_rank(), B = cta_count();
        const int lo = (int)((long long)F * b / B), hi = (int)((long long)F * (b + 1) / B);
        for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
            const int w = ldcg(nxt + i);
            if (in_graph(w)) *vis_p(w) = s;
            else fail(kErrInternal);
        }
        return barrier();
    }

    // ---------------- asynchronous levels-only sweep (whole grid) ----------------
    // A levels-only sweep needs only the eccentricity of the root and the min (degree, id) vertex
    // of the last level (Alg. 2), and both follow from the breadth-first distances alone, which
    // are unique. So the sweep need not run level by level: it relaxes distances through a work
    // queue with no grid barrier between levels, and the result is the same.
    //   adist[v] = (~s) << 32 | dist for sweep stamp s: one 64-bit atomicMin both starts a new
    //   sweep's value (a later sweep has a smaller high word) and keeps the shorter distance.
    //   A warp takes 32 consecutive queue slots and polls them; each item (d, u) found relaxes
    //   u's neighbours to d + 1, and every neighbour whose distance dropped is appended (slots
    //   reserved with one atomic per warp round). An item made stale by a later improvement only
    //   repeats relaxations that change nothing.
    //   Items are handed over with release stores and acquire loads of their slots, so an item's
    //   reservation happens before anything its consumer does.
    //   Termination: every CTA publishes, with release, a monotone count of the items it has
    //   finished, after reserving their children's slots. Let p be the sum of those counts (read
    //   with acquire) and t the reserved-slot count read afterwards. Every counted item and every
    //   child of one was reserved before that read, so if p == t the counted items are exactly
    //   the slots [0, t). A reservation outside them would need a reserving item outside them
    //   first, so none can ever happen: the queue is drained.
    // Then two passes over the queue give the eccentricity (largest final distance), the size
    // (items whose distance is final: one per vertex) and the last level's min (degree, id).
    // Returns 1 when done, 0 on a failed wait or guard, -1 when the queue ran full (the caller
    // repeats the sweep level by level).
    __device__ int sweep_async(int root, int& ecc, unsigned long long& last_key, long long& reached) {
        AsyncCtl* ac = a->actl;
        unsigned long long* q = a->aq;
        const unsigned Q = a->aq_cap;
        const int s = ++sweep_id;
        const unsigned long long tag = (unsigned long long)(~(unsigned)s) << 32;
        const int b = blockIdx.x, B = gridDim.x;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        // queue emptied (slot 0 holds the root), counters cleared
        const long long stride = (long long)B * blockDim.x;
        for (long long i = 1 + (long long)b * blockDim.x + threadIdx.x; i < (long long)Q; i += stride) q[i] = kKeyMax;
        if (threadIdx.x == 0) {
            ac->proc[8 * b] = 0;
            sm->aflag = 0;
        }
        if (b == 0 && threadIdx.x == 0) {
            a->adist[root] = tag;
            q[0] = (unsigned)root;
            ac->head = 0;
            ac->tail = 1ull;
            ac->flag = 0;
        }
        if (!barrier()) return 0;
        const unsigned long long t0 = globaltimer_ns();
        unsigned base = 0, pend = 0;
        unsigned long long item = kKeyMax;
        bool have = false;
        int idle = 0;
        while (true) {
            if (pend == 0) {
                unsigned x = 0;
                if (lane == 0) x = atomicAdd(&ac->head, 32u);
                base = __shfl_sync(0xffffffffu, x, 0);
                pend = 0xffffffffu;
            }
            const unsigned idx = base + (unsigned)lane;
            if (!have && ((pend >> lane) & 1u) && idx < Q) {
                item = ld_acquire_u64(q + idx);
                have = item != kKeyMax;
            }
            const unsigned hm = __ballot_sync(0xffffffffu, have);
            if (hm) {
                relax_async(have, item, tag, q, Q);
                __syncwarp();
                if (lane == 0) red_release_add(&ac->proc[8 * b], (unsigned)__popc(hm));
                pend &= ~hm;
                have = false;
                idle = 0;
                continue;
            }
            ++idle;
            int f = 0;
            if (wid == 0) {
                if (lane == 0) {
                    f = ld_volatile(&ac->flag);
                    if (ld_volatile(a->status) & (kErrTimeout | kErrInternal | kErrTooLarge)) f |= 4;
                    if (!f && (idle & 63) == 0 && (long long)(globaltimer_ns() - t0) > a->limit_ns) {
                        atomicOr(a->status, kErrTimeout);
                        f |= 4;
                    }
                }
                f = __shfl_sync(0xffffffffu, f, 0);
                if (!f && (idle & 7) == 0) {
                    // termination test: finished counts (acquire), then the reserved count
                    unsigned long long p = 0;
                    for (int i = lane; i < B; i += 32) p += ld_acquire(&ac->proc[8 * i]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                    __syncwarp();
                    unsigned long long t = 0;
                    if (lane == 0) {
                        __threadfence();
                        t = ld_relaxed_u64(&ac->tail);
                    }
                    t = __shfl_sync(0xffffffffu, t, 0);
                    if (p == t) {
                        f = 1;
                        if (lane == 0) atomicOr(&ac->flag, 1);
                    }
                }
                if (f && lane == 0) *(volatile int*)&sm->aflag = f;
            } else {
                f = __shfl_sync(0xffffffffu, *(volatile int*)&sm->aflag, 0);
            }
            if (f) break;
        }
        __syncthreads();
        if (!barrier()) return 0;
        if (threadIdx.x == 0) sm->bc[0] = ld_volatile(&ac->flag);
        __syncthreads();
        const int flag = sm->bc[0];
        __syncthreads();
        if (flag & 2) return -1;
        const unsigned long long t_all = ld_relaxed_u64(&ac->tail);
        const unsigned T = t_all < (unsigned long long)Q ? (unsigned)t_all : Q;
        // pass 1: size and eccentricity
        unsigned maxd = 0;
        int cnt = 0;
        for (long long i = (long long)b * blockDim.x + threadIdx.x; i < (long long)T; i += stride) {
            const unsigned long long it = __ldcg(q + i);
            const int v = (int)(unsigned)(it & 0xffffffffu);
            if (!in_graph(v)) {
                fail_at(kSiteLevels, v);
                continue;
            }
            const unsigned long long e = __ldcg(a->adist + v);
            if ((e & 0xffffffff00000000ull) != tag) {
                fail_at(kSiteLevels, v);
                continue;
            }
            if ((unsigned)(it >> 32) == (unsigned)e) {
                ++cnt;
                maxd = max(maxd, (unsigned)e);
            }
        }
        accumulate(cnt, 0xffffffffull - maxd);
        ExResult r1;
        if (!exchange(r1)) return 0;
        ecc = (int)(0xffffffffu - (unsigned)r1.key);
        reached = r1.total;
        if (ecc < 0 || ecc > a->n) {
            fail_at(kSiteLevels, ecc);
            return 0;
        }
        // pass 2: min (degree, id) over the last level
        unsigned long long key = kKeyMax;
        for (long long i = (long long)b * blockDim.x + threadIdx.x; i < (long long)T; i += stride) {
            const unsigned long long it = __ldcg(q + i);
            if ((int)(unsigned)(it >> 32) != ecc) continue;
            const int v = (int)(unsigned)(it & 0xffffffffu);
            if (in_graph(v) && (int)(unsigned)__ldcg(a->adist + v) == ecc) {
                const unsigned long long k = pack_key(__ldg(a->deg + v), v);
                key = k < key ? k : key;
            }
        }
        accumulate(0, key);
        ExResult r2;
        if (!exchange(r2)) return 0;
        last_key = r2.key;
        return 1;
    }

    // One round of the asynchronous sweep for the lanes holding an item (warp-collective).
    __device__ void relax_async(bool have, unsigned long long item, unsigned long long tag, unsigned long long* q,
                                unsigned Q) {
        int u = have ? (int)(unsigned)(item & 0xffffffffu) : -1;
        const unsigned nd = have ? (unsigned)(item >> 32) + 1u : 0u;
        if (have && !in_graph(u)) {
            fail_at(kSiteLevels, u);
            u = -1;
        }
        const unsigned long long val = tag | nd;
        int r[8];
        int dg = 0;
        if (u >= 0) {
            load_row(u, r);
            dg = r[7];
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = -1;
        }
        unsigned long long old[kEllNb];
#pragma unroll
        for (int k = 0; k < kEllNb; ++k) old[k] = k < dg ? atomicMin(a->adist + r[k], val) : val;
        unsigned mask = 0;
#pragma unroll
        for (int k = 0; k < kEllNb; ++k) mask |= (old[k] > val ? 1u : 0u) << k;
        push_async(mask, r, nd, q, Q);
        // neighbours beyond the padded row (degree > 7), 8 per round
        const int extra = dg > kEllNb ? dg - kEllNb : 0;
        const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)((extra + 7) >> 3));
        const int rp = extra ? __ldg(a->rowptr + u) : 0;
        for (int j = 0; j < rounds; ++j) {
            int w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int p = kEllNb + 8 * j + k;
                w[k] = p < dg ? __ldg(a->adj + rp + p) : -1;
            }
            unsigned long long o2[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) o2[k] = w[k] >= 0 ? atomicMin(a->adist + w[k], val) : val;
            unsigned m2 = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) m2 |= (o2[k] > val ? 1u : 0u) << k;
            push_async(m2, w, nd, q, Q);
        }
    }

    // Appends the vertices w[k] (bit k of mask) with distance nd: one slot reservation per warp.
    __device__ void push_async(unsigned mask, const int (&w)[8], unsigned nd, unsigned long long* q, unsigned Q) {
        const int lane = threadIdx.x & 31;
        const int c = __popc(mask);
        const int incl = warp_incl_scan(c);
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot == 0) return;
        unsigned long long x = 0;
        if (lane == 0) x = atomicAdd(&a->actl->tail, (unsigned long long)tot);
        unsigned long long pos = __shfl_sync(0xffffffffu, x, 0) + (unsigned long long)(incl - c);
        __syncwarp();  // the reservation is ordered before every lane's release store below
        bool full = false;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (mask & (1u << k)) {
                if (pos < (unsigned long long)Q) {
                    prefetch_row(w[k]);
                    st_release_u64(q + pos, ((unsigned long long)nd << 32) | (unsigned)w[k]);
                } else {
                    full = true;
                }
                ++pos;
            }
        if (__any_sync(0xffffffffu, full) && lane == 0) atomicOr(&a->actl->flag, 2);
    }

    // Levels-only sweep from root. On return: ecc, the min (degree, id) key of the last level and
    // the number of vertices reached (the component's size).
    __device__ bool sweep_levels(int root, int& ecc, unsigned long long& last_key, long long& reached) {
        if constexpr (kAsync) {
            if (a->adist && async_ok) {
                const int rc = sweep_async(root, ecc, last_key, reached);
                if (rc >= 0) return rc == 1;
                async_ok = false;  // the queue ran full: this and later sweeps run level by level
            }
        }
        Ctl* c = a->ctl;
        const int s = ++sweep_id;
        const int b = cta_rank(), B = cta_count();
        if (b == 0 && threadIdx.x == 0) {
            *vis_p(root) = s;
            a->qa[0] = root;
            sm->cache[0][0] = root;
            if (!kCtaOnly) c->qtail[0] = c->qtail[1] = c->qtail[2] = 0;
        }
        __syncthreads();
        int* cur = a->qa;
        int* nxt = a->qb;
        int F = 1;
        bool in_cache = true;  // CTA 0's shared cache holds the frontier (narrow runs only)
        ecc = 0;
        reached = 1;
        if (!kCtaOnly && a->narrow_thr <= 1) {
            if (!barrier()) return false;
            in_cache = false;
        }
        int cb = 0;
        while (true) {
            if (kCtaOnly || F < a->narrow_thr) {
                unsigned long long lk = kKeyMax;
                if (kCtaOnly || b == 0) {
                    if (!in_cache) {
                        for (int i = threadIdx.x; i < F; i += blockDim.x) sm->cache[cb][i] = ldcg(cur + i);
                        in_cache = true;
                    }
                    // one CTA barrier per level: the level's new-vertex counter is ntail[p], and the
                    // next level's is cleared while this one runs (its last readers finished before
                    // the previous level's barrier)
                    int p = 0;
                    if (threadIdx.x == 0) sm->ntail[0] = 0;
                    __syncthreads();
                    while (true) {
                        // a run of narrow levels on warp 0 (where kWarp is on: in the grid and batch
                        // kernels the extra code cost more through register allocation than it saved);
                        // ntail[p] stays clear for the next CTA level
                        if (kWarp && F <= kWarpLevel) {
                            if (threadIdx.x < 32)
                                run_warp_levels<kCtaOnly, kSmem, kAsync, kBottomUp, kWarp>(a, sm, s, F, cb, cur, nxt, ecc, reached);
                            __syncthreads();
                            F = sm->wr.F;
                            cb = sm->wr.cb;
                            ecc = sm->wr.d;
                            reached = sm->wr.reached;
                            if (sm->wr.bad) return false;
                            cur = sm->wr.qb ? a->qb : a->qa;
                            nxt = sm->wr.qb ? a->qa : a->qb;
                            if (F == 0) {
                                lk = sm->wr.lk;
                                break;
                            }
                            if (!kCtaOnly && F >= a->narrow_thr) break;
                            continue;
                        }
                        if (threadIdx.x == 0) sm->ntail[p == 2 ? 0 : p + 1] = 0;
                        const int* cache = F <= kCache ? sm->cache[cb] : nullptr;
                        expand_narrow(s, cur, cache, F, nxt, sm->cache[cb ^ 1], &sm->ntail[p]);
                        __syncthreads();
                        tick(kPhExpand);
                        const int cnt = sm->ntail[p];
                        stat_add(kStNarrow, 1);
                        if (cnt == 0) {
                            lk = level_min_key(cur, cache, F);
                            F = 0;
                            break;
                        }
                        int* t = cur; cur = nxt; nxt = t;
                        cb ^= 1;
                        F = cnt;
                        reached += cnt;
                        p = p == 2 ? 0 : p + 1;
                        if (++ecc > a->n) {
                            fail_at(kSiteLevels, ecc);
                            return false;
                        }
                        if (!kCtaOnly && F >= a->narrow_thr) break;
                    }
                    if (kCtaOnly) {
                        __syncthreads();
                        last_key = lk;
                        return true;
                    }
                    if (threadIdx.x == 0) {
                        c->pub_F = F;
                        c->pub_cur = (cur == a->qb) ? 1 : 0;
                        c->pub_ecc = ecc;
                        c->pub_key = lk;
                        c->pub_reached = reached;
                        c->qtail[ecc % 3] = 0;
                    }
                }
                tick(kPhOther);
                if (!barrier()) return false;
                tick(kPhWaitNarrow);
                if (threadIdx.x == 0) {
                    sm->bc[0] = ldcg(&c->pub_F);
                    sm->bc[1] = ldcg(&c->pub_cur);
                    sm->bc[2] = ldcg(&c->pub_ecc);
                    sm->bck = __ldcg(&c->pub_key);
                }
                __syncthreads();
                const int Fp = sm->bc[0], pc = sm->bc[1];
                ecc = sm->bc[2];
                lk = sm->bck;
                reached = __ldcg(&c->pub_reached);
                __syncthreads();
                cur = pc ? a->qb : a->qa;
                nxt = pc ? a->qa : a->qb;
                in_cache = false;
                if (Fp == 0) {
                    last_key = lk;
                    return true;
                }
                F = Fp;
                continue;
            }
            // whole grid: balanced slices of the compact queue
            int* tail = &c->qtail[ecc % 3];
            if (b == 0 && threadIdx.x == 0) c->qtail[(ecc + 1) % 3] = 0;
            const int lo = (int)((long long)F * b / B), hi = (int)((long long)F * (b + 1) / B);
            const bool bu = bottom_up(F, reached);
            if (bu) expand_levels_bottom_up(s, cur, lo, hi, nxt, tail);
            else expand_levels(s, cur, nullptr, lo, hi, nxt, nullptr, tail);
            tick(kPhExpand);
            ExResult r;
            if (!exchange(r)) return false;
            tick(kPhExchange);
            stat_add(kStGrid, 1);
            if (r.total == 0) {
                last_key = r.key;
                return true;
            }
            if (bu && !stamp_level(s, nxt, r.total)) return false;
            int* t = cur; cur = nxt; nxt = t;
            F = r.total;
            reached += r.total;
            ++ecc;
            in_cache = false;
        }
    }

    // ---------------- labelled sweep (Alg. 3) ----------------

    // A CTA's part of a level: cnt vertex ids, element j at sh[j] (shared memory) or g[step * j]
    // (global: a staging buffer with step 1, or a label range of perm with step -1).
    struct Slice {
        const int* sh;
        const int* g;
        int step;
        int cnt;
    };

    __device__ int sid(const Slice& s, int j) const { return s.sh ? s.sh[j] : ldcg(s.g + (long long)s.step * j); }

    __device__ Slice perm_range(int first, int cnt) const {
        Slice s;
        s.sh = nullptr;
        s.g = a->perm + (a->n - 1 - first);
        s.step = -1;
        s.cnt = cnt;
        return s;
    }

    __device__ unsigned long long level_key(int d, unsigned long long ord) const {
        return ((unsigned long long)(d + 1) << a->obits) | ord;
    }

    // Bit k set iff the k-th padded-row neighbour is claimed by `key`. All claim loads are issued
    // before any comparison so that they overlap.
    __device__ unsigned owned_mask(const int (&rw)[8], int dg, unsigned long long key) const {
        unsigned long long cl[kEllNb];
#pragma unroll
        for (int k = 0; k < kEllNb; ++k) cl[k] = k < dg ? ld_claim(rw[k]) : ~key;
        unsigned mask = 0;
#pragma unroll
        for (int k = 0; k < kEllNb; ++k) mask |= (cl[k] == key ? 1u : 0u) << k;
        return mask;
    }

    // Labelled, bottom-up, step 1: every frontier vertex publishes its key in fkey, and the slice's
    // min (degree, id) is accumulated, as in phase_a.
    __device__ void publish_keys(int d, unsigned long long ord0, const Slice& s) {
        const int T = blockDim.x;
        unsigned long long mk = kKeyMax;
        for (int j = (int)threadIdx.x; j < s.cnt; j += T) {
            const int u = sid(s, j);
            if (!in_graph(u)) {
                fail(kErrInternal);
                continue;
            }
            a->fkey[u] = level_key(d, ord0 + (unsigned long long)j);
            mk = min(mk, pack_key(__ldg(a->deg + u), u));
        }
        accumulate(0, mk);
    }

    // The round-0 element of a slice and its row, which phase B expects from phase A.
    __device__ void round0_row(const Slice& s, int& u0, int (&r0)[8]) const {
        u0 = -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) r0[k] = 0;
        if ((int)threadIdx.x < s.cnt) {
            const int u = sid(s, threadIdx.x);
            if (in_graph(u)) {
                u0 = u;
                load_row(u, r0);
            }
        }
    }

    // Labelled, bottom-up, step 2 (after an exchange): every unclaimed vertex takes the smallest key
    // published by a neighbour in level d (key tag d + 1) as its claim.
    __device__ void claims_bottom_up(int d) {
        const int T = blockDim.x, n = a->n;
        const unsigned long long tag = (unsigned long long)(d + 1);
        const int stride = cta_count() * T;
        for (int i0 = cta_rank() * T; i0 < n; i0 += stride) {
            const int i = i0 + (int)threadIdx.x;
            const int w = a->v0 + i;
            const bool open = i < n && ld_claim(w) == kClaimNone;
            unsigned long long best = kKeyMax;
            int dg = 0;
            if (open) {
                int r[8];
                load_row(w, r);
                dg = r[7];
                unsigned long long kk[kEllNb];
#pragma unroll
                for (int k = 0; k < kEllNb; ++k) kk[k] = k < dg ? __ldcg(a->fkey + r[k]) : 0ull;
#pragma unroll
                for (int k = 0; k < kEllNb; ++k)
                    if ((kk[k] >> a->obits) == tag && kk[k] < best) best = kk[k];
            }
            for_long_rows(open, w, dg, [&](int src, int x) {
                unsigned long long v = x >= 0 ? __ldcg(a->fkey + x) : kKeyMax;
                if ((v >> a->obits) != tag) v = kKeyMax;
                v = warp_min_u64(v);
                if ((int)(threadIdx.x & 31) == src && v < best) best = v;
                return false;
            });
            if (open && best != kKeyMax) *claim_p(w) = best;
        }
    }

    // Phase A over a slice whose element j has key level_key(d, ord0 + j). Accumulates the min
    // (degree, id) over the slice. The round-0 row stays in (u0, r0) for phase B.
    __device__ void phase_a(int d, unsigned long long ord0, const Slice& s, int& u0, int (&r0)[8],
                            bool with_key = true) {
        const int T = blockDim.x;
        unsigned long long mk = kKeyMax;
        u0 = -1;
#pragma unroll
        for (int k = 0; k < 8; ++k) r0[k] = 0;
        for (int j0 = 0; j0 < s.cnt; j0 += T) {
            const int j = j0 + (int)threadIdx.x;
            int u = -1, dg = 0;
            unsigned long long key = 0;
            if (j < s.cnt) {
                u = sid(s, j);
                if (!in_graph(u)) {
                    fail(kErrInternal);
                    u = -1;
                } else {
                    int rw[8];
                    load_row(u, rw);
                    key = level_key(d, ord0 + (unsigned long long)j);
                    dg = rw[7];
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k)
                        if (k < dg) atomicMin(claim_p(rw[k]), key);
                    mk = min(mk, pack_key(dg, u));
                    if (j0 == 0) {
                        u0 = u;
#pragma unroll
                        for (int k = 0; k < 8; ++k) r0[k] = rw[k];
                    }
                }
            }
            for_long_rows(u >= 0, u, dg, [&](int src, int w) {
                const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
                if (w >= 0) atomicMin(claim_p(w), kk);
                return false;
            });
        }
        if (with_key) accumulate(0, mk);
    }

    // Phase B over the same slice: the children each vertex owns, in key order then row order
    // (= (parent label, degree, id) order). They go to `ncache` (shared) when this CTA has at most
    // kCache of them, else to `stage` at positions reserved through *stail; with lab_base >= 0
    // (single-CTA runs, where final labels are known) also to perm at labels lab_base + rank.
    // boff_base + j indexes this CTA's per-element offsets (disjoint between CTAs: the label of
    // element j minus the component's first label, or j in single-CTA runs).
    // Returns this CTA's child count and, in *out, the slice they form.
    __device__ int phase_b(int d, unsigned long long ord0, const Slice& s, int u0, const int (&r0)[8],
                           int* ncache, int* stage, int* stail, int lab_base, int boff_base, Slice* out) {
        const int T = blockDim.x;
        const int n = a->n;
        // pass 1: counts and CTA-local offsets
        int carry = 0, off0 = 0;
        unsigned m0 = 0;
        for (int j0 = 0; j0 < s.cnt; j0 += T) {
            const int j = j0 + (int)threadIdx.x;
            int c = 0;
            unsigned mask = 0;
            int u = -1, dg = 0;
            unsigned long long key = 0;
            if (j < s.cnt) {
                u = u0;
                int rw[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) rw[k] = r0[k];
                if (j0 != 0) {
                    u = sid(s, j);
                    if (in_graph(u)) load_row(u, rw);
                }
                if (in_graph(u)) {
                    key = level_key(d, ord0 + (unsigned long long)j);
                    dg = rw[7];
                    mask = owned_mask(rw, dg, key);
                    c = __popc(mask);
                } else {
                    u = -1;
                }
            }
            for_long_rows_claims(u >= 0, u, dg, [&](int src, int w, unsigned long long cw) {
                const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
                const int m = __popc(__ballot_sync(0xffffffffu, w >= 0 && cw == kk));
                if ((int)(threadIdx.x & 31) == src) c += m;
            });
            int tot;
            const int ex = cta_scan(c, &tot);
            if (j0 == 0) {
                m0 = mask;
                off0 = ex;
            } else if (j < s.cnt) {
                a->boff[boff_base + j] = carry + ex;
            }
            carry += tot;
        }
        int* dst = ncache;
        if (carry > kCache) {
            if (threadIdx.x == 0) sm->bc[0] = atomicAdd(stail, carry);
            __syncthreads();
            dst = stage + sm->bc[0];
            __syncthreads();
        }
        out->sh = carry > kCache ? nullptr : ncache;
        out->g = carry > kCache ? dst : nullptr;
        out->step = 1;
        out->cnt = carry;
        // pass 2: write the children
        for (int j0 = 0; j0 < s.cnt; j0 += T) {
            const int j = j0 + (int)threadIdx.x;
            int u = -1, dg = 0, pos = 0;
            unsigned long long key = 0;
            if (j < s.cnt) {
                u = u0;
                int rw[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) rw[k] = r0[k];
                unsigned mask = m0;
                pos = off0;
                key = level_key(d, ord0 + (unsigned long long)j);
                if (j0 != 0) {
                    u = sid(s, j);
                    if (in_graph(u)) {
                        load_row(u, rw);
                        mask = owned_mask(rw, rw[7], key);
                        pos = a->boff[boff_base + j];
                    }
                }
                if (in_graph(u)) {
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k)
                        if (mask & (1u << k)) {
                            prefetch_row(rw[k]);
                            dst[pos] = rw[k];
                            if (lab_base >= 0) {
                                const int lab = lab_base + pos;
                                if ((unsigned)lab < (unsigned)n) a->perm[n - 1 - lab] = rw[k]; else fail(kErrInternal);
                            }
                            ++pos;
                        }
                    dg = rw[7];
                } else {
                    u = -1;
                }
            }
            // the rest of a long row, in row order: a round's owned entries take consecutive
            // positions after the owner's earlier children
            for_long_rows_claims(u >= 0, u, dg, [&](int src, int w, unsigned long long cw) {
                const int lane = threadIdx.x & 31;
                const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
                const bool own = w >= 0 && cw == kk;
                const unsigned bal = __ballot_sync(0xffffffffu, own);
                const int base = __shfl_sync(0xffffffffu, pos, src);
                if (own) {
                    const int p = base + __popc(bal & ((1u << lane) - 1u));
                    prefetch_row(w);
                    dst[p] = w;
                    if (lab_base >= 0) {
                        const int lab = lab_base + p;
                        if ((unsigned)lab < (unsigned)n) a->perm[n - 1 - lab] = w; else fail(kErrInternal);
                    }
                }
                if (lane == src) pos += __popc(bal);
            });
        }
        __syncthreads();
        return carry;
    }

    // Min (degree, id) key over a slice, for every thread of the CTA (the last level of a narrow run).
    __device__ unsigned long long slice_min_key(const Slice& s) {
        unsigned long long key = kKeyMax;
        for (int j = threadIdx.x; j < s.cnt; j += blockDim.x) {
            const int u = sid(s, j);
            if (!in_graph(u)) {
                fail(kErrInternal);
                continue;
            }
            int r[8];
            load_row(u, r);
            key = min(key, pack_key(r[7], u));
        }
        return block_min_u64(key, sm->wkey);
    }

    // Labelled levels of at most kWarpLevel vertices, run by warp 0 alone (one vertex per lane):
    // phase_a's claims and phase_b's ownership with a warp scan and __syncwarp instead of CTA scans
    // and barriers, the row kept in registers between the two. Children take labels from
    // lstart + F in (key, row) order and go to the shared cache as the next level (and to perm,
    // which holds every level for the grid or a wider next level). Runs while the levels stay that
    // narrow (and, on the grid, below the narrow threshold); lane 0 leaves the state in sm->wr
    // (F = 0: the sweep ended with the level of lastF vertices at lstart, lk its least vertex key).
    // Called by the 32 threads of warp 0 only.
    __device__ void warp_labelled(int d, int lstart, int F, int cb, Slice cur) {
        const int lane = threadIdx.x & 31;
        const int n = a->n;
        const unsigned lt = (1u << lane) - 1u;
        unsigned long long lk = kKeyMax;
        int lastF = 0, bad = 0;
        while (true) {
            int u = -1, dg = 0;
            int rw[8];
            unsigned long long key = 0;
            // phase A: every neighbour's claim lowered to this vertex's key
            if (lane < F) {
                const int v = sid(cur, lane);
                if (!in_graph(v)) {
                    bad = 1;
                } else {
                    u = v;
                    load_row(v, rw);
                    dg = rw[7];
                    key = level_key(d, (unsigned long long)lane);
#pragma unroll
                    for (int k = 0; k < kEllNb; ++k)
                        if (k < dg) atomicMin(claim_p(rw[k]), key);
                }
            }
            for_long_rows(u >= 0, u, dg, [&](int src, int w) {
                const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
                if (w >= 0) atomicMin(claim_p(w), kk);
                return false;
            });
            __syncwarp();
            tick(kPhClaim);
            // phase B: the children each vertex owns, counted, then numbered in (key, row) order
            const unsigned mask = u >= 0 ? owned_mask(rw, dg, key) : 0u;
            int cnt = __popc(mask);
            for_long_rows_claims(u >= 0, u, dg, [&](int src, int w, unsigned long long cw) {
                const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
                const int m = __popc(__ballot_sync(0xffffffffu, w >= 0 && cw == kk));
                if (lane == src) cnt += m;
            });
            const int incl = warp_incl_scan(cnt);
            const int kids = __shfl_sync(0xffffffffu, incl, 31);
            int q = incl - cnt;
            int* nc = sm->cache[cb ^ 1];
            const int lab0 = lstart + F;  // first label of the next level
            if (u >= 0) {
#pragma unroll
                for (int k = 0; k < kEllNb; ++k)
                    if (mask & (1u << k)) {
                        const int w = rw[k];
                        prefetch_row(w);
                        if (q < kCache) nc[q] = w;
                        const int lab = lab0 + q;
                        if ((unsigned)lab < (unsigned)n) a->perm[n - 1 - lab] = w; else bad = 1;
                        ++q;
                    }
            }
            for_long_rows_claims(u >= 0, u, dg, [&](int src, int w, unsigned long long cw) {
                const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
                const bool own = w >= 0 && cw == kk;
                const unsigned bal = __ballot_sync(0xffffffffu, own);
                const int base = __shfl_sync(0xffffffffu, q, src);
                if (own) {
                    const int qq = base + __popc(bal & lt);
                    prefetch_row(w);
                    if (qq < kCache) nc[qq] = w;
                    const int lab = lab0 + qq;
                    if ((unsigned)lab < (unsigned)n) a->perm[n - 1 - lab] = w; else bad = 1;
                }
                if (lane == src) q += __popc(bal);
            });
            __syncwarp();
            tick(kPhOwn);
            stat_add(kStNarrow, 1);
            if (kids == 0) {
                lk = warp_min_u64(u >= 0 ? pack_key(dg, u) : kKeyMax);
                lastF = F;
                F = 0;
                break;
            }
            lstart += F;
            F = kids;
            cb ^= 1;
            if (F <= kCache) {
                cur.sh = sm->cache[cb];
                cur.g = nullptr;
                cur.step = 1;
                cur.cnt = F;
            } else {
                cur = perm_range(lstart, F);
            }
            if (++d > n) {
                if (lane == 0) fail_at(kSiteLevels, d);
                bad = 1;
                break;
            }
            if (F > kWarpLevel || (!kCtaOnly && F >= a->narrow_thr)) break;
        }
        bad = __any_sync(0xffffffffu, bad) ? 1 : 0;
        if (lane == 0) {
            if (bad) fail(kErrInternal);
            sm->wr.F = F;
            sm->wr.d = d;
            sm->wr.lstart = lstart;
            sm->wr.cb = cb;
            sm->wr.lastF = lastF;
            sm->wr.lk = lk;
            sm->wr.bad = bad;
        }
    }

    // perm[n-1-(first+j)] = slice element j.
    __device__ void write_labels(const Slice& s, int first) {
        const int n = a->n;
        for (int j = threadIdx.x; j < s.cnt; j += blockDim.x) {
            const int lab = first + j;
            const int v = sid(s, j);
            if ((unsigned)lab < (unsigned)n) a->perm[n - 1 - lab] = v; else fail(kErrInternal);
        }
    }

    // The slices of a level numbered at labels [lstart, lstart + F), for the tier that runs it
    // next: CTA 0 alone below narrow_thr; the CTAs of cluster 0 below mid_thr (middle tier on);
    // otherwise the whole grid, in balanced slices.
    __device__ void choose_tier(int F, int lstart, bool& narrow, bool& mid, Slice& cur) const {
        const int b = cta_rank(), B = cta_count();
        narrow = F < a->narrow_thr;
        mid = !narrow && a->mid_k > 0 && F < a->mid_thr;
        if (narrow) {
            cur = perm_range(lstart, b == 0 ? F : 0);
        } else if (mid) {
            const int K = a->mid_k;
            const int lo = b < K ? (int)((long long)F * b / K) : 0, hi = b < K ? (int)((long long)F * (b + 1) / K) : 0;
            cur = perm_range(lstart + lo, hi - lo);
        } else {
            const int lo = (int)((long long)F * b / B), hi = (int)((long long)F * (b + 1) / B);
            cur = perm_range(lstart + lo, hi - lo);
        }
    }

    // Labelled sweep from root, labels from nv. On return: ecc, the min (degree, id) key of the
    // last level, and the component size (labels nv .. nv+size-1).
    __device__ bool sweep_labelled(int root, int nv, int& ecc, unsigned long long& last_key, int& size) {
        Ctl* c = a->ctl;
        const int b = cta_rank(), B = cta_count();
        const unsigned long long slot = kCtaOnly ? 0ull : ((1ull << a->obits) - 1ull) / (unsigned long long)B;
        if (b == 0 && threadIdx.x == 0) {
            *claim_p(root) = 0;
            a->perm[a->n - 1 - nv] = root;
            sm->cache[0][0] = root;
            if (!kCtaOnly) c->qtail[0] = c->qtail[1] = c->qtail[2] = 0;
        }
        __syncthreads();
        int d = 0;          // index of the current level
        int lstart = nv;    // label of its first vertex
        int cb = 0;         // shared cache buffer holding the current slice (when cached)
        Slice cur;
        cur.sh = sm->cache[0];
        cur.g = nullptr;
        cur.step = 1;
        cur.cnt = (b == 0) ? 1 : 0;
        bool narrow = kCtaOnly || a->narrow_thr > 1;
        bool mid = false;   // the middle tier runs the current level
        int F = 1;          // level size (known in narrow runs and after redistribution)
        // the last completed level (grid runs detect the end one level late)
        int prev_start = nv, prev_size = 1;
        unsigned long long prev_key = kKeyMax;
        while (true) {
            if (narrow) {
                unsigned long long lk = kKeyMax;
                int lastF = 0;
                if (kCtaOnly || b == 0) {
                    while (true) {
                        if (kWarp && F <= kWarpLevel) {
                            // a run of narrow levels on warp 0 (where kWarp is on, as above)
                            if (threadIdx.x < 32)
                                run_warp_labelled<kCtaOnly, kSmem, kAsync, kBottomUp, kWarp>(a, sm, d, lstart, F, cb, cur.sh, cur.g, cur.step);
                            __syncthreads();
                            F = sm->wr.F;
                            d = sm->wr.d;
                            lstart = sm->wr.lstart;
                            cb = sm->wr.cb;
                            if (sm->wr.bad) return false;
                            if (F == 0) {
                                lk = sm->wr.lk;
                                lastF = sm->wr.lastF;
                                break;
                            }
                            if (F <= kCache) {
                                cur.sh = sm->cache[cb];
                                cur.g = nullptr;
                                cur.step = 1;
                                cur.cnt = F;
                            } else {
                                cur = perm_range(lstart, F);
                            }
                            if (!kCtaOnly && F >= a->narrow_thr) break;
                            continue;
                        }
                        int u0;
                        int r0[8];
                        // no (degree, id) minimum per level: it is taken over the last level only
                        phase_a(d, 0, cur, u0, r0, false);
                        if (threadIdx.x == 0) sm->tail = 0;  // read by thread 0 alone, in phase_b
                        __syncthreads();
                        tick(kPhClaim);
                        Slice nxt;
                        int* stage = (d & 1) ? a->qa : a->qb;
                        const int kids = phase_b(d, 0, cur, u0, r0, sm->cache[cb ^ 1], stage, &sm->tail,
                                                 lstart + F, 0, &nxt);
                        tick(kPhOwn);
                        stat_add(kStNarrow, 1);
                        if (kids == 0) {
                            lk = slice_min_key(cur);
                            lastF = F;
                            F = 0;
                            break;
                        }
                        lstart += F;
                        F = kids;
                        cur = nxt;
                        cb ^= 1;
                        if (++d > a->n) {
                            fail_at(kSiteLevels, d);
                            return false;
                        }
                        if (!kCtaOnly && F >= a->narrow_thr) break;
                    }
                    if (kCtaOnly) {
                        last_key = lk;
                        ecc = d;
                        size = lstart + lastF - nv;
                        return true;
                    }
                    if (threadIdx.x == 0) {
                        c->pub_F = F;
                        c->pub_start = lstart;
                        c->pub_ecc = d;
                        c->pub_key = lk;
                        c->pub_lastF = lastF;
                        c->qtail[0] = c->qtail[1] = c->qtail[2] = 0;
                    }
                }
                tick(kPhOther);
                if (!barrier()) return false;
                tick(kPhWaitNarrow);
                if (threadIdx.x == 0) {
                    sm->bc[0] = ldcg(&c->pub_F);
                    sm->bc[1] = ldcg(&c->pub_start);
                    sm->bc[2] = ldcg(&c->pub_ecc);
                    sm->bc[3] = ldcg(&c->pub_lastF);
                    sm->bck = __ldcg(&c->pub_key);
                }
                __syncthreads();
                F = sm->bc[0];
                lstart = sm->bc[1];
                d = sm->bc[2];
                const int lastF2 = sm->bc[3];
                lk = sm->bck;
                __syncthreads();
                if (F == 0) {
                    last_key = lk;
                    ecc = d;
                    size = lstart + lastF2 - nv;
                    return true;
                }
                // the middle tier or the whole grid from here: slices of the level's label range in perm
                choose_tier(F, lstart, narrow, mid, cur);
                continue;
            }
            if constexpr (!kCtaOnly) {
                if (mid) {
                    // ---- middle tier: levels run by the CTAs of cluster 0, ord = b * mslot + j ----
                    // Same phases as a whole-grid level; the exchange goes through distributed
                    // shared memory. The run ends when a level leaves [narrow_thr, mid_thr) or gets
                    // out of balance: the next level is counted and numbered, published, and every
                    // CTA takes its slice of it from perm after the grid barrier.
                    const int K = a->mid_k;
                    if (b < K) {
                        const unsigned long long mslot = ((1ull << a->obits) - 1ull) / (unsigned long long)K;
                        int F2 = 0, fin_start = 0, fin_size = 0, fin_ecc = 0;
                        unsigned long long fin_key = kKeyMax;
                        while (true) {
                            if ((unsigned long long)cur.cnt > mslot) fail(kErrTooLarge);  // every member's exchange fails
                            const unsigned long long ord0 = (unsigned long long)b * mslot;
                            int u0;
                            int r0[8];
                            phase_a(d, ord0, cur, u0, r0);
                            if (threadIdx.x == 0) atomicAdd(&sm->acc_cnt, cur.cnt);
                            tick(kPhClaim);
                            ExResult r;
                            if (!exchange_mid(r)) return false;
                            tick(kPhExchange);
                            stat_add(kStGrid, 1);
                            if (r.total == 0) {  // level d is empty: the sweep ended with level d - 1
                                fin_key = mid_min_key(cepoch - 1);
                                fin_ecc = d - 1;
                                fin_start = prev_start;
                                fin_size = prev_size;
                                break;
                            }
                            write_labels(cur, lstart + r.pre);
                            tick(kPhLabels);
                            if (b == 0 && threadIdx.x == 0) c->qtail[(d + 2) % 3] = 0;
                            Slice nxt;
                            int* stage = (d & 1) ? a->qa : a->qb;
                            const int kids = phase_b(d, ord0, cur, u0, r0, sm->cache[cb ^ 1], stage,
                                                     &c->qtail[(d + 1) % 3], -1, lstart + r.pre - nv, &nxt);
                            tick(kPhOwn);
                            prev_start = lstart;
                            prev_size = r.total;
                            lstart += r.total;
                            if (++d > a->n) {
                                fail_at(kSiteLevels, d);
                                return false;
                            }
                            cur = nxt;
                            if (cur.sh) cb ^= 1;
                            const int fair = (r.total + K - 1) / K;
                            if (r.total < a->narrow_thr || r.total >= a->mid_thr || r.maxcnt > 2 * fair + 64) {
                                if (threadIdx.x == 0) atomicAdd(&sm->acc_cnt, kids);
                                ExResult r2;
                                if (!exchange_mid(r2)) return false;
                                if (r2.total == 0) {
                                    fin_key = mid_min_key(cepoch - 1);
                                    fin_ecc = d - 1;
                                    fin_start = prev_start;
                                    fin_size = prev_size;
                                    break;
                                }
                                write_labels(cur, lstart + r2.pre);
                                F2 = r2.total;
                                break;
                            }
                        }
                        if (b == 0 && threadIdx.x == 0) {
                            c->pub_F = F2;
                            c->pub_start = F2 > 0 ? lstart : fin_start;
                            c->pub_ecc = F2 > 0 ? d : fin_ecc;
                            c->pub_lastF = fin_size;
                            c->pub_key = fin_key;
                        }
                    }
                    tick(kPhOther);
                    if (!barrier()) return false;
                    tick(kPhWaitNarrow);
                    if (threadIdx.x == 0) {
                        sm->bc[0] = ldcg(&c->pub_F);
                        sm->bc[1] = ldcg(&c->pub_start);
                        sm->bc[2] = ldcg(&c->pub_ecc);
                        sm->bc[3] = ldcg(&c->pub_lastF);
                        sm->bck = __ldcg(&c->pub_key);
                    }
                    __syncthreads();
                    F = sm->bc[0];
                    lstart = sm->bc[1];
                    d = sm->bc[2];
                    const int lastF3 = sm->bc[3];
                    const unsigned long long lk3 = sm->bck;
                    __syncthreads();
                    if (F == 0) {
                        last_key = lk3;
                        ecc = d;
                        size = lstart + lastF3 - nv;
                        return true;
                    }
                    choose_tier(F, lstart, narrow, mid, cur);
                    continue;
                }
            }
            // ---- whole-grid level d: this CTA's slice, ord = b * slot + j ----
            if ((unsigned long long)cur.cnt > slot) {
                // the slice's orders would spill into the next CTA's (only with a forced key width:
                // the host otherwise sizes the grid so that slot >= n); every CTA's next wait sees it
                fail(kErrTooLarge);
                return false;
            }
            const unsigned long long ord0 = (unsigned long long)b * slot;
            int u0;
            int r0[8];
            // bottom-up by the size of the previous level (this one's is known after the exchange)
            const bool bu = bottom_up(prev_size, lstart - nv);
            if (bu) {
                publish_keys(d, ord0, cur);
                round0_row(cur, u0, r0);
            } else {
                phase_a(d, ord0, cur, u0, r0);
            }
            if (threadIdx.x == 0) atomicAdd(&sm->acc_cnt, cur.cnt);
            tick(kPhClaim);
            ExResult r;
            if (!exchange(r)) return false;
            tick(kPhExchange);
            stat_add(kStGrid, 1);
            if (r.total == 0) {
                last_key = prev_key;
                ecc = d - 1;
                size = prev_start + prev_size - nv;
                return true;
            }
            if (bu) {
                claims_bottom_up(d);
                if (!barrier()) return false;
                tick(kPhClaim);
            }
            write_labels(cur, lstart + r.pre);
            tick(kPhLabels);
            if (b == 0 && threadIdx.x == 0) c->qtail[(d + 2) % 3] = 0;
            Slice nxt;
            int* stage = (d & 1) ? a->qa : a->qb;
            const int kids = phase_b(d, ord0, cur, u0, r0, sm->cache[cb ^ 1], stage, &c->qtail[(d + 1) % 3], -1,
                                     lstart + r.pre - nv, &nxt);
            tick(kPhOwn);
            prev_start = lstart;
            prev_size = r.total;
            prev_key = r.key;
            lstart += r.total;
            ++d;
            cur = nxt;
            if (cur.sh) cb ^= 1;
            const int fair = (r.total + B - 1) / B;
            if (r.total < a->narrow_thr || (a->mid_k > 0 && r.total < a->mid_thr) || r.maxcnt > 2 * fair + 64) {
                // number level d now and redistribute it (or hand it to CTA 0 or the middle tier)
                if (threadIdx.x == 0) atomicAdd(&sm->acc_cnt, kids);
                ExResult r2;
                if (!exchange(r2)) return false;
                if (r2.total == 0) {
                    last_key = prev_key;
                    ecc = d - 1;
                    size = lstart - nv;
                    return true;
                }
                write_labels(cur, lstart + r2.pre);
                if (!barrier()) return false;
                tick(kPhRedist);
                F = r2.total;
                choose_tier(F, lstart, narrow, mid, cur);
            }
        }
    }

    // Degree-zero vertices are the first components in start-rule order: labels 0..Z-1 in
    // increasing id (an ordered compaction).
    __device__ bool label_isolated(int& Z) {
        const int n = a->n;
        const int R = cta_rank(), C = cta_count();
        const int lo = (int)((long long)n * R / C);
        const int hi = (int)((long long)n * (R + 1) / C);
        int cnt = 0;
        for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) cnt += (__ldg(a->deg + a->v0 + i) == 0);
        accumulate(cnt, kKeyMax);
        ExResult r;
        if (!exchange(r)) return false;
        Z = r.total;
        if (Z == 0) return true;
        int carry = r.pre;
        for (int i0 = lo; i0 < hi; i0 += blockDim.x) {
            const int i = i0 + (int)threadIdx.x;
            const int f = (i < hi && __ldg(a->deg + a->v0 + i) == 0) ? 1 : 0;
            int tot;
            const int ex = cta_scan(f, &tot);
            if (f) {
                const int lab = carry + ex;
                a->perm[n - 1 - lab] = a->v0 + i;
                *claim_p(a->v0 + i) = 0;
            }
            carry += tot;
        }
        return barrier();
    }

    __device__ bool reset_claims(int nv, int size) {
        const int n = a->n;
        const int stride = cta_count() * blockDim.x;
        for (int i = cta_rank() * blockDim.x + threadIdx.x; i < size; i += stride) {
            const int v = ldcg(a->perm + (n - 1 - (nv + i)));
            if (!in_graph(v)) continue;
            *claim_p(v) = kClaimNone;
            if constexpr (kBottomUp) {
                if (a->fkey) a->fkey[v] = 0;  // no stale level tag for the next sweep
            }
        }
        return barrier();
    }

    // Start of the next component: min (degree, id) over the vertices not yet numbered.
    __device__ bool next_start(unsigned long long& out) {
        unsigned long long m = kKeyMax;
        const int stride = cta_count() * blockDim.x;
        for (int i = cta_rank() * blockDim.x + threadIdx.x; i < a->n; i += stride) {
            const int v = a->v0 + i;
            if (ld_claim(v) == kClaimNone) {
                const unsigned long long k = pack_key(__ldg(a->deg + v), v);
                m = k < m ? k : m;
            }
        }
        accumulate(0, m);
        ExResult r;
        if (!exchange(r)) return false;
        out = r.key;
        return true;
    }

    // One connected component: sweeps from its start vertex r (Alg. 2), labelled traversal
    // (Alg. 3) with labels from nv. On return, size = the component's vertex count. With
    // all_left >= 0 (the number of vertices not yet numbered), the call stops after the first
    // sweep when the component is smaller than that, is small enough for the component table to
    // order it at least as fast, and holds less than 3/4 of the vertices left, returning
    // size = -1 (nothing numbered).
    __device__ bool component(int r, int nv, int& size, long long all_left = -1) {
        if (!in_graph(r) || nv < 0 || nv >= a->n) {
            fail_at(kSiteStart, r);
            return false;
        }
        int ecc_prev;
        unsigned long long k1;
        long long reached;
        if (a->fused == 2) {
            // the first sweep labelled as well: a labelled traversal gives the same eccentricity and
            // last level as a levels-only one, and its level code is the faster of the two on the
            // whole grid. Its labels are discarded.
            int sz = 0;
            if (!sweep_labelled(r, nv, ecc_prev, k1, sz)) return false;
            reached = sz;
            tick(kPhOther);
            if (!reset_claims(nv, sz)) return false;
            tick(kPhOther);
        } else if (!sweep_levels(r, ecc_prev, k1, reached)) {
            return false;
        }
        // The start vertex's component does not hold every vertex left: the others get a component
        // table. The component is finished here, its sweep kept, when the table would order it no
        // faster (the whole grid's size on the grid; beyond the one-thread limit on a CTA) or when
        // it holds at least 3/4 of the vertices left (the rest, ordered concurrently afterwards,
        // costs less than the sweep would again): it takes the first labels either way. Otherwise
        // it is left to the table, to run beside the others, and its sweep is discarded.
        const long long keep_min = !kCtaOnly ? (long long)a->cc_big : (kSmem ? 0 : (long long)kTinyMax + 1);
        if (all_left >= 0 && reached < all_left && reached < keep_min && 4 * reached < 3 * all_left) {
            size = -1;
            return true;
        }
        stat_add(kStSweeps, 1);
        stat_add(kStTraversals, 1);
        stat_add(kStLevels, ecc_prev + 1);
        r = (int)(unsigned)(k1 & 0xffffffffu);
        int ecc_root = 0;
        size = 0;
        if (a->fused) {
            while (true) {
                int ecc;
                unsigned long long k2;
                if (!sweep_labelled(r, nv, ecc, k2, size)) return false;
                stat_add(kStSweeps, 1);
                stat_add(kStTraversals, 1);
                stat_add(kStLevels, ecc + 1);
                if (ecc <= ecc_prev) {
                    ecc_root = ecc;
                    break;
                }
                ecc_prev = ecc;
                tick(kPhOther);
                if (!reset_claims(nv, size)) return false;
                tick(kPhOther);
                r = (int)(unsigned)(k2 & 0xffffffffu);
            }
        } else {
            while (true) {
                int ecc;
                unsigned long long k2;
                if (!sweep_levels(r, ecc, k2, reached)) return false;
                stat_add(kStSweeps, 1);
                stat_add(kStTraversals, 1);
                stat_add(kStLevels, ecc + 1);
                if (ecc <= ecc_prev) break;
                ecc_prev = ecc;
                r = (int)(unsigned)(k2 & 0xffffffffu);
            }
            unsigned long long k2;
            if (!sweep_labelled(r, nv, ecc_root, k2, size)) return false;
            stat_add(kStTraversals, 1);
            stat_add(kStLevels, ecc_root + 1);
        }
        stat_add(kStComponents, 1);
        stat_max(kStMaxEcc, ecc_root);
        if (size <= 0) {
            fail(kErrInternal);
            return false;
        }
        return true;
    }

    // ---------------- tiny components: one thread each ----------------
    // A component of a few dozen vertices gives a level-synchronous traversal nothing to share
    // out: each level is a few vertices between CTA barriers. One thread runs the serial method on
    // it instead, so a CTA orders up to blockDim tiny components at once. Rows are stored in
    // (degree, id) order, so a FIFO traversal that appends each dequeued vertex's unvisited
    // neighbours in row order numbers the component as Alg. 1 does (parents in label order,
    // children by increasing degree, ties by id); the level boundaries give Alg. 2 its eccentricity
    // and the last level's minimum (degree, id) vertex. Only the calling thread touches the
    // component's vertices, queue slice and labels (components are disjoint), so plain loads and
    // stores suffice. Visit stamps are negative: the level-synchronous sweeps use positive ones.

    // One traversal from root with stamp `stamp`, the queue in q[0, z). Returns the eccentricity
    // (-1 on a malformed row or a component larger than z); reached = vertices found; last_key =
    // min (degree, id) key of the last level. q holds the Cuthill-McKee order from root.
    __device__ int tiny_bfs(int root, int stamp, int* q, int z, int& reached, unsigned long long& last_key) const {
        *vis_p(root) = stamp;
        q[0] = root;
        int head = 0, tail = 1, lend = 1, ecc = 0;
        unsigned long long lmin = kKeyMax;
        while (true) {
            const int u = q[head++];
            int r[8];
            load_row(u, r);
            const int d = r[7];
            lmin = min(lmin, pack_key(d, u));
#pragma unroll
            for (int k = 0; k < kEllNb; ++k) {
                if (k < d) {
                    const int w = r[k];
                    if (!in_graph(w)) return -1;
                    if (*vis_p(w) != stamp) {
                        if (tail >= z) return -1;
                        *vis_p(w) = stamp;
                        q[tail++] = w;
                        if constexpr (!kSmem) asm volatile("prefetch.global.L1 [%0];" ::"l"(a->ell + 2 * (size_t)w));
                    }
                }
            }
            if (d > kEllNb) {
                const int* row = a->adj + __ldg(a->rowptr + u);
                for (int k = kEllNb; k < d; ++k) {
                    const int w = __ldg(row + k);
                    if (!in_graph(w)) return -1;
                    if (*vis_p(w) != stamp) {
                        if (tail >= z) return -1;
                        *vis_p(w) = stamp;
                        q[tail++] = w;
                    }
                }
            }
            if (head == lend) {
                if (tail == lend) break;  // the level just dequeued was the last
                ++ecc;
                lend = tail;
                lmin = kKeyMax;
            }
        }
        reached = tail;
        last_key = lmin;
        return ecc;
    }

    // Orders the component of table entry t = (start vertex, first label, size, -) by the calling
    // thread alone: Alg. 2's sweeps from the start vertex while the eccentricity grows strictly,
    // then the last root's traversal is the numbering. q: the component's queue slice (t.z ints).
    // Statistics go to st (shared or global, added atomically). Returns false on a failure, with
    // the status set.
    __device__ bool order_tiny(const int4& t, int* q, long long* st) {
        const int z = t.z, y = t.y;
        int stamp = -1, reached = 0;
        unsigned long long k;
        int ecc_prev = tiny_bfs(t.x, stamp--, q, z, reached, k);
        if (ecc_prev < 0 || reached != z) {
            fail_at(kSiteSize, t.x);
            return false;
        }
        long long sweeps = 1, levels = ecc_prev + 1;
        int ecc;
        while (true) {
            const int r = (int)(unsigned)(k & 0xffffffffu);
            ecc = tiny_bfs(r, stamp--, q, z, reached, k);
            if (ecc < 0 || reached != z) {
                fail_at(kSiteSize, r);
                return false;
            }
            ++sweeps;
            levels += ecc + 1;
            if (ecc <= ecc_prev) break;
            ecc_prev = ecc;
        }
        // q[0, z) is the Cuthill-McKee order from the last root: labels y .. y + z - 1, reversed
        const int n = a->n;
        for (int i = 0; i < z; ++i) a->perm[n - 1 - (y + i)] = q[i];
        // the same accounting as component(): without fused sweeps the numbering is one more
        // traversal after the last sweep
        const long long trav = a->fused ? sweeps : sweeps + 1;
        if (!a->fused) levels += ecc + 1;
        atomicAdd((unsigned long long*)&st[kStSweeps], (unsigned long long)sweeps);
        atomicAdd((unsigned long long*)&st[kStTraversals], (unsigned long long)trav);
        atomicAdd((unsigned long long*)&st[kStLevels], (unsigned long long)levels);
        atomicAdd((unsigned long long*)&st[kStComponents], 1ull);
        atomicMax((unsigned long long*)&st[kStMaxEcc], (unsigned long long)ecc);
        return true;
    }

    // ---------------- component table ----------------
    // Finds the components still unnumbered after labels [0, nv) and writes the component table
    // cc_tab (sorted by start key, label offsets from nv; see rcm_cc.cuh). Returns the number of
    // components, -1 when there are more than cc_cap (the caller continues one by one), -2 on a
    // failed wait. sort_smem holds sort_cap keys + sort_cap ints of shared memory; larger tables
    // sort in cc_gkey / cc_gidx.
    __device__ int cc_prepare(int nv, unsigned long long* sort_smem, int sort_cap) {
        const int n = a->n, v0 = a->v0;
        int* counter = kCtaOnly ? &sm->bc[4] : &a->ctl->ncomp;
        // the unnumbered vertices, compacted in the first pass so that the others run over them
        // alone (after a first component that held most of the graph, a small fraction); the
        // frontier queue is idle between components. The grid's counter starts at 0 (the control
        // block is cleared per ordering, and this runs once per ordering).
        int* list = a->qb;
        int* lcount = kCtaOnly ? &sm->bc[5] : &a->ctl->cc_open;
        const int stride = cta_count() * blockDim.x;
        const int lane = threadIdx.x & 31;
        if (kCtaOnly) {
            if (threadIdx.x == 0) *lcount = 0;
            __syncthreads();
        }
        for (int i0 = cta_rank() * blockDim.x; i0 < n; i0 += stride) {
            const int i = i0 + (int)threadIdx.x;
            const int v = v0 + i;
            const bool open = i < n && ld_claim(v) == kClaimNone;
            if (open) {
                a->cc_parent[v] = v;
                a->cc_size[v] = 0;
                a->cc_key[v] = kKeyMax;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, open);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(lcount, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (open) list[base + __popc(bal & ((1u << lane) - 1u))] = v;
            }
        }
        if (cta_rank() == 0 && threadIdx.x == 0) *counter = 0;
        if (!barrier()) return -2;
        if (threadIdx.x == 0) sm->bc[0] = kCtaOnly ? *lcount : ldcg(lcount);
        __syncthreads();
        const int L = sm->bc[0];
        __syncthreads();
        if (L > n) {
            fail_at(kSiteTotal, L);
            return -2;
        }
        for (int i0 = cta_rank() * blockDim.x; i0 < L; i0 += stride) {
            const int i = i0 + (int)threadIdx.x;
            const bool open = i < L;
            const int v = open ? ldcg(list + i) : v0;
            int d = 0;
            if (open) {
                int r[8];
                load_row(v, r);
                d = r[7];
#pragma unroll
                for (int k = 0; k < kEllNb; ++k)
                    if (k < d && r[k] < v && !cc_union(a->cc_parent, v, r[k], v0, v0 + n)) fail_at(kSiteParent, v);
            }
            for_long_rows(open, v, d, [&](int src, int w) {
                const int vv = __shfl_sync(0xffffffffu, v, src);
                if (w >= 0 && w < vv && !cc_union(a->cc_parent, vv, w, v0, v0 + n)) fail_at(kSiteParent, vv);
                return false;
            });
        }
        if (!barrier()) return -2;
        for (int i = cta_rank() * blockDim.x + threadIdx.x; i < L; i += stride) {
            const int v = ldcg(list + i);
            const int r = cc_root((volatile int*)a->cc_parent, v, v0, v0 + n);
            if (r < 0) fail_at(kSiteParent, v);
            if (r == v) {
                const int k = atomicAdd(counter, 1);
                if (k < a->cc_cap) a->cc_roots[k] = v;
            }
        }
        if (!barrier()) return -2;
        if (threadIdx.x == 0) sm->bc[0] = kCtaOnly ? *counter : ldcg(counter);
        __syncthreads();
        const int C = sm->bc[0];
        __syncthreads();
        if (C > a->cc_cap) return -1;
        // sizes and start keys per root (lanes with the same root combine first)
        for (int i0 = cta_rank() * blockDim.x; i0 < L; i0 += stride) {
            const int i = i0 + (int)threadIdx.x;
            bool ok = i < L;
            const int v = ok ? ldcg(list + i) : v0;
            const int root = ok ? cc_root((volatile int*)a->cc_parent, v, v0, v0 + n) : -1;
            if (ok && root < 0) {
                fail_at(kSiteParent, v);
                ok = false;
            }
            unsigned long long key = ok ? pack_key(__ldg(a->deg + v), v) : kKeyMax;
            const unsigned grp = __match_any_sync(0xffffffffu, root);
            unsigned m = grp;
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const unsigned long long k2 = __shfl_sync(grp, key, src);
                key = k2 < key ? k2 : key;
            }
            if (ok && lane == __ffs(grp) - 1) {
                atomicAdd(&a->cc_size[root], __popc(grp));
                atomicMin(&a->cc_key[root], key);
            }
        }
        if (!barrier()) return -2;
        // one CTA: sort by key, label offsets from nv
        if (cta_rank() == 0) {
            int P = 1;
            while (P < C) P <<= 1;
            unsigned long long* sk = P <= sort_cap ? sort_smem : a->cc_gkey;
            int* si = P <= sort_cap ? (int*)(sort_smem + sort_cap) : a->cc_gidx;
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                sk[i] = i < C ? __ldcg(a->cc_key + a->cc_roots[i]) : kKeyMax;
                si[i] = i < C ? i : 0;
            }
            __syncthreads();
            for (int k = 2; k <= P; k <<= 1) {
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int i = threadIdx.x; i < P; i += blockDim.x) {
                        const int ixj = i ^ j;
                        if (ixj > i) {
                            const bool asc = (i & k) == 0;
                            const unsigned long long x = sk[i], y = sk[ixj];
                            if ((x > y) == asc) {
                                sk[i] = y;
                                sk[ixj] = x;
                                const int t = si[i];
                                si[i] = si[ixj];
                                si[ixj] = t;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            int carry = nv;
            for (int i0 = 0; i0 < C; i0 += blockDim.x) {
                const int i = i0 + (int)threadIdx.x;
                const int root = i < C ? a->cc_roots[si[i]] : v0;
                const int sz = i < C ? ldcg(a->cc_size + root) : 0;
                int tot;
                const int ex = cta_scan(sz, &tot);
                if (i < C) a->cc_tab[i] = make_int4((int)(unsigned)(sk[i] & 0xffffffffu), carry + ex, sz, root);
                carry += tot;
            }
            if (threadIdx.x == 0 && carry != n) fail_at(kSiteTotal, carry);
        }
        if (!barrier()) return -2;
        // a failed guard above leaves the table unusable (CTA runs have no exchange to report it)
        if (kCtaOnly && (ld_volatile(a->status) & kErrInternal)) return -2;
        return C;
    }

    // The whole ordering of this graph, one component after another in start-rule order.
    // Returns false on a failed wait or guard.
    __device__ bool run() {
        const int n = a->n;
        int Z = 0;
        if (!label_isolated(Z)) return false;
        stat_add(kStIsolated, Z);
        stat_add(kStComponents, Z);
        int nv = Z;
        bool first = true, tried = false;
        while (nv < n) {
            if (!first && !tried && a->cc_cap > 0) {
                // more than one component: start keys and label ranges of all of them at once
                tried = true;
                const int C = cc_prepare(nv, sm_sort, sm_sort_cap);
                if (C == -2) return false;
                if (C > 0) {
                    if constexpr (!kSmem) {
                        // tiny components first, one per thread, all at once
                        for (int i = threadIdx.x; i < C; i += blockDim.x) {
                            const int4 t = a->cc_tab[i];
                            if (t.z > kTinyMax) continue;
                            if (!tab_ok(t, nv)) {
                                fail_at(kSiteTable, i);
                                break;
                            }
                            if (!order_tiny(t, a->qa + t.y, sm->st)) break;
                        }
                        __syncthreads();
                        if (ld_volatile(a->status) & (kErrInternal | kErrTimeout | kErrTooLarge)) return false;
                    }
                    for (int i = 0; i < C; ++i) {
                        const int4 t = a->cc_tab[i];
                        if (!kSmem && t.z <= kTinyMax) continue;
                        if (!tab_ok(t, nv)) {
                            fail_at(kSiteTable, i);
                            return false;
                        }
                        int size;
                        if (!component(t.x, t.y, size)) return false;
                        if (size != t.z) {
                            fail_at(kSiteSize, i);
                            return false;
                        }
                    }
                    return true;
                }
            }
            unsigned long long k0;
            tick(kPhOther);
            if (!next_start(k0)) return false;
            tick(kPhOther);
            if (k0 == kKeyMax) {
                fail(kErrInternal);
                return false;
            }
            int size;
            const long long left = (first && a->cc_cap > 0) ? (long long)(n - nv) : -1;
            first = false;
            if (!component((int)(unsigned)(k0 & 0xffffffffu), nv, size, left)) return false;
            if (size < 0) continue;
            nv += size;
        }
        return true;
    }
};

template <bool kCtaOnly, bool kSmem, bool kAsync, bool kBottomUp, bool kWarp>
__device__ __noinline__ void run_warp_levels(const EngineArgs* a, EngineSmem* sm, int s, int F, int cb, int* cur,
                                             int* nxt, int ecc, long long reached) {
    Engine<kCtaOnly, kSmem, kAsync, kBottomUp, kWarp> e;
    e.a = a;
    e.sm = sm;
    e.warp_levels(s, F, cb, cur, nxt, ecc, reached);
}

template <bool kCtaOnly, bool kSmem, bool kAsync, bool kBottomUp, bool kWarp>
__device__ __noinline__ void run_warp_labelled(const EngineArgs* a, EngineSmem* sm, int d, int lstart, int F, int cb,
                                               const int* sh, const int* g, int step) {
    Engine<kCtaOnly, kSmem, kAsync, kBottomUp, kWarp> e;
    e.a = a;
    e.sm = sm;
    typename Engine<kCtaOnly, kSmem, kAsync, kBottomUp, kWarp>::Slice cur;
    cur.sh = sh;
    cur.g = g;
    cur.step = step;
    cur.cnt = F;
    e.warp_labelled(d, lstart, F, cb, cur);
}

}  // namespace rcm
