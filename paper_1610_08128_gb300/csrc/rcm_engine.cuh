// rcm_engine.cuh -- the device-side RCM engine: start vertex, pseudo-peripheral sweeps and the
// labelled level loop, generic over the executor that runs it.
//
//   kCtaOnly = false : one graph, all CTAs of a cooperative persistent grid. Levels with a small
//                      frontier run on CTA 0 alone (CTA barriers) while the others wait at the next
//                      grid barrier; wide levels use the whole grid with bounded grid barriers.
//   kCtaOnly = true  : one graph per CTA (batched engine); every level uses CTA barriers only.
//
// Per component (Sec. III-B: Alg. 3 once per connected component, in start-rule order):
//   1. start r0 = lowest-id vertex of minimum degree not yet numbered (min-reduction of packed
//      (degree, id) keys);
//   2. sweep 1: levels-only BFS from r0 (the level structure of Alg. 2 / the do-while of Alg. 4);
//      the next root is the min (degree, id) vertex of the last level (REDUCE in Alg. 4);
//   3. sweeps 2.. (fused mode): labelled BFS (Alg. 3) from the current root. If its eccentricity
//      does not exceed the previous sweep's, the search stops (loop test of Alg. 2) and the labels
//      just computed are the final ones, because the root is the last vertex swept. Otherwise the
//      labels are discarded and the next sweep starts from the last level's min (degree, id).
//      (Separate mode: all sweeps levels-only, then one labelled traversal from the root.)
// Labelled level (body of Alg. 3), frontier kept in label order:
//   phase A  SpMSpV over (select2nd, min): each frontier vertex u with label l_u performs
//            claim[w] = min(claim[w], l_u) on every neighbour. No read of w is needed: vertices
//            numbered earlier already hold a smaller claim (their parent's label, or their own
//            label for a root), so the min leaves them unchanged.
//   phase B  SELECT + SortPerm + "+nv" (Alg. 3): u owns w iff claim[w] == l_u. Rows are pre-sorted
//            by (degree, id) and the frontier is scanned in label order, so an exclusive prefix sum
//            of owned-children counts over the frontier gives every child its rank in (parent
//            label, degree, id) order.
// The reversal of Alg. 1 is fused: the vertex with label L is written to perm[n-1-L]; the level
// queues of the labelled sweeps live inside perm.
#pragma once

#include "rcm_internal.cuh"

namespace rcm {

struct EngineArgs {
    int n;                 // vertices of this graph
    int v0;                // global id of its first vertex (adjacency holds global ids)
    const int* rowptr;     // global rows
    const int* adj;        // sorted rows (first deg[v] entries of each row valid)
    const int* deg;        // global
    int* claim;            // global
    int* vis;              // global
    int* qa;               // this graph's queue (n ints)
    int* qb;               // this graph's queue (n ints)
    int* boff;             // this graph's offsets (n ints)
    int* perm;             // this graph's output segment (n ints); holds global ids while running
    Ctl* ctl;
    int narrow_thr;
    int fused;
    long long limit_ns;
};

enum { kStComponents = 0, kStSweeps, kStTraversals, kStLevels, kStMaxEcc, kStIsolated, kStNarrow, kStGrid };

template <bool kCtaOnly>
struct Engine {
    EngineArgs a;
    unsigned gen;
    int sweep_id;
    int red_k;
    long long st[8];
    int* s_scan;                 // 33 ints of shared memory
    unsigned long long* s_min;   // 32 u64 of shared memory
    int* s_bcast;                // 4 ints of shared memory
    int* s_cnt;                  // 1 int of shared memory

    __device__ void init(const EngineArgs& args, int* scan, unsigned long long* mn, int* bc, int* cnt) {
        a = args;
        gen = 0;
        sweep_id = 0;
        red_k = 0;
        for (int i = 0; i < 8; ++i) st[i] = 0;
        s_scan = scan;
        s_min = mn;
        s_bcast = bc;
        s_cnt = cnt;
    }

    __device__ bool in_graph(int v) const { return (unsigned)(v - a.v0) < (unsigned)a.n; }

    __device__ bool sync() {
        if (kCtaOnly) {
            __syncthreads();
            return true;
        }
        return grid_barrier(a.ctl, gridDim.x, gen, a.limit_ns);
    }

    __device__ int bcast(const int* p) {
        if (threadIdx.x == 0) s_bcast[0] = ldcg(p);
        __syncthreads();
        int r = s_bcast[0];
        __syncthreads();
        return r;
    }

    __device__ unsigned long long bcast64(const unsigned long long* p) {
        if (threadIdx.x == 0) {
            unsigned long long v = __ldcg(p);
            s_bcast[0] = (int)(unsigned)(v & 0xffffffffu);
            s_bcast[1] = (int)(unsigned)(v >> 32);
        }
        __syncthreads();
        unsigned long long r = ((unsigned long long)(unsigned)s_bcast[1] << 32) | (unsigned)s_bcast[0];
        __syncthreads();
        return r;
    }

    __device__ void fail(int bits) { atomicOr(&a.ctl->status, bits); }

    __device__ int cta_rank() const { return kCtaOnly ? 0 : (int)blockIdx.x; }
    __device__ int cta_count() const { return kCtaOnly ? 1 : (int)gridDim.x; }

    // Min of key(i) over i in [0, count) across the executor; every thread gets the result.
    template <class KeyF>
    __device__ bool argmin(int count, KeyF key, unsigned long long& out) {
        unsigned long long m = kKeyMax;
        const int stride = cta_count() * blockDim.x;
        for (int i = cta_rank() * blockDim.x + threadIdx.x; i < count; i += stride) {
            unsigned long long k = key(i);
            m = k < m ? k : m;
        }
        m = block_min_u64(m, s_min);
        if (kCtaOnly) {
            out = m;
            return true;
        }
        const int slot = red_k % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->argmin[(red_k + 1) % 3] = kKeyMax;
        ++red_k;
        if (threadIdx.x == 0 && m != kKeyMax) atomicMin(&a.ctl->argmin[slot], m);
        if (!sync()) return false;
        out = bcast64(&a.ctl->argmin[slot]);
        return true;
    }

    // ---------------- levels-only breadth-first level ----------------
    // Frontier cur[0..F) in any order, strided from `first` by `stride` (CTA-uniform bounds).
    // Newly reached vertices get stamp s in vis[] and are appended to nxt through *cnt
    // (one atomic per warp and neighbour slot).
    __device__ void expand_levels(int s, const int* cur, int F, int* nxt, int* cnt, int first, int stride) {
        const int lane = threadIdx.x & 31;
        for (int i0 = first; i0 < F; i0 += stride) {
            const int i = i0 + threadIdx.x;
            int beg = 0, len = 0;
            if (i < F) {
                const int u = ldcg(cur + i);
                if (!in_graph(u)) {
                    fail(kErrInternal);
                } else {
                    beg = __ldg(a.rowptr + u);
                    len = __ldg(a.deg + u);
                }
            }
            const int mx = __reduce_max_sync(0xffffffffu, len);
            for (int k = 0; k < mx; ++k) {
                bool first_touch = false;
                int w = 0;
                if (k < len) {
                    w = __ldg(a.adj + beg + k);
                    if (ldcg(a.vis + w) != s) first_touch = atomicExch(a.vis + w, s) != s;
                }
                const unsigned m = __ballot_sync(0xffffffffu, first_touch);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int base = 0;
                    if (lane == leader) base = atomicAdd(cnt, __popc(m));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (first_touch) nxt[base + __popc(m & ((1u << lane) - 1u))] = w;
                }
            }
        }
    }

    // Levels-only sweep from root. On return: ecc, and the last non-empty level lastQ[0..lastF).
    __device__ bool sweep_levels(int root, int& ecc, const int*& lastQ, int& lastF) {
        Ctl* c = a.ctl;
        const int s = ++sweep_id;
        if (cta_rank() == 0 && threadIdx.x == 0) {
            a.vis[root] = s;
            a.qa[0] = root;
            if (!kCtaOnly) c->cnt[0] = c->cnt[1] = c->cnt[2] = 0;
        }
        if (!sync()) return false;
        int* cur = a.qa;
        int* nxt = a.qb;
        int F = 1;
        ecc = 0;
        while (true) {
            if (kCtaOnly || F < a.narrow_thr) {
                int last = F;
                if (kCtaOnly || blockIdx.x == 0) {
                    while (F > 0 && (kCtaOnly || F < a.narrow_thr)) {
                        if (threadIdx.x == 0) *s_cnt = 0;
                        __syncthreads();
                        expand_levels(s, cur, F, nxt, s_cnt, 0, blockDim.x);
                        __syncthreads();
                        const int Fn = *s_cnt;
                        __syncthreads();
                        ++st[kStNarrow];
                        if (Fn == 0) {
                            last = F;
                            F = 0;
                            break;
                        }
                        int* t = cur; cur = nxt; nxt = t;
                        F = Fn;
                        ++ecc;
                    }
                    if (kCtaOnly) {
                        lastQ = cur;
                        lastF = last;
                        return true;
                    }
                    if (threadIdx.x == 0) {
                        c->pub_F = F;
                        c->pub_cur = (cur == a.qb) ? 1 : 0;
                        c->pub_ecc = ecc;
                        c->pub_lastF = last;
                        c->cnt[ecc % 3] = 0;
                    }
                }
                if (!sync()) return false;
                const int Fp = bcast(&c->pub_F);
                const int pc = bcast(&c->pub_cur);
                ecc = bcast(&c->pub_ecc);
                cur = pc ? a.qb : a.qa;
                nxt = pc ? a.qa : a.qb;
                if (Fp == 0) {
                    lastQ = cur;
                    lastF = bcast(&c->pub_lastF);
                    return true;
                }
                F = Fp;
                continue;
            }
            int* cnt = &c->cnt[ecc % 3];
            if (blockIdx.x == 0 && threadIdx.x == 0) c->cnt[(ecc + 1) % 3] = 0;
            expand_levels(s, cur, F, nxt, cnt, blockIdx.x * blockDim.x, gridDim.x * blockDim.x);
            if (!sync()) return false;
            const int Fn = bcast(cnt);
            ++st[kStGrid];
            if (Fn == 0) {
                lastQ = cur;
                lastF = F;
                return true;
            }
            int* t = cur; cur = nxt; nxt = t;
            F = Fn;
            ++ecc;
        }
    }

    // ---------------- labelled level (body of Alg. 3) ----------------
    // Frontier = labels [start, start+F); the vertex with label L is perm[n-1-L]. On return
    // total = size of the next level, numbered start+F .. start+F+total-1.
    template <bool kGrid>
    __device__ bool labelled_level(int start, int F, int& total) {
        const int n = a.n;
        const int next = start + F;
        const int T = blockDim.x;
        int lo = 0, hi = F;
        if (kGrid) {
            lo = (int)((long long)F * blockIdx.x / gridDim.x);
            hi = (int)((long long)F * (blockIdx.x + 1) / gridDim.x);
        }
        // phase A: claim[w] = min(claim[w], label(u))
        for (int i = lo + (int)threadIdx.x; i < hi; i += T) {
            const int u = ldcg(a.perm + (n - 1 - (start + i)));
            if (!in_graph(u)) {
                fail(kErrInternal);
                continue;
            }
            const int lu = start + i;
            const int beg = __ldg(a.rowptr + u), len = __ldg(a.deg + u);
            for (int k = 0; k < len; ++k) atomicMin(a.claim + __ldg(a.adj + beg + k), lu);
        }
        if (kGrid) {
            if (!sync()) return false;
        } else {
            __syncthreads();
        }
        // phase B1: owned-children counts and CTA-local exclusive offsets in frontier order
        int carry = 0;
        for (int i0 = lo; i0 < hi; i0 += T) {
            const int i = i0 + (int)threadIdx.x;
            int cnt = 0;
            if (i < hi) {
                const int u = ldcg(a.perm + (n - 1 - (start + i)));
                if (in_graph(u)) {
                    const int lu = start + i;
                    const int beg = __ldg(a.rowptr + u), len = __ldg(a.deg + u);
                    for (int k = 0; k < len; ++k) cnt += (ldcg(a.claim + __ldg(a.adj + beg + k)) == lu);
                }
            }
            int tot;
            const int ex = block_excl_scan(cnt, &tot, s_scan);
            if (i < hi) a.boff[i] = carry + ex;
            carry += tot;
        }
        int pre = 0;
        if (kGrid) {
            if (threadIdx.x == 0) a.ctl->blocksum[blockIdx.x] = carry;
            if (!sync()) return false;
            int x = 0, y = 0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += T) {
                const int v = ldcg(a.ctl->blocksum + b);
                y += v;
                if (b < (int)blockIdx.x) x += v;
            }
            pre = block_sum(x, s_scan);
            total = block_sum(y, s_scan);
        } else {
            total = carry;
        }
        // phase B2: children at next + pre + offset, in (parent label, degree, id) order
        for (int i = lo + (int)threadIdx.x; i < hi; i += T) {
            const int u = ldcg(a.perm + (n - 1 - (start + i)));
            if (!in_graph(u)) continue;
            const int lu = start + i;
            const int beg = __ldg(a.rowptr + u), len = __ldg(a.deg + u);
            int lab = next + pre + a.boff[i];
            for (int k = 0; k < len; ++k) {
                const int w = __ldg(a.adj + beg + k);
                if (ldcg(a.claim + w) == lu) {
                    if ((unsigned)lab < (unsigned)n) {
                        a.perm[n - 1 - lab] = w;
                    } else {
                        fail(kErrInternal);
                    }
                    ++lab;
                }
            }
        }
        if (kGrid) {
            if (!sync()) return false;
        } else {
            __syncthreads();
        }
        return true;
    }

    // Labelled sweep from root, labels from nv. On return: ecc and the last level's label range
    // [lastStart, lastStart + lastF).
    __device__ bool sweep_labelled(int root, int nv, int& ecc, int& lastStart, int& lastF) {
        Ctl* c = a.ctl;
        if (cta_rank() == 0 && threadIdx.x == 0) {
            a.claim[root] = nv;
            a.perm[a.n - 1 - nv] = root;
        }
        if (kCtaOnly || a.narrow_thr <= 1) {
            if (!sync()) return false;
        }
        int start = nv, F = 1;
        ecc = 0;
        while (true) {
            if (kCtaOnly || F < a.narrow_thr) {
                int last = F;
                if (kCtaOnly || blockIdx.x == 0) {
                    __syncthreads();
                    while (F > 0 && (kCtaOnly || F < a.narrow_thr)) {
                        int total;
                        labelled_level<false>(start, F, total);
                        ++st[kStNarrow];
                        if (total == 0) {
                            last = F;
                            F = 0;
                            break;
                        }
                        start += F;
                        F = total;
                        ++ecc;
                    }
                    if (kCtaOnly) {
                        lastStart = start;
                        lastF = last;
                        return true;
                    }
                    if (threadIdx.x == 0) {
                        c->pub_F = F;
                        c->pub_start = start;
                        c->pub_ecc = ecc;
                        c->pub_lastF = last;
                    }
                }
                if (!sync()) return false;
                const int Fp = bcast(&c->pub_F);
                start = bcast(&c->pub_start);
                ecc = bcast(&c->pub_ecc);
                if (Fp == 0) {
                    lastStart = start;
                    lastF = bcast(&c->pub_lastF);
                    return true;
                }
                F = Fp;
                continue;
            }
            int total = 0;
            if (!labelled_level<true>(start, F, total)) return false;
            ++st[kStGrid];
            if (total == 0) {
                lastStart = start;
                lastF = F;
                return true;
            }
            start += F;
            F = total;
            ++ecc;
        }
    }

    // Degree-zero vertices are the first components in start-rule order: they take labels
    // 0..Z-1 in increasing id (an ordered compaction).
    __device__ bool label_isolated(int& Z) {
        const int n = a.n;
        const int R = cta_rank(), C = cta_count();
        const int lo = (int)((long long)n * R / C);
        const int hi = (int)((long long)n * (R + 1) / C);
        int cnt = 0;
        for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) cnt += (__ldg(a.deg + a.v0 + i) == 0);
        cnt = block_sum(cnt, s_scan);
        int carry = 0;
        if (kCtaOnly) {
            Z = cnt;
        } else {
            if (threadIdx.x == 0) a.ctl->blocksum[blockIdx.x] = cnt;
            if (!sync()) return false;
            int x = 0, y = 0;
            for (int b = threadIdx.x; b < C; b += blockDim.x) {
                const int v = ldcg(a.ctl->blocksum + b);
                y += v;
                if (b < R) x += v;
            }
            carry = block_sum(x, s_scan);
            Z = block_sum(y, s_scan);
        }
        if (Z == 0) return true;
        for (int i0 = lo; i0 < hi; i0 += blockDim.x) {
            const int i = i0 + (int)threadIdx.x;
            const int f = (i < hi && __ldg(a.deg + a.v0 + i) == 0) ? 1 : 0;
            int tot;
            const int ex = block_excl_scan(f, &tot, s_scan);
            if (f) {
                const int lab = carry + ex;
                a.perm[n - 1 - lab] = a.v0 + i;
                a.claim[a.v0 + i] = lab;
            }
            carry += tot;
        }
        return sync();
    }

    __device__ bool reset_claims(int nv, int size) {
        const int n = a.n;
        const int stride = cta_count() * blockDim.x;
        for (int i = cta_rank() * blockDim.x + threadIdx.x; i < size; i += stride) {
            const int v = ldcg(a.perm + (n - 1 - (nv + i)));
            if (in_graph(v)) a.claim[v] = kIntMax;
        }
        return sync();
    }

    // The whole ordering of this graph. Returns false on a failed wait or guard.
    __device__ bool run() {
        const int n = a.n;
        int Z = 0;
        if (!label_isolated(Z)) return false;
        st[kStIsolated] = Z;
        st[kStComponents] = Z;
        int nv = Z;
        const int* deg = a.deg;
        const int* claim = a.claim;
        const int v0 = a.v0;
        while (nv < n) {
            unsigned long long k0;
            if (!argmin(n, [&](int i) {
                    const int v = v0 + i;
                    return ldcg(claim + v) == kIntMax ? pack_key(__ldg(deg + v), v) : kKeyMax;
                }, k0))
                return false;
            if (k0 == kKeyMax) {
                fail(kErrInternal);
                return false;
            }
            ++st[kStComponents];
            int r = (int)(unsigned)(k0 & 0xffffffffu);
            int ecc_prev, lastF;
            const int* lastQ;
            if (!sweep_levels(r, ecc_prev, lastQ, lastF)) return false;
            ++st[kStSweeps];
            ++st[kStTraversals];
            st[kStLevels] += ecc_prev + 1;
            unsigned long long k1;
            if (!argmin(lastF, [&](int i) {
                    const int v = ldcg(lastQ + i);
                    return pack_key(__ldg(deg + v), v);
                }, k1))
                return false;
            r = (int)(unsigned)(k1 & 0xffffffffu);
            int size = 0, ecc_root = 0;
            if (a.fused) {
                while (true) {
                    int ecc, ls, lf;
                    if (!sweep_labelled(r, nv, ecc, ls, lf)) return false;
                    ++st[kStSweeps];
                    ++st[kStTraversals];
                    st[kStLevels] += ecc + 1;
                    size = ls + lf - nv;
                    if (ecc <= ecc_prev) {
                        ecc_root = ecc;
                        break;
                    }
                    ecc_prev = ecc;
                    unsigned long long k2;
                    if (!argmin(lf, [&](int i) {
                            const int v = ldcg(a.perm + (n - 1 - (ls + i)));
                            return pack_key(__ldg(deg + v), v);
                        }, k2))
                        return false;
                    if (!reset_claims(nv, size)) return false;
                    r = (int)(unsigned)(k2 & 0xffffffffu);
                }
            } else {
                while (true) {
                    int ecc;
                    if (!sweep_levels(r, ecc, lastQ, lastF)) return false;
                    ++st[kStSweeps];
                    ++st[kStTraversals];
                    st[kStLevels] += ecc + 1;
                    if (ecc <= ecc_prev) break;
                    ecc_prev = ecc;
                    unsigned long long k2;
                    if (!argmin(lastF, [&](int i) {
                            const int v = ldcg(lastQ + i);
                            return pack_key(__ldg(deg + v), v);
                        }, k2))
                        return false;
                    r = (int)(unsigned)(k2 & 0xffffffffu);
                }
                int ls, lf;
                if (!sweep_labelled(r, nv, ecc_root, ls, lf)) return false;
                ++st[kStTraversals];
                st[kStLevels] += ecc_root + 1;
                size = ls + lf - nv;
            }
            if (ecc_root > st[kStMaxEcc]) st[kStMaxEcc] = ecc_root;
            if (size <= 0) {
                fail(kErrInternal);
                return false;
            }
            nv += size;
        }
        return true;
    }
};

}  // namespace rcm
