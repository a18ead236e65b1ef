// Primal network simplex for the uncapacitated min-cost flow, one CTA per
// instance (the min-cost flow of the network-simplex section: block search
// pivoting, run to optimality).  The kernel is persistent: each CTA takes
// instances from a device counter, largest first.
//
// GPU layout.  Pricing is the parallel part: the whole CTA evaluates a block
// of arcs (reduced cost c - pi(tail) + pi(head)) and reduces to the most
// negative one, the next block prefetched into L2.  The two half-cycles of the
// entering arc are found by the whole CTA with the preorder ancestor test
// pos(a) <= pos(b) < pos(a) + size(a) (a ballot scan over preorder positions;
// no depths are kept; trees in global memory are walked by two lanes
// instead).  One warp then finds the leaving arc, changes the flow and
// re-roots the cut path.  The spanning tree is kept as an explicit preorder
// array (ord, pos, size), so re-hanging the cut subtree is a handful of
// contiguous segment moves done by all threads plus one potential shift -- no
// pointer chasing over the subtree.  Up to 9216 nodes the node arrays live in
// shared memory with 16-bit indices (24 bytes per node); larger trees keep
// 32-bit arrays in global memory.
//
// Big-M start: node i has an artificial arc to (supply >= 0) or from (< 0) an
// extra root, of cost big (more than any path of real arcs) plus an optional
// per-node offset >= 0 that a warm start uses to place its tree components'
// potentials; zero-flow tree arcs point to the root (strongly feasible tree),
// and the leaving arc is the last blocking arc met when the cycle is walked
// from the apex in the direction of the entering arc, which rules out cycling.
// An instance may instead carry its own strongly feasible start (warm start).
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"
#include "netsimplex.cuh"
#include "prims.cuh"

namespace pd {

PD_D uint64_t ns_now() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

PD_D void arc_ends(const NSInst& I, int64_t a, int32_t* t, int32_t* h) {
    if (a < I.mst) {  // m + n < 2^31, so 32-bit division is exact
        int32_t i = (int32_t)a / (int32_t)I.nT;
        *t = i;
        *h = (int32_t)I.nS + ((int32_t)a - i * (int32_t)I.nT);
    } else if (a < I.m) {
        *t = I.tail[a - I.mst];
        *h = I.head[a - I.mst];
    } else {
        int32_t i = (int32_t)(a - I.m);
        if (I.supply[i] >= 0) {
            *t = i;
            *h = I.n;
        } else {
            *t = I.n;
            *h = i;
        }
    }
}

PD_D int64_t arc_cost(const NSInst& I, int64_t a, int64_t big) {
    if (a < I.mst) return I.cmat[a];
    if (a < I.m) return I.cost[a - I.mst];
    return I.art ? big + I.art[a - I.m] : big;  // artificial arc of node a - m
}

// Node arrays of the spanning tree.  IX = uint16_t: compact layout in shared
// memory (parent, subtree size, preorder position and the preorder itself as
// 16-bit indices); IX = int32_t: global memory.  Flow and direction of the
// pred arc share one word: bit 31 = the arc points from the node to its parent.
template <typename IX>
struct Tree {
    int64_t* pi;
    int32_t* pred;
    uint32_t* fu;
    IX* par;
    IX* sz;
    IX* ps;
    IX* od;
    PD_D int32_t parent(int32_t v) const {
        IX p = par[v];
        return p == (IX)~(IX)0 ? -1 : (int32_t)p;
    }
    PD_D void set_parent(int32_t v, int32_t p) { par[v] = p < 0 ? (IX)~(IX)0 : (IX)p; }
    PD_D int32_t flow(int32_t v) const { return (int32_t)(fu[v] & 0x7fffffffu); }
    PD_D bool up(int32_t v) const { return (fu[v] >> 31) != 0; }
    PD_D void set_fu(int32_t v, int32_t f, bool u) { fu[v] = (uint32_t)f | (u ? 0x80000000u : 0u); }
    PD_D void add_flow(int32_t v, int32_t d) { fu[v] = (uint32_t)((int32_t)fu[v] + d); }  // flow stays in [0, 2^31)
};

constexpr int NS_LMAX = 512;     // half-cycle entries kept in shared memory
constexpr int NS_PR = 8;         // cost-matrix loads in flight per thread while pricing
constexpr int NS_SEGSM = 65;     // re-hang segments kept in shared memory (paths shorter than 32)
constexpr int NS_REGS = 9;       // re-hang buffered in registers when it moves at most 9 * 1024 positions

template <typename IX>
__device__ __forceinline__ void ns_body(NSInst& G, NSInst& I, Tree<IX>& T) {
    constexpr unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t n = I.n, root = n, N1 = n + 1;
    const int64_t M = I.m + n;  // arcs including the artificial ones (< 2^31)
    const int64_t big = I.big;
    __shared__ int32_t pa[NS_LMAX], pb[NS_LMAX];
    int32_t* gpa = I.path;
    int32_t* gpb = I.path + N1;
    __shared__ int32_t s_la, s_lb;
    __shared__ int32_t s_wkey[2][32];    // per-warp pricing minima (clamped), double-buffered
    __shared__ uint32_t s_widx[2][32];
    __shared__ int64_t s_wval[2][32];    // exact reduced cost of each warp's winner
    __shared__ int32_t s_cnt[2][32];
    __shared__ int64_t s_dpi;
    __shared__ int32_t s_go, s_status, s_scan;
    __shared__ int32_t s_L0, s_S, s_pr, s_nseg, s_segsm;
    __shared__ int32_t sseg[3][NS_SEGSM];
    const int32_t SEGN = 2 * n + 3;

    // ---- initial tree: the one given in the record, or the root star -----
    if (I.init_tree) {
        for (int32_t v = tid; v < N1; v += NS_THREADS) {
            const int32_t f = G.flow[v];
            const bool u = G.up[v] != 0;
            T.pi[v] = G.pi[v];
            T.pred[v] = G.pred[v];
            T.set_parent(v, G.parent[v]);
            T.sz[v] = (IX)G.size[v];
            T.ps[v] = (IX)G.pos[v];
            T.od[v] = (IX)G.ord[v];
            T.set_fu(v, f, u);
        }
        if (tid == 0) s_status = 0;
    }
    for (int32_t i = tid; i < n && !I.init_tree; i += NS_THREADS) {
        int64_t s = I.supply[i];
        T.set_parent(i, root);
        T.pred[i] = (int32_t)(I.m + i);
        T.set_fu(i, (int32_t)(s >= 0 ? s : -s), s >= 0);
        const int64_t ca = I.art ? big + I.art[i] : big;  // the artificial arc's cost
        T.pi[i] = s >= 0 ? ca : -ca;                      // its reduced cost is 0
        T.od[1 + i] = (IX)i;
        T.ps[i] = (IX)(1 + i);
        T.sz[i] = (IX)1;
    }
    if (tid == 0 && !I.init_tree) {
        T.set_parent(root, -1);
        T.pred[root] = -1;
        T.set_fu(root, 0, false);
        T.pi[root] = 0;
        T.od[0] = (IX)root;
        T.ps[root] = 0;
        T.sz[root] = (IX)N1;
        s_status = 0;
    }
    __syncthreads();
    const uint64_t t0 = ns_now();
    int64_t pivots = 0, degen = 0, nscan = 0;
    const int64_t B = I.block < 1 ? 1 : I.block;
    int64_t next = 0;  // first arc of the next pricing block (same in every thread)
    int pb_buf = 0;

    for (;;) {
        // ---- pricing: blocks of B arcs from `next`; the most negative reduced
        // cost of the first block that has one enters.  Every thread ends with
        // the same (ent, rc).  Across threads the reduction compares a 32-bit
        // key, -bits(float(-rc)), which is monotone in rc (equal only within
        // float rounding; ties go to the smallest arc index): any arc of
        // negative reduced cost is a valid entering arc, and the choice stays
        // deterministic.
        int64_t scanned = 0, a0 = next;
        int64_t ent = -1, rc = 0;
        while (scanned < M) {
            const int64_t aend = a0 + B < M ? a0 + B : M;
            const int64_t len = aend - a0;
            {
                // the costs never change: pull the next block into L2 while this
                // one is priced (and, when this block has the entering arc,
                // while the pivot runs)
                const int64_t pf = (aend >= M ? 0 : aend) + 8 * (int64_t)tid;
                if (pf + 8 <= I.mst && 8 * (int64_t)tid < B)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(I.cmat + pf));
            }
            // per thread: the most negative reduced cost (lb) and its arc (li);
            // arcs are visited in ascending order, so the strict < keeps the
            // smallest index among equal costs.  Arc ids are below 2^31.
            int64_t lb = 0;
            int32_t li = -1;
            // consecutive lanes take consecutive arcs: coalesced 4-byte loads,
            // and the sink potentials pi(nS + j) they read are consecutive
            // 8-byte words of shared memory (no bank conflicts)
            const int32_t iend = (int32_t)(aend < I.mst ? aend : I.mst);
            const int32_t nT = (int32_t)I.nT, nS = (int32_t)I.nS;
            const int32_t step_i = NS_THREADS / nT, step_j = NS_THREADS - step_i * nT;
            for (int32_t base = (int32_t)a0; base < iend; base += NS_PR * NS_THREADS) {
                int32_t cv[NS_PR];
#pragma unroll
                for (int q = 0; q < NS_PR; q++) {
                    const int32_t a = base + tid + q * NS_THREADS;  // no overflow: m + n + 8 NS_THREADS < 2^31
                    cv[q] = a < iend ? __ldcg(I.cmat + a) : 0;
                }
                // row i and column j of arc base + tid, then NS_THREADS arcs further per step
                const int32_t a1 = base + tid;
                int32_t i = a1 / nT, j = a1 - i * nT;
#pragma unroll
                for (int q = 0; q < NS_PR; q++) {
                    const int32_t a = a1 + q * NS_THREADS;
                    if (a < iend) {
                        const int64_t r = (int64_t)cv[q] - T.pi[i] + T.pi[nS + j];
                        if (r < lb) {
                            lb = r;
                            li = a;
                        }
                    }
                    i += step_i;
                    j += step_j;
                    if (j >= nT) {
                        j -= nT;
                        ++i;
                    }
                }
            }
            // explicit arcs (the diagonal node's, or a whole arc list), then the
            // artificial arcs of the initial tree
            for (int64_t a = (a0 > I.mst ? a0 : I.mst) + tid; a < aend; a += NS_THREADS) {
                int32_t t, h;
                arc_ends(I, a, &t, &h);
                const int64_t r = arc_cost(I, a, big) - T.pi[t] + T.pi[h];
                if (r < lb) {
                    lb = r;
                    li = (int32_t)a;
                }
            }
            const int32_t key = lb < 0 ? -__float_as_int((float)(-lb)) : 0;
            const int32_t wmin = __reduce_min_sync(FULL, key);
            const uint32_t cand = (wmin < 0 && key == wmin) ? (uint32_t)li : 0xffffffffu;
            const uint32_t widx = __reduce_min_sync(FULL, cand);
            if (lane == 0) {
                s_wkey[pb_buf][wid] = wmin;
                s_widx[pb_buf][wid] = widx;
            }
            if (wmin < 0 && cand == widx) s_wval[pb_buf][wid] = lb;
            __syncthreads();
            const int32_t k2 = s_wkey[pb_buf][lane];
            const uint32_t i2 = s_widx[pb_buf][lane];
            const int32_t bmin = __reduce_min_sync(FULL, k2);
            const uint32_t c2 = (bmin < 0 && k2 == bmin) ? i2 : 0xffffffffu;
            const uint32_t bidx = __reduce_min_sync(FULL, c2);
            scanned += len;
            nscan += len;
            a0 = aend >= M ? 0 : aend;
            if (bmin < 0) {
                const int wl = __ffs(__ballot_sync(FULL, c2 == bidx)) - 1;
                rc = s_wval[pb_buf][wl];
                ent = bidx;
                next = a0;
                pb_buf ^= 1;
                break;
            }
            pb_buf ^= 1;
        }
        if (ent < 0) break;  // no arc with a negative reduced cost: optimal
        if (pivots >= I.max_pivots) {
            if (tid == 0) s_status = 2;
            break;
        }
        pivots++;

        // ---- the two half-cycles: from i up to (not including) the apex, and
        // from j up to the apex.  PA(0) = i, PA(la - 1) = the child of the apex
        // on i's side; PB likewise from j.
        int32_t i, j;
        arc_ends(I, ent, &i, &j);
        // lanes 0 and 1 of warp 0 walk up from i and from j until they reach
        // an ancestor of the other end (preorder test pos(v) <= pos(x) <
        // pos(v) + size(v)); on the shared-memory layout a side longer than
        // I.walk nodes is left to the CTA-wide scan below (a step of the walk
        // is a dependent shared-memory round trip, the scan costs about
        // N / 1024 positions per thread and two barriers, whatever the path)
        if (wid == 0) {
            if (lane < 2) {
                int32_t u = lane == 0 ? i : j;
                const int32_t tgt = lane == 0 ? (int32_t)T.ps[j] : (int32_t)T.ps[i];
                int32_t* sp = lane == 0 ? pa : pb;
                int32_t* gp = lane == 0 ? gpa : gpb;
                const int32_t cap = sizeof(IX) == 2 ? I.walk : n;
                int32_t len = 0;
                for (;;) {
                    if (u < 0 || len >= n) {  // no ancestor found within n steps: corrupt tree
                        len = -1;
                        break;
                    }
                    const int32_t pu = T.ps[u];
                    if (pu <= tgt && tgt < pu + (int32_t)T.sz[u]) break;
                    if (len >= cap) {  // too long for one lane: the scan finds it
                        len = -2;
                        break;
                    }
                    if (len < NS_LMAX) sp[len] = u; else gp[len] = u;
                    len++;
                    u = T.parent(u);
                }
                if (lane == 0) s_la = len; else s_lb = len;
            }
            __syncwarp();
            if (lane == 0) s_scan = (s_la == -2 || s_lb == -2) ? 1 : 0;
        }
        if constexpr (sizeof(IX) == 2) {
            __syncthreads();
            if (s_scan) {
                // whole CTA: a node is on i's side iff it is an ancestor of i (or i)
                // and not of j, by the preorder test pos(v) <= pos(x) < pos(v) +
                // size(v).  Each warp scans a contiguous range of preorder positions
                // (so matches come out ordered from the apex down) and counts its
                // matches; the few warps with matches scan their range again and
                // write each match at its rank.
                const int32_t pi_ = T.ps[i], pj = T.ps[j];
                const int32_t C = (((N1 + 31) / 32) + 31) & ~31;  // positions per warp
                const int32_t x0 = wid * C;
                // an ancestor's position is at most the descendant's: no warp looks
                // past max(pos(i), pos(j))
                const int32_t xmax = pi_ > pj ? pi_ : pj;
                const int32_t iters = xmax < x0 ? 0 : min(C >> 5, ((xmax - x0) >> 5) + 1);
                auto sides = [&](int32_t it, uint32_t* bI, uint32_t* bJ) {
                    const int32_t x = x0 + (it << 5) + lane;
                    bool inI = false, inJ = false;
                    if (x < N1) {
                        const int32_t e = x + (int32_t)T.sz[T.od[x]];
                        const bool ai = x <= pi_ && pi_ < e, aj = x <= pj && pj < e;
                        inI = ai && !aj;
                        inJ = aj && !ai;
                    }
                    *bI = __ballot_sync(FULL, inI);
                    *bJ = __ballot_sync(FULL, inJ);
                };
                int32_t cI = 0, cJ = 0;
                for (int32_t it = 0; it < iters; it++) {
                    uint32_t bI, bJ;
                    sides(it, &bI, &bJ);
                    cI += __popc(bI);
                    cJ += __popc(bJ);
                }
                if (lane == 0) {
                    s_cnt[0][wid] = cI;
                    s_cnt[1][wid] = cJ;
                }
                __syncthreads();
                const int32_t mI = s_cnt[0][lane], mJ = s_cnt[1][lane];
                int32_t oI = __reduce_add_sync(FULL, lane < wid ? mI : 0);
                int32_t oJ = __reduce_add_sync(FULL, lane < wid ? mJ : 0);
                const int32_t la = __reduce_add_sync(FULL, mI), lb = __reduce_add_sync(FULL, mJ);
                const uint32_t below = (1u << lane) - 1u;
                const int32_t iters2 = (cI + cJ) > 0 ? iters : 0;  // warps without a match skip
                for (int32_t it = 0; it < iters2; it++) {
                    uint32_t bI, bJ;
                    sides(it, &bI, &bJ);
                    if ((bI | bJ) == 0) continue;
                    const int32_t x = x0 + (it << 5) + lane;
                    if ((bI >> lane) & 1u) {
                        const int32_t t = la - 1 - (oI + __popc(bI & below));
                        const int32_t v = T.od[x];
                        if (t < NS_LMAX) pa[t] = v; else gpa[t] = v;
                    }
                    if ((bJ >> lane) & 1u) {
                        const int32_t t = lb - 1 - (oJ + __popc(bJ & below));
                        const int32_t v = T.od[x];
                        if (t < NS_LMAX) pb[t] = v; else gpb[t] = v;
                    }
                    oI += __popc(bI);
                    oJ += __popc(bJ);
                }
                if (tid == 0) {
                    s_la = la;
                    s_lb = lb;
                }
                __syncthreads();
            }
        }

        // ---- pivot (one warp): leaving arc, flow change, re-rooting ----------
        if (wid == 0) {
            const int32_t la = s_la, lb = s_lb;
#define PA(t) ((t) < NS_LMAX ? pa[t] : gpa[t])
#define PB(t) ((t) < NS_LMAX ? pb[t] : gpb[t])
            // leaving arc: last blocking arc walking from the apex along the
            // cycle -- on the i-side the one closest to i (smallest index), on
            // the j-side the one closest to the apex (largest index), j-side
            // preferred on ties.
            uint32_t li_f = 0xffffffffu, li_t = 0xffffffffu;  // i-side: smallest flow, then smallest index
            int32_t lj_f = INT32_MAX, lj_t = -1;                // j-side: smallest flow, then largest index
            for (int32_t t = lane; t < la; t += 32) {
                const uint32_t w = T.fu[PA(t)];
                if (w >> 31) {  // points up: against the cycle on the i-side
                    const uint32_t f = w & 0x7fffffffu;
                    if (f < li_f) {  // t grows within a lane: ties keep the smaller index
                        li_f = f;
                        li_t = (uint32_t)t;
                    }
                }
            }
            for (int32_t t = lane; t < lb; t += 32) {
                const uint32_t w = T.fu[PB(t)];
                if (!(w >> 31)) {
                    const int32_t f = (int32_t)w;
                    if (f <= lj_f) {  // ties take the larger index
                        lj_f = f;
                        lj_t = t;
                    }
                }
            }
            const uint32_t mfi = __reduce_min_sync(FULL, li_f);
            const uint32_t mti = __reduce_min_sync(FULL, li_f == mfi ? li_t : 0xffffffffu);
            const int32_t mfj = (int32_t)__reduce_min_sync(FULL, (uint32_t)lj_f);
            const int32_t mtj = __reduce_max_sync(FULL, lj_f == mfj ? lj_t : -1);
            const int32_t fi = mfi == 0xffffffffu ? INT32_MAX : (int32_t)mfi;
            const int32_t ti = mti == 0xffffffffu ? INT32_MAX : (int32_t)mti;
            const int32_t fj = mfj, tj = mtj;
            int side;
            int32_t delta, tl;
            if (la < 0 || lb < 0) {
                side = -1;
                delta = 0;
                tl = 0;
            } else if (tj >= 0 && fj <= fi) {
                side = 2;
                delta = fj;
                tl = tj;
            } else if (ti != INT32_MAX) {
                side = 1;
                delta = fi;
                tl = ti;
            } else {
                side = 0;
                delta = 0;
                tl = 0;
            }
            if (side <= 0) {
                if (lane == 0) {
                    s_status = side == 0 ? 3 : 4;
                    s_go = 0;
                }
            } else {
                if (delta > 0) {
                    for (int32_t t = lane; t < la; t += 32) {
                        int32_t x = PA(t);
                        T.add_flow(x, T.up(x) ? -delta : delta);
                    }
                    for (int32_t t = lane; t < lb; t += 32) {
                        int32_t x = PB(t);
                        T.add_flow(x, T.up(x) ? delta : -delta);
                    }
                } else if (lane == 0) {
                    degen++;
                }
                const int32_t leave = side == 1 ? PA(tl) : PB(tl);
                const int32_t S = T.sz[leave];
                const int32_t q = side == 1 ? i : j, r = side == 1 ? j : i;
                __syncwarp();
                // the cut subtree leaves the chain above `leave` and joins r's chain
                if (side == 1) {
                    for (int32_t t = tl + 1 + lane; t < la; t += 32) T.sz[PA(t)] = (IX)((int32_t)T.sz[PA(t)] - S);
                    for (int32_t t = lane; t < lb; t += 32) T.sz[PB(t)] = (IX)((int32_t)T.sz[PB(t)] + S);
                } else {
                    for (int32_t t = tl + 1 + lane; t < lb; t += 32) T.sz[PB(t)] = (IX)((int32_t)T.sz[PB(t)] - S);
                    for (int32_t t = lane; t < la; t += 32) T.sz[PA(t)] = (IX)((int32_t)T.sz[PA(t)] + S);
                }
                __syncwarp();
                const int32_t k = tl;  // path q = v0 .. vk = leave
#define PV(t) (side == 1 ? PA(t) : PB(t))
                if (lane == 0) {
                    // potentials of the cut subtree shift so that the entering
                    // arc gets reduced cost 0
                    s_dpi = side == 1 ? rc : -rc;
                    s_L0 = T.ps[leave];
                    s_pr = T.ps[r];
                    s_S = S;
                    s_nseg = 2 * k + 1;
                    s_segsm = k < 32 ? 1 : 0;
                }
                if (k < 32) {
                    // one lane per path node: segments of the re-rooted order,
                    // new subtree sizes, and the reversed parent/pred/flow chain
                    const bool on = lane <= k;
                    int32_t vt = on ? PV(lane) : 0;
                    int32_t vp = (on && lane > 0) ? PV(lane - 1) : 0;
                    int32_t a_st = 0, a_len = 0, b_st = 0, b_len = 0, L = 0;
                    int32_t opred = 0, oflow = 0, oup = 0;
                    if (on) {
                        if (lane == 0) {
                            a_st = T.ps[q];
                            a_len = T.sz[q];
                            L = a_len;
                        } else {
                            int32_t pvt = T.ps[vt], pvp = T.ps[vp];
                            a_st = pvt;
                            a_len = pvp - pvt;
                            b_st = pvp + (int32_t)T.sz[vp];
                            b_len = pvt + (int32_t)T.sz[vt] - b_st;
                            L = a_len + b_len;
                        }
                        opred = T.pred[vt];
                        oflow = T.flow(vt);
                        oup = T.up(vt) ? 1 : 0;
                    }
                    int32_t incl = L;
                    for (int off = 1; off < 32; off <<= 1) {
                        int32_t o = __shfl_up_sync(FULL, incl, off);
                        if (lane >= off) incl += o;
                    }
                    const int32_t excl = incl - L;  // output offset of A_t
                    const int32_t ppred = __shfl_up_sync(FULL, opred, 1);
                    const int32_t pflow = __shfl_up_sync(FULL, oflow, 1);
                    const int32_t pup = __shfl_up_sync(FULL, oup, 1);
                    __syncwarp();
                    if (on) {
                        if (lane == 0) {
                            sseg[0][0] = a_st;
                            sseg[1][0] = a_len;
                            sseg[2][0] = 0;
                            T.pred[vt] = (int32_t)ent;
                            T.set_fu(vt, delta, i == q);  // the entering arc runs i -> j
                            T.set_parent(vt, r);
                            T.sz[vt] = (IX)S;
                        } else {
                            sseg[0][2 * lane - 1] = a_st;
                            sseg[1][2 * lane - 1] = a_len;
                            sseg[2][2 * lane - 1] = excl;
                            sseg[0][2 * lane] = b_st;
                            sseg[1][2 * lane] = b_len;
                            sseg[2][2 * lane] = excl + a_len;
                            T.pred[vt] = ppred;
                            T.set_fu(vt, pflow, !pup);
                            T.set_parent(vt, vp);
                            T.sz[vt] = (IX)(S - excl);
                        }
                    }
                } else if (lane == 0) {
                    // long path: the same steps on one lane, segments in global memory
                    int32_t* gs = I.seg;
                    int32_t ns = 0, out = 0;
                    gs[ns] = T.ps[q];
                    gs[SEGN + ns] = T.sz[q];
                    gs[2 * SEGN + ns] = out;
                    out += T.sz[q];
                    ns++;
                    for (int32_t t = 1; t <= k; t++) {
                        int32_t vt = PV(t), vp = PV(t - 1);
                        int32_t a_len = (int32_t)T.ps[vp] - (int32_t)T.ps[vt];
                        int32_t b_st = (int32_t)T.ps[vp] + (int32_t)T.sz[vp];
                        int32_t b_len = (int32_t)T.ps[vt] + (int32_t)T.sz[vt] - b_st;
                        gs[ns] = T.ps[vt];
                        gs[SEGN + ns] = a_len;
                        gs[2 * SEGN + ns] = out;
                        I.tmp[t] = out;  // offset of A_t; new size of v_t is S minus it
                        out += a_len;
                        ns++;
                        gs[ns] = b_st;
                        gs[SEGN + ns] = b_len;
                        gs[2 * SEGN + ns] = out;
                        out += b_len;
                        ns++;
                    }
                    int32_t prev_pred = (int32_t)ent;
                    bool prev_up = (i == q);
                    int32_t prev_flow = delta;
                    int32_t prev_par = r;
                    for (int32_t t = 0; t <= k; t++) {
                        int32_t vt = PV(t);
                        int32_t op = T.pred[vt];
                        bool ou = T.up(vt);
                        int32_t of = T.flow(vt);
                        T.pred[vt] = prev_pred;
                        T.set_fu(vt, prev_flow, prev_up);
                        T.set_parent(vt, prev_par);
                        prev_pred = op;
                        prev_up = !ou;
                        prev_flow = of;
                        prev_par = vt;
                    }
                    T.sz[q] = (IX)S;
                    for (int32_t t = 1; t <= k; t++) T.sz[PV(t)] = (IX)(S - I.tmp[t]);
                }
#undef PV
                if (lane == 0) {
                    // wall-clock limit, checked every 128 pivots: stop after this pivot
                    const bool late = (pivots & 127) == 0 && ns_now() - t0 > I.time_limit_ns;
                    s_go = late ? 0 : 1;
                    if (late) s_status = 2;
                }
            }
#undef PA
#undef PB
        }
        __syncthreads();
        if (!s_go) break;
        // ---- parallel re-hang: move the cut segment after r, re-rooted ------
        {
            const int32_t L0 = s_L0, S = s_S, pr = s_pr, nseg = s_nseg;
            const int64_t dpi = s_dpi;
            const int32_t* sst = s_segsm ? sseg[0] : I.seg;
            const int32_t* sot = s_segsm ? sseg[2] : I.seg + 2 * SEGN;
            int32_t lo, hi, ins;  // ins: first index of the new segment in the new order
            if (pr < L0) {
                lo = pr + 1;
                hi = L0 + S;
                ins = pr + 1;
            } else {
                lo = L0;
                hi = pr + 1;
                ins = pr + 1 - S;
            }
            auto new_node = [&](int32_t x) -> int32_t {
                if (x >= ins && x < ins + S) {
                    int32_t o = x - ins;
                    int32_t sl = 0, sh = nseg - 1;  // last segment with output offset <= o
                    while (sl < sh) {
                        int32_t mid = (sl + sh + 1) >> 1;
                        if (sot[mid] <= o)
                            sl = mid;
                        else
                            sh = mid - 1;
                    }
                    int32_t node = T.od[sst[sl] + (o - sot[sl])];
                    T.pi[node] += dpi;
                    return node;
                }
                return pr < L0 ? (int32_t)T.od[x - S] : (int32_t)T.od[x + S];
            };
            // new order of [lo, hi) computed from the old one, then written; the
            // next pricing reads only potentials (final before the barrier), and
            // every later reader of the order passes a pricing barrier first
            if (sizeof(IX) == 2 && hi - lo <= NS_REGS * NS_THREADS) {
                int32_t vals[NS_REGS];
#pragma unroll
                for (int r2 = 0; r2 < NS_REGS; r2++) {
                    int32_t x = lo + tid + r2 * NS_THREADS;
                    vals[r2] = x < hi ? new_node(x) : 0;
                }
                __syncthreads();
#pragma unroll
                for (int r2 = 0; r2 < NS_REGS; r2++) {
                    int32_t x = lo + tid + r2 * NS_THREADS;
                    if (x < hi) {
                        T.od[x] = (IX)vals[r2];
                        T.ps[vals[r2]] = (IX)x;
                    }
                }
            } else {  // a longer move: the new order goes through global memory
                for (int32_t x = lo + tid; x < hi; x += NS_THREADS) I.tmp[x] = new_node(x);
                __syncthreads();
                for (int32_t x = lo + tid; x < hi; x += NS_THREADS) {
                    int32_t node = I.tmp[x];
                    T.od[x] = (IX)node;
                    T.ps[node] = (IX)x;
                }
            }
        }
    }
    // ---- result: node arrays back to the global record ---------------------
    __syncthreads();
    for (int32_t v = tid; v < N1; v += NS_THREADS) {
        G.pi[v] = T.pi[v];
        G.pred[v] = T.pred[v];
        const uint32_t w = T.fu[v];  // read once: outside the compact layout it is G.flow's own word
        G.flow[v] = (int32_t)(w & 0x7fffffffu);
        G.up[v] = (w >> 31) ? 1 : 0;
        G.parent[v] = T.parent(v);
        G.size[v] = (int32_t)T.sz[v];
        G.pos[v] = (int32_t)T.ps[v];
    }
    __shared__ unsigned long long s_obj, s_art;
    if (tid == 0) {
        s_obj = 0;
        s_art = 0;
    }
    __syncthreads();
    unsigned long long obj = 0, art = 0;
    for (int32_t v = tid; v < n; v += NS_THREADS) {
        int64_t a = T.pred[v], f = T.flow(v);
        if (a >= I.m) {
            if (f != 0) art++;
        } else if (f > 0) {
            obj += (unsigned long long)(arc_cost(I, a, big) * f);
        }
    }
    atomicAdd(&s_obj, obj);
    atomicAdd(&s_art, art);
    __syncthreads();
    if (tid == 0) {
        G.pivots = pivots;
        G.degenerate = degen;
        G.scanned = nscan;
        G.status = s_status;
        G.opt = (int64_t)s_obj;
        if (s_status == 0 && s_art) G.status = 1;
    }
}

__device__ __forceinline__ void ns_instance(NSInst& G) {
    NSInst I = G;
    const int32_t N1 = I.n + 1;
    if (I.smem_nodes) {
        // 1: every node array in shared memory (24 B a node); 2: pred and the
        // packed flow in global memory (only the pivot's paths touch them), the
        // arrays every pivot scans in shared memory (16 B a node); 3: the
        // potentials in global memory too, the four 16-bit arrays (parent,
        // size, position, order) in shared memory (8 B a node)
        extern __shared__ __align__(16) unsigned char dyn[];
        unsigned char* p = dyn;
        Tree<uint16_t> T;
        if (I.smem_nodes == 3) {
            T.pi = I.pi;
        } else {
            T.pi = (int64_t*)p;
            p += sizeof(int64_t) * N1;
        }
        if (I.smem_nodes == 1) {
            T.pred = (int32_t*)p;
            p += sizeof(int32_t) * N1;
            T.fu = (uint32_t*)p;
            p += sizeof(uint32_t) * N1;
        } else {
            T.pred = I.pred;
            T.fu = (uint32_t*)I.flow;  // packed while solving, unpacked on exit
        }
        T.par = (uint16_t*)p;
        p += sizeof(uint16_t) * N1;
        T.sz = (uint16_t*)p;
        p += sizeof(uint16_t) * N1;
        T.ps = (uint16_t*)p;
        p += sizeof(uint16_t) * N1;
        T.od = (uint16_t*)p;
        ns_body<uint16_t>(G, I, T);
    } else {
        Tree<int32_t> T;
        T.pi = I.pi;
        T.pred = I.pred;
        T.fu = (uint32_t*)I.flow;  // packed flow / direction while solving; unpacked on exit
        T.par = I.parent;
        T.sz = I.size;
        T.ps = I.pos;
        T.od = I.ord;
        ns_body<int32_t>(G, I, T);
    }
}

// Persistent: every CTA takes the next instance of `order` (largest first, so
// the batch finishes close to its total work / CTAs) until none is left.
__global__ void __launch_bounds__(NS_THREADS) k_netsimplex(NSInst* insts, const int32_t* __restrict__ order,
                                                           int32_t count, int32_t* __restrict__ next) {
    __shared__ int32_t s_k;
    for (;;) {
        if (threadIdx.x == 0) s_k = atomicAdd(next, 1);
        __syncthreads();
        const int32_t k = s_k;
        __syncthreads();
        if (k >= count) break;
        ns_instance(insts[order[k]]);
        __syncthreads();
    }
}

// Bytes of dynamic shared memory for the node arrays of N1 nodes in layout
// 1 (all of them), 2 (all but pred and the packed flow) or 3 (the four
// 16-bit arrays).
size_t ns_smem_bytes(int64_t N1, int layout) {
    const size_t per = layout == 1 ? 8 + 4 + 4 + 2 + 2 + 2 + 2 : layout == 2 ? 8 + 2 + 2 + 2 + 2 : 2 + 2 + 2 + 2;
    return (size_t)N1 * per + 64;
}

// The shared-memory layout N1 nodes can use: 1, else 2, else 3, else 0 (global).
// All three keep 16-bit node indices.
int ns_smem_layout(int64_t N1, int max_optin) {
    if (N1 >= 65535) return 0;  // 16-bit indices, 65535 marks "no parent"
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_netsimplex) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int layout = 1; layout <= 3; layout++)
        if (fa.sharedSizeBytes + ns_smem_bytes(N1, layout) <= (size_t)max_optin) return layout;
    return 0;
}

// The dynamic shared memory limit of a kernel is one attribute per device for
// the whole process.  Several host threads launch k_netsimplex at once (the
// batch workers, the allocation-free solve), so the limit is raised once per
// device to the largest size any instance can ask for and never lowered: a
// launch can then never see another thread's smaller value.
cudaError_t ns_kernel_setup() {
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (done[dev]) return cudaSuccess;
    int max_optin = 0;
    e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_netsimplex);
    if (e != cudaSuccess) return e;
    const size_t most = (size_t)max_optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(k_netsimplex, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    if (e != cudaSuccess) return e;
    done[dev] = true;
    return cudaSuccess;
}

__global__ void k_i64_to_i32_cost(const int64_t* __restrict__ c, int64_t m, int32_t* __restrict__ o,
                                  unsigned long long* __restrict__ bad) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    int64_t v = c[a];
    if (v < 0 || v >= (int64_t(1) << 31)) atomicAdd(bad, 1ull);
    o[a] = (int32_t)v;
}

__global__ void k_abs_sum(const int64_t* __restrict__ s, int64_t n, unsigned long long* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) {
        int64_t x = s[i];
        v = (unsigned long long)(x < 0 ? -x : x);
        if (v >= (1ull << 40)) v = 1ull << 40;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// One network simplex instance on an arc list, ready to launch (buffers of
// this context; nothing is launched).  cmax = largest arc cost.
pd_status ns_prepare_arcs(Ctx* c, int32_t n, int64_t m, int64_t mst, int64_t nS, int64_t nT, const int32_t* cmat,
                          const int32_t* tail, const int32_t* head, const int32_t* cost, const int64_t* supply,
                          int64_t cmax, const pd_opts& o, NSPrep* p, cudaStream_t st) {
    *p = NSPrep{};
    if (n <= 0) return PD_OK;
    int64_t N1 = (int64_t)n + 1;
    NSInst& h = p->h;
    h.n = n;
    h.m = m;
    h.mst = mst;
    h.nS = nS;
    h.nT = nT > 0 ? nT : 1;
    h.cmat = cmat;
    h.tail = tail;
    h.head = head;
    h.cost = cost;
    h.supply = supply;
    h.pi = bufT<int64_t>(c, B_NS_PI, N1);
    h.parent = bufT<int32_t>(c, B_NS_PARENT, N1);
    h.pred = bufT<int32_t>(c, B_NS_PRED, N1);
    h.flow = bufT<int32_t>(c, B_NS_FLOW, N1);
    h.up = bufT<uint8_t>(c, B_NS_UP, N1);
    h.ord = bufT<int32_t>(c, B_NS_ORD, N1);
    h.pos = bufT<int32_t>(c, B_NS_POS, N1);
    h.size = bufT<int32_t>(c, B_NS_SIZE, N1);
    h.tmp = bufT<int32_t>(c, B_NS_TMP, N1);
    h.path = bufT<int32_t>(c, B_NS_PATH, 2 * N1);
    h.seg = bufT<int32_t>(c, B_NS_SEG, 3 * (2 * N1 + 3));
    if (!h.pi || !h.parent || !h.pred || !h.flow || !h.up || !h.ord || !h.pos || !h.size || !h.tmp || !h.path ||
        !h.seg)
        return PD_ENOMEM;
    int64_t M = m + n;
    // arc ids, plus one pricing step past the last arc, stay below 2^31
    if (M >= (int64_t(1) << 31) - 1 - 8 * NS_THREADS)
        return fail(c, PD_ECAPACITY, "network simplex needs fewer than 2^31 - 8193 arcs");
    // default block: one pass of the CTA (8 arcs per thread), more for very
    // large networks; blocks start at multiples of 8 (vector loads)
    int64_t blk = o.ns_block > 0 ? o.ns_block : tuned_block(c, M);
    if (blk <= 0) blk = std::max<int64_t>(8 * NS_THREADS, (int64_t)sqrt((double)M));
    blk = (blk + 7) & ~(int64_t)7;
    h.block = blk;
    h.walk = o.ns_walk >= 0 ? std::min<int32_t>(o.ns_walk, NS_LMAX) : tuned_walk(c, M);
    h.max_pivots = o.max_rounds > 0 ? o.max_rounds : (int64_t(1) << 40);
    h.time_limit_ns = (o.time_limit_ms > 0 ? (uint64_t)o.time_limit_ms : 60000ull) * 1000000ull;
    // flows are int32: the total supply must stay below 2^31
    {
        unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
        if (!sm) return PD_ENOMEM;
        PD_TRY_CUDA(c, cudaMemsetAsync(sm + 16, 0, sizeof(unsigned long long), st));
        k_abs_sum<<<grid_for(n, 256), 256, 0, st>>>(supply, n, sm + 16); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small + 16, sm + 16, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        if ((unsigned long long)c->h_small[16] >= (1ull << 31)) return fail(c, PD_ECAPACITY, "total supply >= 2^31");
    }
    // big-M: more than any path cost; |potentials| stay below ~3 big
    if (cmax > (INT64_MAX / 8) / N1) return fail(c, PD_EOVERFLOW, "network simplex big-M would overflow");
    h.big = N1 * (cmax + 1) + 1;
    int max_optin = 0;
    PD_TRY_CUDA(c, cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    h.smem_nodes = o.ns_smem != 0 ? ns_smem_layout(N1, max_optin) : 0;
    p->smem = h.smem_nodes ? ns_smem_bytes(N1, h.smem_nodes) : 0;
    p->ready = true;
    return PD_OK;
}

pd_status ns_run(Ctx* c, const NSInst* h, int count, size_t smem, NSInst* d, NSInst* r, cudaStream_t st) {
    if (count <= 0) return PD_OK;
    PD_TRY_CUDA(c, ns_kernel_setup());
    int per_sm = 0;
    PD_TRY_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_netsimplex, NS_THREADS, smem));
    if (per_sm < 1) return fail(c, PD_ECAPACITY, "network simplex kernel does not fit on an SM");
    const int grid = std::min(count, per_sm * std::max(c->sm_count, 1));
    // largest instances first (nodes, then arcs), ties by position
    std::vector<int32_t> order((size_t)count);
    for (int q = 0; q < count; q++) order[(size_t)q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return h[x].n != h[y].n ? h[x].n > h[y].n : h[x].m > h[y].m;
    });
    int32_t* dord = bufT<int32_t>(c, B_NS_ORDER, count + 1);
    if (!dord) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemcpyAsync(d, h, sizeof(NSInst) * count, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(dord, order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(dord + count, 0, sizeof(int32_t), st));
    cudaEvent_t e0, e1;
    PD_TRY_CUDA(c, cudaEventCreate(&e0));
    PD_TRY_CUDA(c, cudaEventCreate(&e1));
    PD_TRY_CUDA(c, cudaEventRecord(e0, st));
    k_netsimplex<<<grid, NS_THREADS, smem, st>>>(d, dord, count, dord + count); pd::count_launch();
    cudaError_t le = cudaGetLastError();
    if (le == cudaSuccess) le = cudaEventRecord(e1, st);
    if (le == cudaSuccess) le = cudaMemcpyAsync(r, d, sizeof(NSInst) * count, cudaMemcpyDeviceToHost, st);
    if (le == cudaSuccess) le = cudaStreamSynchronize(st);
    float nms = 0.f;
    if (le == cudaSuccess) le = cudaEventElapsedTime(&nms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (le != cudaSuccess) return cuda_fail(c, le, "k_netsimplex");
    c->last_ns_ms += nms;
    return PD_OK;
}

// Pinned staging of a wave: records in, records out, order (+ counter),
// certificate jobs, certificate counts.
struct WaveLayout {
    size_t in, out, ord, jobs, cert, total;
    explicit WaveLayout(int count) {
        auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
        in = 0;
        out = in + al(sizeof(NSInst) * count);
        ord = out + al(sizeof(NSInst) * count);
        jobs = ord + al(sizeof(int32_t) * (count + 1));
        cert = jobs + al(sizeof(CertJob) * count);
        total = cert + al(2 * sizeof(unsigned long long) * count);
    }
};

constexpr int WAVE_CERT_BLOCKS = 8;  // blocks per pair of the batched certificate (grid-stride)

pd_status ns_run_wave(Ctx* c, const NSInst* h, int count, size_t smem, const CertJob* jobs, NSInst* r,
                      unsigned long long* cert, cudaStream_t st) {
    if (count <= 0) return PD_OK;
    PD_TRY_CUDA(c, ns_kernel_setup());
    int per_sm = 0;
    PD_TRY_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_netsimplex, NS_THREADS, smem));
    if (per_sm < 1) return fail(c, PD_ECAPACITY, "network simplex kernel does not fit on an SM");
    const int grid = std::min(count, per_sm * std::max(c->sm_count, 1));
    const WaveLayout L(count);
    if (c->wave_pin_bytes < L.total) {
        if (c->wave_exec) cudaGraphExecDestroy(c->wave_exec);
        c->wave_exec = nullptr;
        if (c->wave_pin) cudaFreeHost(c->wave_pin);
        c->wave_pin = nullptr;
        c->wave_pin_bytes = 0;
        PD_TRY_CUDA(c, cudaMallocHost(&c->wave_pin, L.total));
        c->wave_pin_bytes = L.total;
    }
    if (!c->wave_stream) PD_TRY_CUDA(c, cudaStreamCreateWithFlags(&c->wave_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : c->wave_ev)
        if (!e) PD_TRY_CUDA(c, cudaEventCreate(&e));
    unsigned char* pin = (unsigned char*)c->wave_pin;
    NSInst* p_in = (NSInst*)(pin + L.in);
    NSInst* p_out = (NSInst*)(pin + L.out);
    int32_t* p_ord = (int32_t*)(pin + L.ord);
    CertJob* p_jobs = (CertJob*)(pin + L.jobs);
    unsigned long long* p_cert = (unsigned long long*)(pin + L.cert);
    NSInst* d = bufT<NSInst>(c, B_NS_INST, count);
    int32_t* dord = bufT<int32_t>(c, B_NS_ORDER, count + 1);
    CertJob* djobs = bufT<CertJob>(c, B_NS_JOBS, count);
    unsigned long long* dcert = bufT<unsigned long long>(c, B_NS_CERT, 2 * count);
    if (!d || !dord || !djobs || !dcert) return PD_ENOMEM;
    // this wave's contents into the pinned staging the graph copies from;
    // largest instances first (nodes, then arcs), ties by position
    memcpy(p_in, h, sizeof(NSInst) * count);
    for (int q = 0; q < count; q++) p_ord[q] = q;
    std::stable_sort(p_ord, p_ord + count, [&](int32_t x, int32_t y) {
        return h[x].n != h[y].n ? h[x].n > h[y].n : h[x].m > h[y].m;
    });
    p_ord[count] = 0;
    for (int q = 0; q < count; q++) {
        if (jobs[q].rec < 0 || jobs[q].rec >= count) return fail(c, PD_EINVAL, "certificate job without a record");
        p_jobs[q] = jobs[q];
        p_jobs[q].inst = d + jobs[q].rec;
    }
    // the executable is reused while everything it was captured with is the same
    uint64_t key = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
    mix((uint64_t)count);
    mix((uint64_t)grid);
    mix((uint64_t)smem);
    mix((uint64_t)(uintptr_t)pin);
    mix((uint64_t)(uintptr_t)d);
    mix((uint64_t)(uintptr_t)dord);
    mix((uint64_t)(uintptr_t)djobs);
    mix((uint64_t)(uintptr_t)dcert);
    cudaStream_t gs = c->wave_stream;
    if (!c->wave_exec || c->wave_key != key) {
        if (c->wave_exec) cudaGraphExecDestroy(c->wave_exec);
        c->wave_exec = nullptr;
        PD_TRY_CUDA(c, cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(d, p_in, sizeof(NSInst) * count, cudaMemcpyHostToDevice, gs);
        cudaMemcpyAsync(dord, p_ord, sizeof(int32_t) * (count + 1), cudaMemcpyHostToDevice, gs);
        cudaMemcpyAsync(djobs, p_jobs, sizeof(CertJob) * count, cudaMemcpyHostToDevice, gs);
        cudaMemsetAsync(dcert, 0, 2 * sizeof(unsigned long long) * count, gs);
        k_netsimplex<<<grid, NS_THREADS, smem, gs>>>(d, dord, count, dord + count);
        k_certify_batch<<<dim3(WAVE_CERT_BLOCKS, count), 256, 0, gs>>>(djobs, dcert);
        cudaMemcpyAsync(p_out, d, sizeof(NSInst) * count, cudaMemcpyDeviceToHost, gs);
        cudaMemcpyAsync(p_cert, dcert, 2 * sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, gs);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(gs, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->wave_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->wave_exec = nullptr;
            return cuda_fail(c, e, "capture of the batch wave");
        }
        c->wave_key = key;
    }
    PD_TRY_CUDA(c, cudaEventRecord(c->wave_ev[2], st));  // the wave follows the work queued on st
    PD_TRY_CUDA(c, cudaStreamWaitEvent(gs, c->wave_ev[2], 0));
    // device time of the whole graph (the simplex is nearly all of it: the
    // other nodes move a few hundred bytes per pair)
    PD_TRY_CUDA(c, cudaEventRecord(c->wave_ev[0], gs));
    PD_TRY_CUDA(c, cudaGraphLaunch(c->wave_exec, gs));
    PD_TRY_CUDA(c, cudaEventRecord(c->wave_ev[1], gs));
    pd::count_launch();  // the persistent simplex
    pd::count_launch();  // the batched certificate
    c->wave_launches++;
    PD_TRY_CUDA(c, cudaStreamSynchronize(gs));
    float nms = 0.f;
    PD_TRY_CUDA(c, cudaEventElapsedTime(&nms, c->wave_ev[0], c->wave_ev[1]));
    c->last_ns_ms += nms;
    memcpy(r, p_out, sizeof(NSInst) * count);
    memcpy(cert, p_cert, 2 * sizeof(unsigned long long) * count);
    return PD_OK;
}

pd_status ns_status(Ctx* c, const NSInst& r) {
    if (r.status == 2) return fail(c, PD_ETIMEOUT, "network simplex pivot cap or time limit reached");
    if (r.status == 1) return fail(c, PD_EINFEASIBLE, "network has no feasible flow");
    if (r.status == 3) return fail(c, PD_EINFEASIBLE, "network simplex found an unbounded cycle");
    if (r.status != 0) return fail(c, PD_ECUDA, "network simplex failed");
    return PD_OK;
}

// Network simplex on an arc list (one CTA), result in this context's
// instance record.
static pd_status ns_solve_arcs(Ctx* c, int32_t n, int64_t m, int64_t mst, int64_t nS, int64_t nT,
                               const int32_t* cmat, const int32_t* tail, const int32_t* head, const int32_t* cost,
                               const int64_t* supply, int64_t cmax, const pd_opts& o, NSInst* out,
                               cudaStream_t st) {
    *out = NSInst{};
    NSPrep p;
    PD_TRY(ns_prepare_arcs(c, n, m, mst, nS, nT, cmat, tail, head, cost, supply, cmax, o, &p, st));
    if (!p.ready) return PD_OK;
    NSInst* d = bufT<NSInst>(c, B_NS_INST, 1);
    if (!d) return PD_ENOMEM;
    PD_TRY(ns_run(c, &p.h, 1, p.smem, d, out, st));
    return ns_status(c, *out);
}

// ---------------------------------------------------------------------------
// transportation form of the condensed problem, and its certificate on WS
// ---------------------------------------------------------------------------

__global__ void k_side_flags(const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB, int64_t N,
                             int64_t* __restrict__ fs, int64_t* __restrict__ ft) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= N) return;
    int64_t s = cntA[u] - cntB[u];
    fs[u] = s > 0;
    ft[u] = s < 0;
}

__global__ void k_side_lists(const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB, int64_t N,
                             const int64_t* __restrict__ os, const int64_t* __restrict__ ot, int32_t* __restrict__ S,
                             int32_t* __restrict__ T, int64_t* __restrict__ sup, int64_t nS) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= N) return;
    int64_t s = cntA[u] - cntB[u];
    if (s > 0) {
        S[os[u]] = (int32_t)u;
        sup[os[u]] = s;
    } else if (s < 0) {
        T[ot[u]] = (int32_t)u;
        sup[nS + ot[u]] = s;
    }
}

// Arc i*nT + j: source i -> sink j at min(l2, diag(i) + diag(j)) (the route
// through the diagonal node has unbounded capacity); then the arcs of the
// diagonal node if its supply |B| - |A| is not 0.
__global__ void k_transport_arcs(const int32_t* __restrict__ S, const int32_t* __restrict__ T, int64_t nS,
                                 int64_t nT, int dside, const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                                 int32_t* __restrict__ cmat, int32_t* __restrict__ tail, int32_t* __restrict__ head,
                                 int32_t* __restrict__ cost, unsigned long long* __restrict__ bad, DiagCost dc) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t mst = nS * nT;
    int64_t D = nS + nT;
    int64_t c;
    if (a < mst) {
        int64_t i = a / nT, j = a - i * nT;
        int32_t u = S[i], v = T[j];
        int64_t d = cost_l2(X[u], Y[u], X[v], Y[v]);
        int64_t g = cost_make(X[u], Y[u], dc) + cost_make(X[v], Y[v], dc);
        c = d < g ? d : g;
        if (c >= (int64_t(1) << 31)) atomicAdd(bad, 1ull);
        cmat[a] = (int32_t)c;
        return;
    } else if (dside < 0 && a < mst + nS) {
        int64_t i = a - mst;
        int32_t u = S[i];
        c = cost_make(X[u], Y[u], dc);
        tail[a - mst] = (int32_t)i;
        head[a - mst] = (int32_t)D;
    } else if (dside > 0 && a < mst + nT) {
        int64_t j = a - mst;
        int32_t v = T[j];
        c = cost_make(X[v], Y[v], dc);
        tail[a - mst] = (int32_t)D;
        head[a - mst] = (int32_t)(nS + j);
    } else {
        return;
    }
    if (c >= (int64_t(1) << 31)) atomicAdd(bad, 1ull);
    cost[a - mst] = (int32_t)c;
}

// Total flow over the arcs of a solved arc-list network (rounding slack).
__global__ void k_tree_flow(const NSInst* __restrict__ I, unsigned long long* __restrict__ out) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= I->n) return;
    if (I->pred[v] < I->m && I->flow[v] > 0) atomicAdd(out, (unsigned long long)I->flow[v]);
}

pd_status ns_solve_network(Ctx* c, const pd_network& net, const pd_opts& o, SolveStats* out, cudaStream_t st) {
    int64_t n = net.n_nodes, m = net.n_arcs;
    if (n >= (int64_t(1) << 31) - 2) return fail(c, PD_ECAPACITY, "too many nodes");
    int32_t* tail = bufT<int32_t>(c, B_S_TAIL, m);
    int32_t* c32 = bufT<int32_t>(c, B_NS_COST, m);
    unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
    if (!tail || !c32 || !sm) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, 8 * sizeof(unsigned long long), st));
    if (m > 0) {
        k_arc_tails<<<grid_for(m, 256), 256, 0, st>>>(net.row_ptr, n, m, tail); pd::count_launch();
        k_i64_to_i32_cost<<<grid_for(m, 256), 256, 0, st>>>(net.cost, m, c32, sm); pd::count_launch();
        k_max_cost<<<grid_for(m, 256), 256, 0, st>>>(net.cost, m, sm + 1); pd::count_launch();
    }
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (c->h_small[0]) return fail(c, PD_EOVERFLOW, "arc cost outside [0, 2^31)");
    int64_t cmax = c->h_small[1];
    NSInst r;
    PD_TRY(ns_solve_arcs(c, (int32_t)n, m, 0, 0, 1, nullptr, tail, net.head, c32, net.supply, cmax, o, &r, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, sizeof(unsigned long long), st));
    k_tree_flow<<<grid_for(n, 256), 256, 0, st>>>(bufT<NSInst>(c, B_NS_INST, 1), sm); pd::count_launch();
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    out->opt = r.opt;
    out->slack = c->h_small[0];
    out->pivots = r.pivots;
    out->degenerate = r.degenerate;
    out->scanned = r.scanned;
    out->verified = 1;  // the pricing loop ends only when no arc has a negative reduced cost
    out->method = 1;
    return PD_OK;
}

// The W1 network: the transportation form is tried first when it is not
// much larger than the sparse network (prepared here, launched by the caller,
// checked by ns_finish_w1); otherwise, or if its certificate fails, the
// simplex runs on the sparse network itself.  n_arcs = arcs of the sparse
// network, dsup = |B| - |A| (supply of the merged diagonal node).
pd_status ns_prepare_w1(Ctx* c, const pd_nodes& nodes, int64_t n_arcs, int64_t dsup, const pd_opts& o, W1Prep* w,
                        cudaStream_t st) {
    *w = W1Prep{};
    int64_t N = nodes.n_nodes;
    if (N == 0 || o.ns_transport == 0) return PD_OK;
    int64_t* fs = bufT<int64_t>(c, B_WSFLAG, N);
    int64_t* ft = bufT<int64_t>(c, B_WSOFF, N);
    unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
    if (!fs || !ft || !sm) return PD_ENOMEM;
    k_side_flags<<<grid_for(N, 256), 256, 0, st>>>(nodes.cntA, nodes.cntB, N, fs, ft); pd::count_launch();
    PD_TRY(scan_i64(c, fs, fs, N, (int64_t*)sm + 2, st));
    PD_TRY(scan_i64(c, ft, ft, N, (int64_t*)sm + 3, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    int64_t nS = c->h_small[2], nT = c->h_small[3];
    int64_t mst = nS * nT;
    int64_t mt = mst + (dsup < 0 ? nS : (dsup > 0 ? nT : 0));
    // the transportation form when it is not much larger than the sparse
    // network (ns_transport 1), or whenever its arc ids fit (2)
    if (!((o.ns_transport == 2 || mt <= 2 * n_arcs + 4096) && mt < (int64_t(1) << 31) - 1 - 8 * NS_THREADS))
        return PD_OK;
    int64_t nt = nS + nT + 1;
    int32_t* S = bufT<int32_t>(c, B_TR_S, nS);
    int32_t* T = bufT<int32_t>(c, B_TR_T, nT);
    int64_t* sup = bufT<int64_t>(c, B_TR_SUP, nt);
    int64_t mx = mt - mst;
    int32_t* cmat = bufT<int32_t>(c, B_NS_COST, mst);
    int32_t* tail = bufT<int32_t>(c, B_S_TAIL, mx);
    int32_t* head = bufT<int32_t>(c, B_S_HEAD, mx);
    int32_t* cost = bufT<int32_t>(c, B_TR_XCOST, mx);
    if (!S || !T || !sup || !tail || !head || !cost || !cmat) return PD_ENOMEM;
    k_side_lists<<<grid_for(N, 256), 256, 0, st>>>(nodes.cntA, nodes.cntB, N, fs, ft, S, T, sup, nS); pd::count_launch();
    c->h_small[20] = dsup;
    PD_TRY_CUDA(c, cudaMemcpyAsync(sup + nS + nT, c->h_small + 20, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, 8 * sizeof(unsigned long long), st));
    if (mt > 0)
        k_transport_arcs<<<grid_for(mt, 256), 256, 0, st>>>(S, T, nS, nT, dsup < 0 ? -1 : (dsup > 0 ? 1 : 0),
                                                              nodes.X, nodes.Y, cmat, tail, head, cost, sm, diag_cost(o)); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    if (mst > 0) k_max_cost32<<<grid_for(mst, 256), 256, 0, st>>>(cmat, mst, sm + 1); pd::count_launch();
    if (mx > 0) k_max_cost32<<<grid_for(mx, 256), 256, 0, st>>>(cost, mx, sm + 1); pd::count_launch();
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (c->h_small[0] != 0) return PD_OK;  // a cost does not fit in int32: solve the sparse network
    PD_TRY(ns_prepare_arcs(c, (int32_t)nt, mt, mst, nS, nT, cmat, tail, head, cost, sup, c->h_small[1], o, &w->ns,
                           st));
    w->S = S;
    w->T = T;
    w->nS = nS;
    w->nT = nT;
    w->nt = nt;
    w->dc = diag_cost(o);
    return PD_OK;
}

pd_status ns_finish_w1(Ctx* c, const WsTree& tr, int64_t s, const pd_network* merged, const pd_opts& o,
                       const W1Prep& w, const NSInst* d_res, const NSInst& r, SolveStats* out, cudaStream_t st) {
    *out = SolveStats{};
    if (w.ns.ready) {
        PD_TRY(ns_status(c, r));
        unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
        if (!sm) return PD_ENOMEM;
        PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, 4 * sizeof(unsigned long long), st));
        k_certify_tree<<<grid_for(w.nt, 256), 256, 0, st>>>(d_res, w.S, w.T, w.nS, w.nT, tr, s, w.dc, sm); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        out->pivots = r.pivots;
        out->degenerate = r.degenerate;
        out->scanned = r.scanned;
        if (c->h_small[0] == 0) {
            out->opt = r.opt;
            out->slack = c->h_small[1];
            out->verified = 1;
            out->method = 2;
            return PD_OK;
        }
        out->cert_failures = c->h_small[0];
    }
    if (!merged) {  // the caller solves the sparse network
        out->method = -1;
        return PD_OK;
    }
    int64_t piv = out->pivots, fails = out->cert_failures, scn = out->scanned, deg = out->degenerate;
    PD_TRY(ns_solve_network(c, *merged, o, out, st));
    out->pivots += piv;
    out->scanned += scn;
    out->degenerate += deg;
    out->cert_failures = fails;
    return PD_OK;
}

}  // namespace pd
