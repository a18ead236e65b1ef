// Hierarchical tree (binary radix tree over Morton order), s-WSPD biarcs
// (Algorithms 6-8 as a level-synchronous pair frontier), diagonal arcs
// (Algorithm 9) and the CSR network.
#include "internal.h"
#include "netsimplex.cuh"
#include "prims.cuh"

namespace pd {

// ---------------------------------------------------------------------------
// radix tree (Karras 2012) and bottom-up bounding boxes
// ---------------------------------------------------------------------------

PD_D int code_delta(const uint64_t* __restrict__ code, int64_t N, int64_t i, int64_t j) {
    if (j < 0 || j >= N) return -1;
    return __clzll((long long)(code[i] ^ code[j]));
}

// Internal node i covers [lo, hi] with i at one end; its split is the last
// index below the highest bit where the range's codes differ.  Children:
// c >= 0 internal c, c < 0 leaf ~c.
__global__ void k_karras(const uint64_t* __restrict__ code, int64_t N, int32_t* __restrict__ left,
                         int32_t* __restrict__ right, int32_t* __restrict__ par_int, int32_t* __restrict__ par_leaf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N - 1) return;
    int d = (code_delta(code, N, i, i + 1) - code_delta(code, N, i, i - 1)) > 0 ? 1 : -1;
    int dmin = code_delta(code, N, i, i - d);
    int64_t lmax = 2;
    while (code_delta(code, N, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (code_delta(code, N, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = code_delta(code, N, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (code_delta(code, N, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    if (lo == gamma) {
        left[i] = ~(int32_t)gamma;
        par_leaf[gamma] = (int32_t)i;
    } else {
        left[i] = (int32_t)gamma;
        par_int[gamma] = (int32_t)i;
    }
    if (hi == gamma + 1) {
        right[i] = ~(int32_t)(gamma + 1);
        par_leaf[gamma + 1] = (int32_t)i;
    } else {
        right[i] = (int32_t)(gamma + 1);
        par_int[gamma + 1] = (int32_t)i;
    }
    if (i == 0) par_int[0] = -1;
}

// Each leaf climbs; the second child to arrive at a node computes the node's
// tight box and leftmost member (min X, then min Y) from its two children.
__global__ void k_bbox(int64_t N, const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                       const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                       const int32_t* __restrict__ par_int, const int32_t* __restrict__ par_leaf, int4* bb,
                       int32_t* rep, int32_t* visit) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= N) return;
    int32_t cur = par_leaf[l];
    for (int depth = 0; cur >= 0 && depth < 130; depth++) {  // a radix tree over 64-bit codes is < 65 deep
        __threadfence();
        if (atomicAdd(&visit[cur], 1) == 0) return;
        int4 b[2];
        int32_t r[2];
        int32_t ch[2] = {left[cur], right[cur]};
        for (int q = 0; q < 2; q++) {
            int32_t c = ch[q];
            if (c < 0) {
                int32_t p = ~c;
                b[q] = make_int4(X[p], X[p], Y[p], Y[p]);
                r[q] = p;
            } else {
                b[q] = __ldcg(&bb[c]);
                r[q] = __ldcg(&rep[c]);
            }
        }
        int4 u = make_int4(min(b[0].x, b[1].x), max(b[0].y, b[1].y), min(b[0].z, b[1].z), max(b[0].w, b[1].w));
        int32_t rr = (X[r[1]] < X[r[0]] || (X[r[1]] == X[r[0]] && Y[r[1]] < Y[r[0]])) ? r[1] : r[0];
        __stcg(&bb[cur], u);
        __stcg(&rep[cur], rr);
        cur = par_int[cur];
    }
}

// ---------------------------------------------------------------------------
// s-WSPD as a pair frontier
// ---------------------------------------------------------------------------

struct TNode {
    int32_t mnx, mxx, mny, mxy, rep, l, r;
};

PD_D TNode load_tnode(int32_t ref, const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                      const int4* __restrict__ bb, const int32_t* __restrict__ rep, const int32_t* __restrict__ left,
                      const int32_t* __restrict__ right) {
    TNode t;
    if (ref < 0) {
        int32_t p = ~ref;
        t.mnx = t.mxx = X[p];
        t.mny = t.mxy = Y[p];
        t.rep = p;
        t.l = t.r = 0;
    } else {
        int4 b = bb[ref];
        t.mnx = b.x;
        t.mxx = b.y;
        t.mny = b.z;
        t.mxy = b.w;
        t.rep = rep[ref];
        t.l = left[ref];
        t.r = right[ref];
    }
    return t;
}

// s-well-separated with circumscribed circles of the tight boxes and the
// larger radius for both: in doubled coordinates |C_u - C_v| >= (s+2) D,
// D the larger box diagonal; exact in 128-bit integers.
PD_D bool well_separated(const TNode& a, const TNode& b, int64_t s) {
    int64_t dx = ((int64_t)a.mnx + a.mxx) - ((int64_t)b.mnx + b.mxx);
    int64_t dy = ((int64_t)a.mny + a.mxy) - ((int64_t)b.mny + b.mxy);
    uint64_t ax = (uint64_t)(dx < 0 ? -dx : dx), ay = (uint64_t)(dy < 0 ? -dy : dy);
    unsigned __int128 D2 = (unsigned __int128)ax * ax + (unsigned __int128)ay * ay;
    uint64_t awx = (uint64_t)((int64_t)a.mxx - a.mnx), awy = (uint64_t)((int64_t)a.mxy - a.mny);
    uint64_t bwx = (uint64_t)((int64_t)b.mxx - b.mnx), bwy = (uint64_t)((int64_t)b.mxy - b.mny);
    uint64_t ra = awx * awx + awy * awy, rb = bwx * bwx + bwy * bwy;
    uint64_t R2 = ra > rb ? ra : rb;
    uint64_t k = (uint64_t)(s + 2) * (uint64_t)(s + 2);
    return D2 >= (unsigned __int128)k * R2;
}

PD_D int64_t max_side(const TNode& a) {
    int64_t wx = (int64_t)a.mxx - a.mnx, wy = (int64_t)a.mxy - a.mny;
    return wx > wy ? wx : wy;
}

// Is (a, b), a < b two leaves (Morton ranks), one of the biarcs of the
// s-WSPD?  The pairs of the decomposition partition all leaf pairs, so (a, b)
// lies in exactly one of them: start at the pair of children of the lowest
// common ancestor and follow the same split rule as k_ws_expand (larger box
// side, ties split the second node), always into the child holding a
// (resp. b), until the pair is well separated.  (a, b) is an arc iff a and b
// are the representatives of that pair.  A walk longer than any tree path
// answers false, which the certificate treats as a failure (never as proof).
PD_D bool ws_arc_exists(int32_t a, int32_t b, int64_t N, const int32_t* __restrict__ X,
                        const int32_t* __restrict__ Y, const int4* __restrict__ bb, const int32_t* __restrict__ rep,
                        const int32_t* __restrict__ left, const int32_t* __restrict__ right, int64_t s) {
    if (N < 2 || a >= b || a < 0 || b >= N) return false;
    int32_t z = 0;  // the root covers [0, N - 1]
    int32_t sp = 0;
    int depth = 0;
    for (; depth < 130; depth++) {
        const int32_t lc = left[z], rc = right[z];
        sp = lc >= 0 ? lc : ~lc;  // left child covers [lo, sp], right child [sp + 1, hi]
        if (b <= sp) {
            if (lc < 0) return false;
            z = lc;
        } else if (a > sp) {
            if (rc < 0) return false;
            z = rc;
        } else {
            break;
        }
    }
    if (depth >= 130) return false;
    int32_t P = left[z], Q = right[z];
    for (int it = 0; it < 260; it++) {
        const TNode tp = load_tnode(P, X, Y, bb, rep, left, right);
        const TNode tq = load_tnode(Q, X, Y, bb, rep, left, right);
        if (well_separated(tp, tq, s)) return tp.rep == a && tq.rep == b;
        if (max_side(tp) > max_side(tq)) {
            if (P < 0) return false;
            const int32_t c = tp.l >= 0 ? tp.l : ~tp.l;
            P = a <= c ? tp.l : tp.r;
        } else {
            if (Q < 0) return false;
            const int32_t c = tq.l >= 0 ? tq.l : ~tq.l;
            Q = b <= c ? tq.l : tq.r;
        }
    }
    return false;
}

// Certificate of a transportation optimum against the sparse network: every
// source -> sink pair that carries flow on its direct route must be a WSPD
// biarc (found by ws_arc_exists); routes through the diagonal use arcs that
// always exist.  out[0] = pairs missing, out[1] = total flow over the arcs of
// the sparse network that the flow uses (rounding slack).
__global__ void k_certify_tree(const NSInst* __restrict__ I, const int32_t* __restrict__ S,
                               const int32_t* __restrict__ T, int64_t nS, int64_t nT, WsTree tr, int64_t s,
                               DiagCost dc, unsigned long long* __restrict__ out) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= I->n) return;
    int64_t a = I->pred[v], f = I->flow[v];
    if (a >= I->m || f <= 0) return;
    int64_t mst = nS * nT;
    if (a >= mst) {  // arc of the diagonal node: one arc of the sparse network
        atomicAdd(&out[1], (unsigned long long)f);
        return;
    }
    int64_t i = a / nT, j = a - i * nT;
    int32_t u = S[i], w = T[j];
    int64_t d = cost_l2(tr.X[u], tr.Y[u], tr.X[w], tr.Y[w]);
    int64_t g = cost_make(tr.X[u], tr.Y[u], dc) + cost_make(tr.X[w], tr.Y[w], dc);
    if (g <= d) {  // through the diagonal node: u -> diag -> w, both arcs exist
        atomicAdd(&out[1], (unsigned long long)(2 * f));
        return;
    }
    const int32_t lo = u < w ? u : w, hi = u < w ? w : u;
    if (!ws_arc_exists(lo, hi, tr.N, tr.X, tr.Y, tr.bb, tr.rep, tr.left, tr.right, s)) atomicAdd(&out[0], 1ull);
    atomicAdd(&out[1], (unsigned long long)f);
}

__global__ void k_certify_batch(const CertJob* __restrict__ jobs, unsigned long long* __restrict__ out) {
    const CertJob J = jobs[blockIdx.y];
    const NSInst* I = J.inst;
    unsigned long long* o = out + 2 * (int64_t)blockIdx.y;
    const int64_t mst = J.nS * J.nT;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < I->n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = I->pred[v], f = I->flow[v];
        if (a >= I->m || f <= 0) continue;
        if (a >= mst) {
            atomicAdd(&o[1], (unsigned long long)f);
            continue;
        }
        const int64_t i = a / J.nT, j = a - i * J.nT;
        const int32_t u = J.S[i], w = J.T[j];
        const WsTree& tr = J.tree;
        const int64_t d = cost_l2(tr.X[u], tr.Y[u], tr.X[w], tr.Y[w]);
        const int64_t g = cost_make(tr.X[u], tr.Y[u], J.dc) + cost_make(tr.X[w], tr.Y[w], J.dc);
        if (g <= d) {
            atomicAdd(&o[1], (unsigned long long)(2 * f));
            continue;
        }
        const int32_t lo = u < w ? u : w, hi = u < w ? w : u;
        if (!ws_arc_exists(lo, hi, tr.N, tr.X, tr.Y, tr.bb, tr.rep, tr.left, tr.right, J.s)) atomicAdd(&o[0], 1ull);
        atomicAdd(&o[1], (unsigned long long)f);
    }
}

__global__ void k_frontier_init(int64_t N, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                                int2* __restrict__ F) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N - 1) F[i] = make_int2(left[i], right[i]);
}

__global__ void k_ws_classify(const int2* __restrict__ F, int64_t nf, const int32_t* __restrict__ X,
                              const int32_t* __restrict__ Y, const int4* __restrict__ bb,
                              const int32_t* __restrict__ rep, const int32_t* __restrict__ left,
                              const int32_t* __restrict__ right, int64_t s, int64_t* __restrict__ flag,
                              int64_t* __restrict__ off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int2 p = F[i];
    TNode u = load_tnode(p.x, X, Y, bb, rep, left, right);
    TNode v = load_tnode(p.y, X, Y, bb, rep, left, right);
    int64_t w = well_separated(u, v, s) ? 1 : 0;
    flag[i] = w;
    off[i] = w;
}

// Well-separated pair -> two directed arcs between the representatives;
// otherwise split the node with the larger box side (ties split v) into two
// pairs of the next frontier.
__global__ void k_ws_expand(const int2* __restrict__ F, int64_t nf, const int64_t* __restrict__ flag,
                            const int64_t* __restrict__ off, const int32_t* __restrict__ X,
                            const int32_t* __restrict__ Y, const int4* __restrict__ bb,
                            const int32_t* __restrict__ rep, const int32_t* __restrict__ left,
                            const int32_t* __restrict__ right, int hb, uint64_t* __restrict__ arcs,
                            int2* __restrict__ Fn) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int2 p = F[i];
    TNode u = load_tnode(p.x, X, Y, bb, rep, left, right);
    TNode v = load_tnode(p.y, X, Y, bb, rep, left, right);
    int64_t o = off[i];
    if (flag[i]) {
        if (arcs) {  // null: only the frontier is built (the arcs are counted by the caller)
            arcs[2 * o] = ((uint64_t)u.rep << hb) | (uint64_t)v.rep;
            arcs[2 * o + 1] = ((uint64_t)v.rep << hb) | (uint64_t)u.rep;
        }
    } else {
        int64_t j = i - o;
        if (max_side(u) > max_side(v)) {
            Fn[2 * j] = make_int2(u.l, p.y);
            Fn[2 * j + 1] = make_int2(u.r, p.y);
        } else {
            Fn[2 * j] = make_int2(p.x, v.l);
            Fn[2 * j + 1] = make_int2(p.x, v.r);
        }
    }
}

// Count-only level of the frontier: well-separated pairs are counted, the
// others split (same rule as k_ws_expand) into the next frontier at slots
// taken with block-aggregated atomics -- the next frontier's order may differ
// from run to run, the counts do not.  lv[0] += well-separated pairs, lv[1] = size
// of the next frontier (capacity 2 nf).
__global__ void k_ws_count_split(const int2* __restrict__ F, int64_t nf, const int32_t* __restrict__ X,
                                 const int32_t* __restrict__ Y, const int4* __restrict__ bb,
                                 const int32_t* __restrict__ rep, const int32_t* __restrict__ left,
                                 const int32_t* __restrict__ right, int64_t s, int2* __restrict__ Fn,
                                 unsigned long long* __restrict__ lv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < nf;
    bool ws = false;
    int2 p = make_int2(0, 0);
    TNode u{}, v{};
    if (act) {
        p = F[i];
        u = load_tnode(p.x, X, Y, bb, rep, left, right);
        v = load_tnode(p.y, X, Y, bb, rep, left, right);
        ws = well_separated(u, v, s);
    }
    // block-aggregated: one pair of atomics per block (same-address atomics
    // from every warp of a level of millions of pairs would serialise)
    __shared__ unsigned s_ws[32], s_sp[32];
    __shared__ unsigned long long s_base;
    const unsigned mws = __ballot_sync(0xffffffffu, act && ws), msp = __ballot_sync(0xffffffffu, act && !ws);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        s_ws[wid] = __popc(mws);
        s_sp[wid] = __popc(msp);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tw = 0, ts = 0;
        for (int w = 0; w < nw; w++) {
            tw += s_ws[w];
            const unsigned c = s_sp[w];
            s_sp[w] = ts;  // exclusive prefix of the splits
            ts += c;
        }
        if (tw) atomicAdd(&lv[0], (unsigned long long)tw);
        s_base = ts ? atomicAdd(&lv[1], 2ull * (unsigned long long)ts) : 0ull;
    }
    __syncthreads();
    if (act && !ws) {
        const unsigned long long slot =
            s_base + 2ull * (unsigned long long)(s_sp[wid] + __popc(msp & ((1u << lane) - 1u)));
        if (max_side(u) > max_side(v)) {
            Fn[slot] = make_int2(u.l, p.y);
            Fn[slot + 1] = make_int2(u.r, p.y);
        } else {
            Fn[slot] = make_int2(p.x, v.l);
            Fn[slot + 1] = make_int2(p.x, v.r);
        }
    }
}

// Count-only, three levels per launch: the pair F[i] is tested, its two
// children, then their up to four children, all in registers (the same test
// and split rule as k_ws_count_split); separated pairs are counted and the up
// to eight great-grandchildren go to the next frontier at slots taken with
// block-aggregated atomics.  Equivalent to three launches of
// k_ws_count_split, with a third of the launches, host syncs and frontier
// traffic.  Slots at or above `cap` are not written and lv[2] records it (with
// cap = 8 nf it cannot happen).
// lv[0] += separated pairs, lv[1] = size of the next frontier.
PD_D void ws_split(const TNode& u, const TNode& v, int2 p, int2* c0, int2* c1) {
    if (max_side(u) > max_side(v)) {
        *c0 = make_int2(u.l, p.y);
        *c1 = make_int2(u.r, p.y);
    } else {
        *c0 = make_int2(p.x, v.l);
        *c1 = make_int2(p.x, v.r);
    }
}

__global__ void __launch_bounds__(256) k_ws_count_split3(const int2* __restrict__ F, int64_t nf,
                                                         const int32_t* __restrict__ X,
                                                         const int32_t* __restrict__ Y, const int4* __restrict__ bb,
                                                         const int32_t* __restrict__ rep,
                                                         const int32_t* __restrict__ left,
                                                         const int32_t* __restrict__ right, int64_t s,
                                                         int2* __restrict__ Fn, unsigned long long cap,
                                                         unsigned long long* __restrict__ lv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned cnt = 0;
    int2 L1[2], L2[4], L3[8];
    unsigned m1 = 0, m2 = 0, m3 = 0;  // which entries of each level are live
    if (i < nf) {
        const int2 p = F[i];
        const TNode u = load_tnode(p.x, X, Y, bb, rep, left, right);
        const TNode v = load_tnode(p.y, X, Y, bb, rep, left, right);
        if (well_separated(u, v, s)) cnt++;
        else {
            ws_split(u, v, p, &L1[0], &L1[1]);
            m1 = 3u;
        }
    }
#pragma unroll
    for (int q = 0; q < 2; q++)
        if (m1 >> q & 1u) {
            const TNode u = load_tnode(L1[q].x, X, Y, bb, rep, left, right);
            const TNode v = load_tnode(L1[q].y, X, Y, bb, rep, left, right);
            if (well_separated(u, v, s)) cnt++;
            else {
                ws_split(u, v, L1[q], &L2[2 * q], &L2[2 * q + 1]);
                m2 |= 3u << (2 * q);
            }
        }
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (m2 >> q & 1u) {
            const TNode u = load_tnode(L2[q].x, X, Y, bb, rep, left, right);
            const TNode v = load_tnode(L2[q].y, X, Y, bb, rep, left, right);
            if (well_separated(u, v, s)) cnt++;
            else {
                ws_split(u, v, L2[q], &L3[2 * q], &L3[2 * q + 1]);
                m3 |= 3u << (2 * q);
            }
        }
    // counts and slots: warp sums and prefixes, then one atomic per block
    __shared__ unsigned s_ws[32], s_sp[32];
    __shared__ unsigned long long s_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const unsigned k = __popc(m3);
    unsigned incl = k, wc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    for (int o = 16; o > 0; o >>= 1) wc += __shfl_xor_sync(0xffffffffu, wc, o);
    if (lane == 31) s_sp[wid] = incl;
    if (lane == 0) s_ws[wid] = wc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tw = 0, ts = 0;
        for (int w = 0; w < nw; w++) {
            tw += s_ws[w];
            const unsigned c = s_sp[w];
            s_sp[w] = (unsigned)ts;  // exclusive prefix of the warps' outputs
            ts += c;
        }
        if (tw) atomicAdd(&lv[0], tw);
        s_base = ts ? atomicAdd(&lv[1], ts) : 0ull;
        if (ts && s_base + ts > cap) atomicOr(&lv[2], 1ull);
    }
    __syncthreads();
    unsigned long long slot = s_base + s_sp[wid] + (incl - k);
#pragma unroll
    for (int q = 0; q < 8; q++)
        if (m3 >> q & 1u) {
            if (slot < cap) Fn[slot] = L3[q];
            slot++;
        }
}

// Diagonal arcs: u -> ā if u holds A mass, b̄ -> u if u holds B mass, and
// b̄ -> ā; absent arcs become the all-ones key, which sorts last.
__global__ void k_diag_arcs(int64_t N, const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB, int hb,
                            uint64_t sent, uint64_t* __restrict__ arcs, unsigned long long* __restrict__ counts) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > N) return;
    if (u == N) {
        if (arcs) arcs[2 * N] = ((uint64_t)(N + 1) << hb) | (uint64_t)N;
        return;
    }
    bool a = cntA[u] > 0, b = cntB[u] > 0;
    if (arcs) {  // null: count only
        arcs[2 * u] = a ? (((uint64_t)u << hb) | (uint64_t)N) : sent;
        arcs[2 * u + 1] = b ? (((uint64_t)(N + 1) << hb) | (uint64_t)u) : sent;
    }
    unsigned ma = __ballot_sync(__activemask(), a), mb = __ballot_sync(__activemask(), b);
    if ((threadIdx.x & 31) == (__ffs(__activemask()) - 1)) {
        atomicAdd(&counts[0], (unsigned long long)__popc(ma));
        atomicAdd(&counts[1], (unsigned long long)__popc(mb));
    }
}

// row_ptr from arc keys sorted by (tail, head).
__global__ void k_row_ptr(const uint64_t* __restrict__ key, int64_t m, int hb, int64_t nrows,
                          int64_t* __restrict__ row_ptr) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    int64_t t = (int64_t)(key[a] >> hb);
    int64_t tp = a == 0 ? -1 : (int64_t)(key[a - 1] >> hb);
    for (int64_t r = tp + 1; r <= t; r++) row_ptr[r] = a;
    if (a == m - 1)
        for (int64_t r = t + 1; r <= nrows; r++) row_ptr[r] = m;
}

__global__ void k_head_cost(const uint64_t* __restrict__ key, int64_t m, int hb, int64_t N,
                            const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int32_t* __restrict__ head,
                            int64_t* __restrict__ cost, DiagCost dc) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    uint64_t k = key[a];
    int64_t t = (int64_t)(k >> hb), h = (int64_t)(k & ((1ull << hb) - 1));
    head[a] = (int32_t)h;
    int64_t c = 0;
    if (t < N && h < N)
        c = cost_l2(X[t], Y[t], X[h], Y[h]);
    else if (t < N && h == N)
        c = cost_make(X[t], Y[t], dc);
    else if (t == N + 1 && h < N)
        c = cost_make(X[h], Y[h], dc);
    cost[a] = c;
}

__global__ void k_supply(int64_t N, const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB, int64_t FA,
                         int64_t FB, int64_t* __restrict__ sup) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < N) sup[u] = cntA[u] - cntB[u];
    if (u == N) sup[N] = -FA;
    if (u == N + 1) sup[N + 1] = FB;
}

__global__ void k_mass(int64_t N, const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB,
                       unsigned long long* __restrict__ out) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long a = 0, b = 0;
    if (u < N) {
        a = (unsigned long long)cntA[u];
        b = (unsigned long long)cntB[u];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&out[2], a);
        if (b) atomicAdd(&out[3], b);
    }
}

__global__ void k_check_nodes(const uint64_t* __restrict__ code, const int32_t* __restrict__ X,
                              const int32_t* __restrict__ Y, const int64_t* __restrict__ cntA,
                              const int64_t* __restrict__ cntB, int64_t N, unsigned long long* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t lim = 1 << 30;
    bool b = (i + 1 < N && !(code[i] < code[i + 1])) || X[i] <= -lim || X[i] >= lim || Y[i] <= -lim || Y[i] >= lim ||
             cntA[i] < 0 || cntB[i] < 0;
    if (b) atomicAdd(bad, 1ull);
}

pd_status validate_nodes(Ctx* c, const pd_nodes& nodes, cudaStream_t st) {
    int64_t N = nodes.n_nodes;
    if (N <= 0) return PD_OK;
    unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
    if (!sm) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, sizeof(unsigned long long), st));
    k_check_nodes<<<grid_for(N, 256), 256, 0, st>>>(nodes.morton, nodes.X, nodes.Y, nodes.cntA, nodes.cntB, N, sm); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (c->h_small[0])
        return fail(c, PD_EINVAL,
                    "nodes need strictly increasing Morton codes, |X|,|Y| < 2^30 and non-negative multiplicities");
    return PD_OK;
}

__global__ void k_merge_diag(const int64_t* __restrict__ rp, const int64_t* __restrict__ sup, int64_t N, int64_t m,
                             int64_t* __restrict__ mrp, int64_t* __restrict__ msup) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= N) mrp[i] = rp[i];
    if (i == N + 1) mrp[N + 1] = m - 1;
    if (i < N) msup[i] = sup[i];
    if (i == N) msup[N] = sup[N] + sup[N + 1];
}

// Network of nodes 0..N-1 plus one diagonal node N: rows 0..N-1 unchanged
// (their arcs to ā now point to N), row N = b̄'s row without its last arc
// b̄ -> ā (ā = N is the largest head of b̄'s row and ā's own row is empty).
pd_status merge_diagonal(Ctx* c, const pd_network& net, int64_t N, pd_network* out, cudaStream_t st) {
    int64_t* mrp = bufT<int64_t>(c, B_M_ROWPTR, N + 2);
    int64_t* msup = bufT<int64_t>(c, B_M_SUPPLY, N + 1);
    if (!mrp || !msup) return PD_ENOMEM;
    k_merge_diag<<<grid_for(N + 2, 256), 256, 0, st>>>(net.row_ptr, net.supply, N, net.n_arcs, mrp, msup); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    out->n_nodes = N + 1;
    out->n_arcs = net.n_arcs - 1;
    out->row_ptr = mrp;
    out->head = net.head;
    out->cost = net.cost;
    out->supply = msup;
    return PD_OK;
}

pd_status stage_network(Ctx* c, const pd_nodes& nodes, int64_t s, pd_network* out, float* ms_tree,
                        float* ms_wspd, float* ms_csr, cudaStream_t st, bool count_only, WsTree* tree,
                        const WsTree* given, DiagCost dc) {
    int64_t N = nodes.n_nodes;
    if (N >= (int64_t(1) << 31) - 4) return fail(c, PD_ECAPACITY, "more than 2^31 - 4 condensed nodes");
    if (s < 1) return fail(c, PD_EINVAL, "WSPD parameter s must be >= 1");
    cudaEvent_t ev[4];
    for (int q = 0; q < 4; q++) PD_TRY_CUDA(c, cudaEventCreate(&ev[q]));
    PD_TRY_CUDA(c, cudaEventRecord(ev[0], st));
    int64_t M = N > 1 ? N - 1 : 1;
    unsigned long long* cnts = bufT<unsigned long long>(c, B_SMALL, 64);
    if (!cnts) return PD_ENOMEM;
    const int32_t *left, *right, *rep;
    const int4* bb;
    if (given) {
        if (given->N != N || given->X != nodes.X || given->Y != nodes.Y)
            return fail(c, PD_EINVAL, "the given tree is not over these nodes");
        left = given->left;
        right = given->right;
        bb = given->bb;
        rep = given->rep;
    } else {
        int32_t* l = bufT<int32_t>(c, B_T_LEFT, M);
        int32_t* r = bufT<int32_t>(c, B_T_RIGHT, M);
        int4* b = bufT<int4>(c, B_T_BB, M);
        int32_t* rp = bufT<int32_t>(c, B_T_REP, M);
        int32_t* par_int = bufT<int32_t>(c, B_T_PARENT, M);
        int32_t* par_leaf = bufT<int32_t>(c, B_T_LPARENT, N);
        int32_t* visit = bufT<int32_t>(c, B_T_VISIT, M);
        if (!l || !r || !b || !rp || !par_int || !par_leaf || !visit) return PD_ENOMEM;
        left = l;
        right = r;
        bb = b;
        rep = rp;
        if (N >= 2) {
            k_karras<<<grid_for(N - 1, 256), 256, 0, st>>>(nodes.morton, N, l, r, par_int, par_leaf); pd::count_launch();
            PD_TRY_CUDA(c, cudaMemsetAsync(visit, 0, sizeof(int32_t) * M, st));
            k_bbox<<<grid_for(N, 256), 256, 0, st>>>(N, nodes.X, nodes.Y, l, r, par_int, par_leaf, b, rp, visit); pd::count_launch();
            PD_TRY_CUDA(c, cudaGetLastError());
        }
    }
    PD_TRY_CUDA(c, cudaEventRecord(ev[1], st));
    if (tree) *tree = WsTree{N, nodes.X, nodes.Y, left, right, bb, rep};

    int hb = bits_for((uint64_t)(N + 2));
    int kb = 2 * hb;
    uint64_t sent = (kb >= 64) ? ~0ull : ((1ull << kb) - 1);
    // WSPD frontier, one level at a time
    int64_t nf = N >= 2 ? N - 1 : 0;
    int64_t fcap = nf > 0 ? nf : 1;
    int2* F = bufT<int2>(c, B_F0, fcap);
    if (!F) return PD_ENOMEM;
    if (nf > 0) k_frontier_init<<<grid_for(nf, 256), 256, 0, st>>>(N, left, right, F); pd::count_launch();
    int64_t narcs = 0;
    int64_t acap = 0;
    uint64_t* arcs = nullptr;
    int fb = 0;
    int64_t* h = c->h_small;
    // count only: three levels per launch into a next frontier of 8 nf pairs
    // (at most 2^32, and only if that much memory can be had), else one level
    // into 2 nf
    while (count_only && nf > 0) {
        unsigned long long* lv = cnts + 12;
        const Buf nid = fb ? B_F0 : B_F1;
        int2* Fn = nullptr;
        if (8 * nf <= (int64_t(1) << 32)) {
            Fn = bufT<int2>(c, nid, 8 * nf);
            if (!Fn) c->err.clear();
        }
        PD_TRY_CUDA(c, cudaMemsetAsync(lv, 0, 3 * sizeof(unsigned long long), st));
        if (Fn) {
            k_ws_count_split3<<<grid_for(nf, 256), 256, 0, st>>>(F, nf, nodes.X, nodes.Y, bb, rep, left, right, s, Fn,
                                                                 (unsigned long long)(8 * nf), lv); pd::count_launch();
        } else {
            Fn = bufT<int2>(c, nid, 2 * nf);
            if (!Fn) return PD_ENOMEM;
            k_ws_count_split<<<grid_for(nf, 256), 256, 0, st>>>(F, nf, nodes.X, nodes.Y, bb, rep, left, right, s, Fn,
                                                                lv); pd::count_launch();
        }
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY_CUDA(c, cudaMemcpyAsync(h, lv, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        if (h[2]) return fail(c, PD_ECUDA, "WSPD count: frontier slots overflowed");  // cannot happen: 8 per pair
        narcs += 2 * h[0];
        nf = h[1];
        F = Fn;
        fb ^= 1;
    }
    while (nf > 0) {
        int64_t* flag = bufT<int64_t>(c, B_WSFLAG, nf);
        int64_t* off = bufT<int64_t>(c, B_WSOFF, nf);
        if (!flag || !off) return PD_ENOMEM;
        k_ws_classify<<<grid_for(nf, 256), 256, 0, st>>>(F, nf, nodes.X, nodes.Y, bb, rep, left, right, s, flag, off); pd::count_launch();
        PD_TRY(scan_i64(c, off, off, nf, (int64_t*)cnts + 8, st));
        PD_TRY_CUDA(c, cudaMemcpyAsync(h, (int64_t*)cnts + 8, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        int64_t nws = h[0];
        int64_t need = narcs + 2 * nws + 2 * N + 1;
        if (!count_only && need > acap) {
            // grow the arc buffer, keeping what is there
            int64_t ncap = need + need / 2 + 1024;
            uint64_t* tmp = bufT<uint64_t>(c, B_ARCKEY2, ncap);
            if (!tmp) return PD_ENOMEM;
            if (narcs) PD_TRY_CUDA(c, cudaMemcpyAsync(tmp, arcs, sizeof(uint64_t) * narcs, cudaMemcpyDeviceToDevice, st));
            uint64_t* na = bufT<uint64_t>(c, B_ARCKEY, ncap);
            if (!na) return PD_ENOMEM;
            if (narcs) PD_TRY_CUDA(c, cudaMemcpyAsync(na, tmp, sizeof(uint64_t) * narcs, cudaMemcpyDeviceToDevice, st));
            arcs = na;
            acap = ncap;
        }
        int64_t nn = 2 * (nf - nws);
        int2* Fn = bufT<int2>(c, fb ? B_F0 : B_F1, nn > 0 ? nn : 1);
        if (!Fn) return PD_ENOMEM;
        // F may have moved if its buffer grew: it did not (only Fn's buffer is resized here)
        k_ws_expand<<<grid_for(nf, 256), 256, 0, st>>>(F, nf, flag, off, nodes.X, nodes.Y, bb, rep, left, right, hb,
                                                        count_only ? nullptr : arcs + narcs, Fn); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        narcs += 2 * nws;
        nf = nn;
        F = Fn;
        fb ^= 1;
    }
    PD_TRY_CUDA(c, cudaEventRecord(ev[2], st));
    if (count_only) {
        // only the counts: arcs of the WSPD, diagonal arcs and the masses
        PD_TRY_CUDA(c, cudaMemsetAsync(cnts, 0, 8 * sizeof(unsigned long long), st));
        k_diag_arcs<<<grid_for(N + 1, 256), 256, 0, st>>>(N, nodes.cntA, nodes.cntB, hb, sent, nullptr, cnts); pd::count_launch();
        k_mass<<<grid_for(N, 256), 256, 0, st>>>(N, nodes.cntA, nodes.cntB, cnts); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY_CUDA(c, cudaMemcpyAsync(h, cnts, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaEventRecord(ev[3], st));
        PD_TRY_CUDA(c, cudaEventSynchronize(ev[3]));
        *out = pd_network{N + 2, narcs + h[0] + h[1] + 1, nullptr, nullptr, nullptr, nullptr};
        if (ms_tree) cudaEventElapsedTime(ms_tree, ev[0], ev[1]);
        if (ms_wspd) cudaEventElapsedTime(ms_wspd, ev[1], ev[2]);
        if (ms_csr) cudaEventElapsedTime(ms_csr, ev[2], ev[3]);
        for (int q = 0; q < 4; q++) cudaEventDestroy(ev[q]);
        return PD_OK;
    }
    if (!arcs) {
        acap = 2 * N + 1;
        arcs = bufT<uint64_t>(c, B_ARCKEY, acap);
        if (!arcs) return PD_ENOMEM;
    }
    // diagonal arcs + masses
    PD_TRY_CUDA(c, cudaMemsetAsync(cnts, 0, 8 * sizeof(unsigned long long), st));
    k_diag_arcs<<<grid_for(N + 1, 256), 256, 0, st>>>(N, nodes.cntA, nodes.cntB, hb, sent, arcs + narcs, cnts); pd::count_launch();
    k_mass<<<grid_for(N, 256), 256, 0, st>>>(N, nodes.cntA, nodes.cntB, cnts); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(h, cnts, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int64_t ntot = narcs + 2 * N + 1;
    uint64_t* alt = bufT<uint64_t>(c, B_ARCKEY2, ntot);
    if (!alt) return PD_ENOMEM;
    PD_TRY(sort_u64(c, arcs, alt, nullptr, nullptr, ntot, kb, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    int64_t na = h[0], nb = h[1], FA = h[2], FB = h[3];
    int64_t m = narcs + na + nb + 1;
    int64_t nrows = N + 2;
    out->n_nodes = nrows;
    out->n_arcs = m;
    out->row_ptr = bufT<int64_t>(c, B_ROWPTR, nrows + 1);
    out->head = bufT<int32_t>(c, B_HEAD, m);
    out->cost = bufT<int64_t>(c, B_COST, m);
    out->supply = bufT<int64_t>(c, B_SUPPLY, nrows);
    if (!out->row_ptr || !out->head || !out->cost || !out->supply) return PD_ENOMEM;
    k_row_ptr<<<grid_for(m, 256), 256, 0, st>>>(arcs, m, hb, nrows, out->row_ptr); pd::count_launch();
    k_head_cost<<<grid_for(m, 256), 256, 0, st>>>(arcs, m, hb, N, nodes.X, nodes.Y, out->head, out->cost, dc); pd::count_launch();
    k_supply<<<grid_for(N + 2, 256), 256, 0, st>>>(N, nodes.cntA, nodes.cntB, FA, FB, out->supply); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaEventRecord(ev[3], st));
    PD_TRY_CUDA(c, cudaEventSynchronize(ev[3]));
    if (ms_tree) cudaEventElapsedTime(ms_tree, ev[0], ev[1]);
    if (ms_wspd) cudaEventElapsedTime(ms_wspd, ev[1], ev[2]);
    if (ms_csr) cudaEventElapsedTime(ms_csr, ev[2], ev[3]);
    for (int q = 0; q < 4; q++) cudaEventDestroy(ev[q]);
    return PD_OK;
}

}  // namespace pd
