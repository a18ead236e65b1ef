// Primal network simplex for the uncapacitated min-cost flow, one CTA per
// instance (the min-cost flow of the network-simplex section: block search
// pivoting, run to optimality).
//
// GPU layout.  Pricing is the parallel part: the whole CTA evaluates a block
// of arcs (reduced cost c - pi(tail) + pi(head)) and reduces to the most
// negative one.  The pivot walk (apex, leaving arc, flow change) is sequential
// on one thread.  The spanning tree is kept as an explicit preorder array
// (ord, pos, size), so that re-hanging the cut subtree is a handful of
// contiguous segment moves done by all threads, with per-segment depth shifts
// and one potential shift -- no pointer chasing over the subtree.
//
// Big-M start: node i has an artificial arc to (supply >= 0) or from (< 0) an
// extra root; zero-flow tree arcs point to the root (strongly feasible tree),
// and the leaving arc is the last blocking arc met when the cycle is walked
// from the apex in the direction of the entering arc, which rules out cycling.
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
    if (a < I.mst) {
        int64_t i = a / I.nT;
        *t = (int32_t)i;
        *h = (int32_t)(I.nS + (a - i * I.nT));
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
    return big;
}

PD_D void take_min(int64_t rc, int64_t a, int64_t& lb, int64_t& li) {
    if (rc < lb || (rc == lb && rc < 0 && a < li)) {
        lb = rc;
        li = a;
    }
}

// Bytes of dynamic shared memory for the hot node arrays of n + 1 nodes.
size_t ns_smem_bytes(int64_t N1) { return (size_t)N1 * (8 + 4 + 4 + 4 + 4 + 4 + 1) + 64; }

constexpr int NS_LMAX = 512;  // half-cycle entries kept in shared memory

__global__ void __launch_bounds__(NS_THREADS) k_netsimplex(NSInst* insts, int64_t big) {
    NSInst& G = insts[blockIdx.x];
    NSInst I = G;  // local copy: the hot arrays may be redirected to shared memory
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t n = I.n, root = n, N1 = n + 1;
    const int64_t M = I.m + n;  // arcs including the artificial ones
    extern __shared__ __align__(16) unsigned char dyn[];
    if (I.smem_nodes) {
        unsigned char* p = dyn;
        I.pi = (int64_t*)p;
        p += sizeof(int64_t) * N1;
        I.flow = (int32_t*)p;
        p += sizeof(int32_t) * N1;
        I.parent = (int32_t*)p;
        p += sizeof(int32_t) * N1;
        I.depth = (int32_t*)p;
        p += sizeof(int32_t) * N1;
        I.size = (int32_t*)p;
        p += sizeof(int32_t) * N1;
        I.pos = (int32_t*)p;
        p += sizeof(int32_t) * N1;
        I.up = (uint8_t*)p;
    }
    __shared__ int32_t pa[NS_LMAX], pb[NS_LMAX];
    int32_t* gpa = I.path;
    int32_t* gpb = I.path + N1;
    __shared__ int32_t s_la, s_lb, s_join, s_i, s_j;
    __shared__ int64_t s_ce;

    __shared__ int64_t s_val[32];
    __shared__ int64_t s_idx[32];
    __shared__ int64_t s_best, s_bidx, s_next, s_dpi;
    __shared__ int32_t s_go, s_status;
    // re-hang plan
    __shared__ int32_t s_k, s_L0, s_S, s_pr, s_nseg;
    const int32_t SEGN = 2 * n + 3;
    int32_t* seg_start = I.seg;
    int32_t* seg_len = I.seg + SEGN;
    int32_t* seg_out = I.seg + 2 * SEGN;
    int32_t* seg_dd = I.seg + 3 * SEGN;

    // ---- initial tree: the root star --------------------------------------
    for (int32_t i = tid; i < n; i += NS_THREADS) {
        int64_t s = I.supply[i];
        I.parent[i] = root;
        I.pred[i] = I.m + i;
        I.up[i] = s >= 0;
        I.flow[i] = (int32_t)(s >= 0 ? s : -s);
        I.pi[i] = s >= 0 ? big : -big;  // reduced cost of the artificial arc is 0
        I.depth[i] = 1;
        I.ord[1 + i] = i;
        I.pos[i] = 1 + i;
        I.size[i] = 1;
    }
    if (tid == 0) {
        I.parent[root] = -1;
        I.pred[root] = -1;
        I.up[root] = 0;
        I.flow[root] = 0;
        I.pi[root] = 0;
        I.depth[root] = 0;
        I.ord[0] = root;
        I.pos[root] = 0;
        I.size[root] = N1;
        s_next = 0;
        s_status = 0;
    }
    __syncthreads();
    const uint64_t t0 = ns_now();
    int64_t pivots = 0, degen = 0, nscan = 0;
    const int64_t B = I.block < 1 ? 1 : I.block;

    for (;;) {
        // ---- pricing: blocks of B arcs from s_next, first block holding a
        // negative reduced cost wins (most negative in it, lowest index on ties)
        int64_t scanned = 0, a0 = s_next;
        int64_t best = 0, bidx = -1;
        while (scanned < M) {
            const int64_t aend = a0 + B < M ? a0 + B : M;
            const int64_t len = aend - a0;
            int64_t lb = 0, li = -1;
            // chunks of 8 consecutive arcs per thread, 16-byte vector loads
            for (int64_t c0 = a0 + 8 * (int64_t)tid; c0 < aend; c0 += 8 * NS_THREADS) {
                if (c0 + 8 <= aend && c0 + 8 <= I.mst) {
                    int4 w0 = __ldcs((const int4*)(I.cmat + c0));
                    int4 w1 = __ldcs((const int4*)(I.cmat + c0 + 4));
                    int32_t cv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                    int64_t i = c0 / I.nT, j = c0 - i * I.nT;
                    int64_t pt = I.pi[i];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        int64_t rc = (int64_t)cv[q] - pt + I.pi[I.nS + j];
                        take_min(rc, c0 + q, lb, li);
                        if (++j == I.nT) {
                            j = 0;
                            ++i;
                            if (q < 7) pt = I.pi[i];
                        }
                    }
                } else if (c0 >= I.mst && c0 + 8 <= aend && c0 + 8 <= I.m && ((c0 - I.mst) & 7) == 0) {
                    const int64_t x = c0 - I.mst;
                    int4 t0 = __ldcs((const int4*)(I.tail + x)), t1 = __ldcs((const int4*)(I.tail + x + 4));
                    int4 h0 = __ldcs((const int4*)(I.head + x)), h1 = __ldcs((const int4*)(I.head + x + 4));
                    int4 k0 = __ldcs((const int4*)(I.cost + x)), k1 = __ldcs((const int4*)(I.cost + x + 4));
                    int32_t tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
                    int32_t hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
                    int32_t cv[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
#pragma unroll
                    for (int q = 0; q < 8; q++) take_min((int64_t)cv[q] - I.pi[tv[q]] + I.pi[hv[q]], c0 + q, lb, li);
                } else {
                    int64_t ce = c0 + 8 < aend ? c0 + 8 : aend;
                    for (int64_t a = c0; a < ce; a++) {
                        int32_t t, h;
                        arc_ends(I, a, &t, &h);
                        take_min(arc_cost(I, a, big) - I.pi[t] + I.pi[h], a, lb, li);
                    }
                }
            }
            // CTA argmin (value, then index)
            for (int off = 16; off > 0; off >>= 1) {
                int64_t ov = __shfl_xor_sync(0xffffffffu, lb, off);
                int64_t oi = __shfl_xor_sync(0xffffffffu, li, off);
                if (ov < lb || (ov == lb && oi >= 0 && (li < 0 || oi < li))) {
                    lb = ov;
                    li = oi;
                }
            }
            if (lane == 0) {
                s_val[wid] = lb;
                s_idx[wid] = li;
            }
            __syncthreads();
            if (wid == 0) {
                lb = s_val[lane];
                li = s_idx[lane];
                for (int off = 16; off > 0; off >>= 1) {
                    int64_t ov = __shfl_xor_sync(0xffffffffu, lb, off);
                    int64_t oi = __shfl_xor_sync(0xffffffffu, li, off);
                    if (ov < lb || (ov == lb && oi >= 0 && (li < 0 || oi < li))) {
                        lb = ov;
                        li = oi;
                    }
                }
                if (lane == 0) {
                    s_best = lb;
                    s_bidx = li;
                }
            }
            __syncthreads();
            best = s_best;
            bidx = s_bidx;
            scanned += len;
            nscan += len;
            a0 = aend >= M ? 0 : aend;
            __syncthreads();
            if (best < 0) break;
        }
        if (best >= 0 || bidx < 0) break;  // optimal
        if (tid == 0) s_go = (pivots < I.max_pivots && ns_now() - t0 <= I.time_limit_ns) ? 1 : 0;
        __syncthreads();
        if (!s_go) {
            if (tid == 0) s_status = 2;
            __syncthreads();
            break;
        }
        pivots++;

        // ---- pivot: apex walk (one thread), then the two recorded half-cycles
        // are processed by warp 0 (leaving arc, flows, ancestor sizes) ---------
        if (wid == 0) {
            if (lane == 0) {
                s_next = a0;
                int64_t e = bidx;
                int32_t i, j;
                arc_ends(I, e, &i, &j);
                s_ce = arc_cost(I, e, big);
                int32_t u = i, v = j, la = 0, lb = 0;
                while (u != v) {
                    int32_t du = I.depth[u], dv = I.depth[v];
                    if (du >= dv) {
                        if (la < NS_LMAX) pa[la] = u; else gpa[la] = u;
                        la++;
                        u = I.parent[u];
                    }
                    if (dv >= du) {
                        if (lb < NS_LMAX) pb[lb] = v; else gpb[lb] = v;
                        lb++;
                        v = I.parent[v];
                    }
                }
                s_la = la;
                s_lb = lb;
                s_join = u;
                s_i = i;
                s_j = j;
            }
            __syncwarp();
            const int32_t la = s_la, lb = s_lb, i = s_i, j = s_j;
#define PA(t) ((t) < NS_LMAX ? pa[t] : gpa[t])
#define PB(t) ((t) < NS_LMAX ? pb[t] : gpb[t])
            // leaving arc: last blocking arc walking from the apex along the
            // cycle -- on the i-side the one closest to i (smallest index), on
            // the j-side the one closest to the apex (largest index), j-side
            // preferred on ties.
            int64_t fi = INT64_MAX, ti = INT32_MAX, fj = INT64_MAX, tj = -1;
            for (int32_t t = lane; t < la; t += 32) {
                int32_t x = PA(t);
                if (I.up[x]) {
                    int64_t f = I.flow[x];
                    if (f < fi || (f == fi && t < ti)) {
                        fi = f;
                        ti = t;
                    }
                }
            }
            for (int32_t t = lane; t < lb; t += 32) {
                int32_t x = PB(t);
                if (!I.up[x]) {
                    int64_t f = I.flow[x];
                    if (f < fj || (f == fj && t > tj)) {
                        fj = f;
                        tj = t;
                    }
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                int64_t of = __shfl_xor_sync(0xffffffffu, fi, off);
                int64_t ot = __shfl_xor_sync(0xffffffffu, ti, off);
                if (of < fi || (of == fi && ot < ti)) {
                    fi = of;
                    ti = ot;
                }
                of = __shfl_xor_sync(0xffffffffu, fj, off);
                ot = __shfl_xor_sync(0xffffffffu, tj, off);
                if (of < fj || (of == fj && ot > tj)) {
                    fj = of;
                    tj = ot;
                }
            }
            int side;
            int64_t delta;
            int32_t tl;
            if (tj >= 0 && fj <= fi) {
                side = 2;
                delta = fj;
                tl = (int32_t)tj;
            } else if (ti != INT32_MAX) {
                side = 1;
                delta = fi;
                tl = (int32_t)ti;
            } else {
                side = 0;
                delta = 0;
                tl = 0;
            }
            if (side == 0) {
                if (lane == 0) {
                    s_status = 3;
                    s_go = 0;
                }
            } else {
                if (delta > 0) {
                    const int32_t d32 = (int32_t)delta;
                    for (int32_t t = lane; t < la; t += 32) {
                        int32_t x = PA(t);
                        I.flow[x] += I.up[x] ? -d32 : d32;
                    }
                    for (int32_t t = lane; t < lb; t += 32) {
                        int32_t x = PB(t);
                        I.flow[x] += I.up[x] ? d32 : -d32;
                    }
                }
                const int32_t leave = side == 1 ? PA(tl) : PB(tl);
                const int32_t S = I.size[leave];
                __syncwarp();
                // the cut subtree leaves the chain above `leave` and joins r's chain
                if (side == 1) {
                    for (int32_t t = tl + 1 + lane; t < la; t += 32) I.size[PA(t)] -= S;
                    for (int32_t t = lane; t < lb; t += 32) I.size[PB(t)] += S;
                } else {
                    for (int32_t t = tl + 1 + lane; t < lb; t += 32) I.size[PB(t)] -= S;
                    for (int32_t t = lane; t < la; t += 32) I.size[PA(t)] += S;
                }
                __syncwarp();
                if (lane == 0) {
                    if (delta == 0) degen++;
                    const int64_t e = bidx;
                    const int32_t q = side == 1 ? i : j, r = side == 1 ? j : i;
                    int64_t rc = s_ce - I.pi[i] + I.pi[j];
                    s_dpi = side == 1 ? rc : -rc;
                    const int32_t k = tl;  // path q = v0 .. vk = leave
#define PV(t) (side == 1 ? PA(t) : PB(t))
                    // new preorder of the cut subtree, re-rooted at q, as segments of the old order
                    const int32_t dr = I.depth[r];
                    int32_t ns = 0, out = 0;
                    seg_start[ns] = I.pos[q];
                    seg_len[ns] = I.size[q];
                    seg_out[ns] = out;
                    seg_dd[ns] = dr + 1 - I.depth[q];
                    out += seg_len[ns];
                    ns++;
                    for (int32_t t = 1; t <= k; t++) {
                        int32_t vt = PV(t), vp = PV(t - 1);
                        int32_t dd = dr + 1 + t - I.depth[vt];
                        int32_t a_len = I.pos[vp] - I.pos[vt];
                        int32_t b_st = I.pos[vp] + I.size[vp];
                        int32_t b_len = I.pos[vt] + I.size[vt] - b_st;
                        seg_start[ns] = I.pos[vt];
                        seg_len[ns] = a_len;
                        seg_out[ns] = out;
                        seg_dd[ns] = dd;
                        out += a_len;
                        ns++;
                        seg_start[ns] = b_st;
                        seg_len[ns] = b_len;
                        seg_out[ns] = out;
                        seg_dd[ns] = dd;
                        out += b_len;
                        ns++;
                    }
                    // new subtree sizes along the path (suffix sums of A_t + B_t)
                    int32_t acc = 0;
                    for (int32_t t = k; t >= 1; t--) {
                        acc += seg_len[2 * t - 1] + seg_len[2 * t];
                        I.tmp[t] = acc;
                    }
                    s_L0 = I.pos[leave];
                    s_pr = I.pos[r];
                    // parent / pred / direction / flow along the reversed path
                    int64_t prev_pred = e;
                    uint8_t prev_up = (uint8_t)(i == q ? 1 : 0);  // e runs i -> j
                    int32_t prev_flow = (int32_t)delta;
                    int32_t prev_par = r;
                    for (int32_t t = 0; t <= k; t++) {
                        int32_t vt = PV(t);
                        int64_t op = I.pred[vt];
                        uint8_t ou = I.up[vt];
                        int32_t of = I.flow[vt];
                        I.pred[vt] = prev_pred;
                        I.up[vt] = prev_up;
                        I.flow[vt] = prev_flow;
                        I.parent[vt] = prev_par;
                        prev_pred = op;
                        prev_up = (uint8_t)!ou;
                        prev_flow = of;
                        prev_par = vt;
                    }
                    I.size[q] = S;
                    for (int32_t t = 1; t <= k; t++) I.size[PV(t)] = I.tmp[t];
#undef PV
                    s_k = k;
                    s_nseg = ns;
                    s_S = S;
                    s_go = 1;
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
            // new order over the affected index range [lo, hi)
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
            for (int32_t x = lo + tid; x < hi; x += NS_THREADS) {
                int32_t node;
                if (x >= ins && x < ins + S) {
                    int32_t o = x - ins;
                    int32_t sl = 0, sh = nseg - 1;  // last segment with seg_out <= o
                    while (sl < sh) {
                        int32_t mid = (sl + sh + 1) >> 1;
                        if (seg_out[mid] <= o)
                            sl = mid;
                        else
                            sh = mid - 1;
                    }
                    int32_t sidx = sl;
                    node = I.ord[seg_start[sidx] + (o - seg_out[sidx])];
                    I.depth[node] += seg_dd[sidx];
                    I.pi[node] += dpi;
                } else if (pr < L0) {
                    // [pr+1, L0) shifted right by S
                    node = I.ord[x - S];
                } else {
                    // [L0+S, pr] shifted left by S
                    node = I.ord[x + S];
                }
                I.tmp[x] = node;
            }
            __syncthreads();
            for (int32_t x = lo + tid; x < hi; x += NS_THREADS) {
                int32_t node = I.tmp[x];
                I.ord[x] = node;
                I.pos[node] = x;
            }
            __syncthreads();
        }
    }
    // ---- result ------------------------------------------------------------
    __syncthreads();
    if (I.smem_nodes) {
        for (int32_t v = tid; v < N1; v += NS_THREADS) {
            G.pi[v] = I.pi[v];
            G.flow[v] = I.flow[v];
            G.parent[v] = I.parent[v];
            G.depth[v] = I.depth[v];
            G.size[v] = I.size[v];
            G.pos[v] = I.pos[v];
            G.up[v] = I.up[v];
        }
    }
    if (tid == 0) {
        G.pivots = pivots;
        G.degenerate = degen;
        G.scanned = nscan;
        G.status = s_status;
    }
    // objective over tree arcs, and feasibility (no flow left on artificial arcs)
    __shared__ unsigned long long s_obj, s_art;
    if (tid == 0) {
        s_obj = 0;
        s_art = 0;
    }
    __syncthreads();
    unsigned long long obj = 0, art = 0;
    for (int32_t v = tid; v < n; v += NS_THREADS) {
        int64_t a = I.pred[v], f = I.flow[v];
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
        G.opt = (int64_t)s_obj;
        if (s_status == 0 && s_art) G.status = 1;
    }
}

}  // namespace pd

namespace pd {

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

// Network simplex on an arc list (one CTA).  cmax = largest arc cost.
pd_status ns_solve_arcs(Ctx* c, int32_t n, int64_t m, int64_t mst, int64_t nS, int64_t nT, const int32_t* cmat,
                        const int32_t* tail, const int32_t* head, const int32_t* cost, const int64_t* supply,
                        int64_t cmax, const pd_opts& o, NSOut* out, cudaStream_t st) {
    *out = NSOut{};
    if (n <= 0) return PD_OK;
    int64_t N1 = (int64_t)n + 1;
    NSInst h{};
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
    h.pred = bufT<int64_t>(c, B_NS_PRED, N1);
    h.depth = bufT<int32_t>(c, B_NS_DEPTH, N1);
    h.flow = bufT<int32_t>(c, B_NS_FLOW, N1);
    h.up = bufT<uint8_t>(c, B_NS_UP, N1);
    h.ord = bufT<int32_t>(c, B_NS_ORD, N1);
    h.pos = bufT<int32_t>(c, B_NS_POS, N1);
    h.size = bufT<int32_t>(c, B_NS_SIZE, N1);
    h.tmp = bufT<int32_t>(c, B_NS_TMP, N1);
    h.path = bufT<int32_t>(c, B_NS_PATH, 2 * N1);
    h.seg = bufT<int32_t>(c, B_NS_SEG, 4 * (2 * N1 + 3));
    NSInst* d = bufT<NSInst>(c, B_NS_INST, 1);
    if (!h.pi || !h.parent || !h.pred || !h.depth || !h.flow || !h.up || !h.ord || !h.pos || !h.size || !h.tmp ||
        !h.path || !h.seg || !d)
        return PD_ENOMEM;
    int64_t M = m + n;
    int64_t blk = o.ns_block > 0 ? o.ns_block : (int64_t)sqrt((double)M);
    if (blk < 2048) blk = 2048;
    blk = (blk + 7) & ~(int64_t)7;  // blocks start at multiples of 8 (vector loads)
    h.block = blk;
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
    int64_t big = N1 * (cmax + 1) + 1;
    size_t smem = ns_smem_bytes(N1);
    int max_optin = 0;
    PD_TRY_CUDA(c, cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    h.smem_nodes = (o.ns_smem != 0 && smem + 6144 <= (size_t)max_optin) ? 1 : 0;
    if (!h.smem_nodes) smem = 0;
    PD_TRY_CUDA(c, cudaFuncSetAttribute(k_netsimplex, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PD_TRY_CUDA(c, cudaMemcpyAsync(d, &h, sizeof(NSInst), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0, e1;
    PD_TRY_CUDA(c, cudaEventCreate(&e0));
    PD_TRY_CUDA(c, cudaEventCreate(&e1));
    PD_TRY_CUDA(c, cudaEventRecord(e0, st));
    k_netsimplex<<<1, NS_THREADS, smem, st>>>(d, big); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaEventRecord(e1, st));
    NSInst r;
    PD_TRY_CUDA(c, cudaMemcpyAsync(&r, d, sizeof(NSInst), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    float nms = 0.f;
    cudaEventElapsedTime(&nms, e0, e1);
    c->last_ns_ms += nms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->opt = r.opt;
    out->pivots = r.pivots;
    out->degenerate = r.degenerate;
    out->scanned = r.scanned;
    out->status = r.status;
    if (r.status == 2) return fail(c, PD_ETIMEOUT, "network simplex pivot cap or time limit reached");
    if (r.status == 1) return fail(c, PD_EINFEASIBLE, "network has no feasible flow");
    if (r.status == 3) return fail(c, PD_EINFEASIBLE, "network simplex found an unbounded cycle");
    if (r.status != 0) return fail(c, PD_ECUDA, "network simplex failed");
    return PD_OK;
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
                                 int32_t* __restrict__ cost, unsigned long long* __restrict__ bad) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t mst = nS * nT;
    int64_t D = nS + nT;
    int64_t c;
    if (a < mst) {
        int64_t i = a / nT, j = a - i * nT;
        int32_t u = S[i], v = T[j];
        int64_t d = cost_l2(X[u], Y[u], X[v], Y[v]);
        int64_t g = cost_diag(X[u], Y[u]) + cost_diag(X[v], Y[v]);
        c = d < g ? d : g;
        if (c >= (int64_t(1) << 31)) atomicAdd(bad, 1ull);
        cmat[a] = (int32_t)c;
        return;
    } else if (dside < 0 && a < mst + nS) {
        int64_t i = a - mst;
        int32_t u = S[i];
        c = cost_diag(X[u], Y[u]);
        tail[a - mst] = (int32_t)i;
        head[a - mst] = (int32_t)D;
    } else if (dside > 0 && a < mst + nT) {
        int64_t j = a - mst;
        int32_t v = T[j];
        c = cost_diag(X[v], Y[v]);
        tail[a - mst] = (int32_t)D;
        head[a - mst] = (int32_t)(nS + j);
    } else {
        return;
    }
    if (c >= (int64_t(1) << 31)) atomicAdd(bad, 1ull);
    cost[a - mst] = (int32_t)c;
}

// Certificate: every source->sink pair that carries flow on its direct route
// must be an arc of the sparse network (then the transport optimum, a lower
// bound on the sparse optimum, is attained on the sparse network).  Also
// counts the arcs of the sparse network the flow uses (rounding slack).
__global__ void k_certify_transport(const NSInst* __restrict__ I, const int32_t* __restrict__ S,
                                    const int32_t* __restrict__ T, int64_t nS, int64_t nT,
                                    const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                                    const int64_t* __restrict__ rp, const int32_t* __restrict__ hd,
                                    unsigned long long* __restrict__ out) {
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
    int64_t d = cost_l2(X[u], Y[u], X[w], Y[w]);
    int64_t g = cost_diag(X[u], Y[u]) + cost_diag(X[w], Y[w]);
    if (g <= d) {  // through the diagonal node: u -> diag -> w, both arcs exist
        atomicAdd(&out[1], (unsigned long long)(2 * f));
        return;
    }
    int64_t lo = rp[u], hi = rp[u + 1] - 1;
    bool found = false;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t h = hd[mid];
        if (h == w) {
            found = true;
            break;
        }
        if (h < w)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    if (!found) atomicAdd(&out[0], 1ull);
    atomicAdd(&out[1], (unsigned long long)f);
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
    NSOut r;
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

// The W1 network: try the transportation form with the certificate first
// when it is not much larger than the sparse network, else (or if the
// certificate fails) run the simplex on the sparse network itself.
pd_status ns_solve_w1(Ctx* c, const pd_nodes& nodes, const pd_network& ws, const pd_network& merged,
                      const pd_opts& o, SolveStats* out, cudaStream_t st) {
    *out = SolveStats{};
    int64_t N = nodes.n_nodes;
    if (N == 0) return ns_solve_network(c, merged, o, out, st);
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
    // masses: diagonal supply |B| - |A| from the merged network's last node
    int64_t dsup = 0;
    PD_TRY_CUDA(c, cudaMemcpyAsync(&dsup, merged.supply + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    int64_t mst = nS * nT;
    int64_t mt = mst + (dsup < 0 ? nS : (dsup > 0 ? nT : 0));
    bool try_transport = o.ns_transport != 0 && mt <= 2 * ws.n_arcs + 4096 && mt < (int64_t(1) << 31);
    if (try_transport) {
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
        PD_TRY_CUDA(c, cudaMemcpyAsync(sup + nS + nT, &dsup, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, 8 * sizeof(unsigned long long), st));
        if (mt > 0)
            k_transport_arcs<<<grid_for(mt, 256), 256, 0, st>>>(S, T, nS, nT, dsup < 0 ? -1 : (dsup > 0 ? 1 : 0),
                                                                  nodes.X, nodes.Y, cmat, tail, head, cost, sm); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        if (mst > 0) k_max_cost32<<<grid_for(mst, 256), 256, 0, st>>>(cmat, mst, sm + 1); pd::count_launch();
        if (mx > 0) k_max_cost32<<<grid_for(mx, 256), 256, 0, st>>>(cost, mx, sm + 1); pd::count_launch();
        PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        if (c->h_small[0] == 0) {
            NSOut r;
            PD_TRY(ns_solve_arcs(c, (int32_t)nt, mt, mst, nS, nT, cmat, tail, head, cost, sup, c->h_small[1], o, &r,
                                 st));
            PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, 4 * sizeof(unsigned long long), st));
            k_certify_transport<<<grid_for(nt, 256), 256, 0, st>>>(bufT<NSInst>(c, B_NS_INST, 1), S, T, nS, nT,
                                                                    nodes.X, nodes.Y, ws.row_ptr, ws.head, sm); pd::count_launch();
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
    }
    int64_t piv = out->pivots, fails = out->cert_failures, scn = out->scanned;
    PD_TRY(ns_solve_network(c, merged, o, out, st));
    out->pivots += piv;
    out->scanned += scn;
    out->cert_failures = fails;
    return PD_OK;
}

}  // namespace pd
