// The paper's split tree (WSPD section): the bounding box of a point set is
// cut in the middle of its longest side, recursively, down to single points.
// It is the tree the paper builds its WSPD on; the default tree of this
// library is the radix tree over Morton order (wspd.cu), and this one is the
// option pd_opts.tree = 1.
//
// GPU layout: the recursion runs level by level over a permutation of the
// nodes.  Every segment of positions [lo, hi] is one tree node of the current
// level; per level one pass reduces each segment's tight box and leftmost
// member (warp-aggregated atomics, records indexed by lo), one pass flags the
// points on the lower half of the longest side, an exclusive scan of the flags
// gives each point's rank within its side, and one pass scatters the points
// into the two halves (a stable partition, so the leaf order is exactly the
// sequential recursion's) and writes the tree node.  A node of 2^31 integer
// extent is at most 78 levels deep: a cut halves the longest side, so the sum
// of the two sides drops by a quarter at every level.
//
// Node numbering is the radix tree's (root 0, a child covering [lo, split]
// is numbered split, one covering [split + 1, hi] split + 1, leaves ~position),
// and the nodes are renumbered by their leaf position, so the WSPD frontier,
// the network builder and the tree certificate run unchanged on this tree.
#include "internal.h"
#include "prims.cuh"

namespace pd {

namespace {

constexpr unsigned FULL = 0xffffffffu;

PD_D uint64_t left_key(int32_t x, int32_t y) {  // min over a set = its leftmost point (min X, then min Y)
    return ((uint64_t)(uint32_t)(x + (1 << 30)) << 32) | (uint32_t)(y + (1 << 30));
}

}  // namespace

__global__ void k_sp_init(int64_t N, int32_t* __restrict__ ord, int32_t* __restrict__ seg,
                          int32_t* __restrict__ shi, int32_t* __restrict__ snum) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    ord[p] = (int32_t)p;
    seg[p] = 0;
    if (p == 0) {
        shi[0] = (int32_t)(N - 1);
        snum[0] = 0;
    }
}

// Heads of the segments still to cut: empty box, no leftmost point yet.
__global__ void k_sp_reset(int64_t N, const int32_t* __restrict__ seg, const int32_t* __restrict__ shi,
                           int4* __restrict__ sbb, unsigned long long* __restrict__ srep) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || seg[p] != p || shi[p] <= p) return;
    sbb[p] = make_int4(INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN);
    srep[p] = ~0ull;
}

// Tight box and leftmost point of every segment still to cut: lanes of a warp
// in the same segment combine first, one atomic per segment and warp.
__global__ void k_sp_box(int64_t N, const int32_t* __restrict__ ord, const int32_t* __restrict__ seg,
                         const int32_t* __restrict__ shi, const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                         int4* __restrict__ sbb, unsigned long long* __restrict__ srep) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t lo = -1, x = 0, y = 0;
    if (p < N) {
        const int32_t l = seg[p];
        if (shi[l] > l) {
            lo = l;
            const int32_t v = ord[p];
            x = X[v];
            y = Y[v];
        }
    }
    const unsigned peers = __match_any_sync(FULL, lo);
    int32_t mnx = x, mxx = x, mny = y, mxy = y;
    uint64_t key = left_key(x, y);
    for (int l = 0; l < 32; l++) {
        const int32_t ox = __shfl_sync(FULL, x, l), oy = __shfl_sync(FULL, y, l);
        if ((peers >> l) & 1u) {
            mnx = min(mnx, ox);
            mxx = max(mxx, ox);
            mny = min(mny, oy);
            mxy = max(mxy, oy);
            const uint64_t k = left_key(ox, oy);
            key = k < key ? k : key;
        }
    }
    if (lo >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
        atomicMin(&sbb[lo].x, mnx);
        atomicMax(&sbb[lo].y, mxx);
        atomicMin(&sbb[lo].z, mny);
        atomicMax(&sbb[lo].w, mxy);
        atomicMin(&srep[lo], (unsigned long long)key);
    }
}

// 1 for a point on the lower half of its segment's longest side (x on ties):
// twice its coordinate below min + max.  The segment's leftmost point names
// itself in srepn.
__global__ void k_sp_flag(int64_t N, const int32_t* __restrict__ ord, const int32_t* __restrict__ seg,
                          const int32_t* __restrict__ shi, const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                          const int4* __restrict__ sbb, const unsigned long long* __restrict__ srep,
                          int32_t* __restrict__ srepn, int64_t* __restrict__ flag) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int32_t lo = seg[p];
    int64_t f = 0;
    if (shi[lo] > lo) {
        const int32_t v = ord[p];
        const int4 b = sbb[lo];
        const bool by_x = (int64_t)b.y - b.x >= (int64_t)b.w - b.z;
        const int64_t c2 = 2 * (int64_t)(by_x ? X[v] : Y[v]);
        f = c2 < (by_x ? (int64_t)b.x + b.y : (int64_t)b.z + b.w) ? 1 : 0;
        if (left_key(X[v], Y[v]) == srep[lo]) srepn[lo] = v;
    }
    flag[p] = f;
}

// Stable partition of every segment being cut (lower half first) into the
// next level's arrays; each such segment's head writes its tree node (number
// snum[lo]) and the records of its two halves.  rank = exclusive scan of the
// flags (N + 1 entries).  active: halves of two or more points; bad: a cut
// that left one side empty (duplicate points).
__global__ void k_sp_scatter(int64_t N, const int32_t* __restrict__ ord, const int32_t* __restrict__ seg,
                             const int32_t* __restrict__ shi, const int32_t* __restrict__ snum,
                             const int64_t* __restrict__ flag, const int64_t* __restrict__ rank,
                             const int4* __restrict__ sbb, const int32_t* __restrict__ srepn,
                             int32_t* __restrict__ ord2, int32_t* __restrict__ seg2, int32_t* __restrict__ shi2,
                             int32_t* __restrict__ snum2, int32_t* __restrict__ left, int32_t* __restrict__ right,
                             int4* __restrict__ bb, int32_t* __restrict__ repn,
                             unsigned long long* __restrict__ active, unsigned long long* __restrict__ bad) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int32_t lo = seg[p], hi = shi[lo], v = ord[p];
    if (hi <= lo) {  // a single point: it keeps its place
        ord2[p] = v;
        seg2[p] = (int32_t)p;
        shi2[p] = (int32_t)p;
        return;
    }
    const int64_t r0 = rank[lo];
    const int32_t cL = (int32_t)(rank[(int64_t)hi + 1] - r0), n = hi - lo + 1;
    if (cL == 0 || cL == n) {
        if (p == lo) atomicAdd(bad, 1ull);
        ord2[p] = v;
        seg2[p] = lo;
        if (p == lo) shi2[lo] = lo;  // stop cutting it
        return;
    }
    const int32_t lr = (int32_t)(rank[p] - r0);
    int32_t np, nlo;
    if (flag[p]) {
        np = lo + lr;
        nlo = lo;
    } else {
        np = lo + cL + ((int32_t)(p - lo) - lr);
        nlo = lo + cL;
    }
    ord2[np] = v;
    seg2[np] = nlo;
    if (p == lo) {
        const int32_t w = snum[lo], rlo = lo + cL;
        left[w] = cL == 1 ? ~lo : rlo - 1;
        right[w] = n - cL == 1 ? ~rlo : rlo;
        bb[w] = sbb[lo];
        repn[w] = srepn[lo];
        shi2[lo] = rlo - 1;
        snum2[lo] = rlo - 1;
        shi2[rlo] = hi;
        snum2[rlo] = rlo;
        if (cL >= 2) atomicAdd(active, 1ull);
        if (n - cL >= 2) atomicAdd(active, 1ull);
    }
}

// Leaf order -> positions: nodes gathered into their leaf position, the
// representatives renamed from node indices to positions.
__global__ void k_sp_gather(int64_t N, const int32_t* __restrict__ ord, const int32_t* __restrict__ X,
                            const int32_t* __restrict__ Y, const int64_t* __restrict__ cA,
                            const int64_t* __restrict__ cB, const uint64_t* __restrict__ code, int32_t* __restrict__ X2,
                            int32_t* __restrict__ Y2, int64_t* __restrict__ cA2, int64_t* __restrict__ cB2,
                            uint64_t* __restrict__ code2, int32_t* __restrict__ pos) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int32_t v = ord[p];
    X2[p] = X[v];
    Y2[p] = Y[v];
    cA2[p] = cA[v];
    cB2[p] = cB[v];
    code2[p] = code[v];
    pos[v] = (int32_t)p;
}

__global__ void k_sp_rep_pos(int64_t M, const int32_t* __restrict__ repn, const int32_t* __restrict__ pos,
                             int32_t* __restrict__ rep) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < M) rep[w] = pos[repn[w]];
}

pd_status stage_split_tree(Ctx* c, pd_nodes* nodes, WsTree* tree, int32_t** perm_out, cudaStream_t st) {
    const int64_t N = nodes->n_nodes;
    if (N >= (int64_t(1) << 31) - 4) return fail(c, PD_ECAPACITY, "more than 2^31 - 4 condensed nodes");
    const int64_t M = N > 1 ? N - 1 : 1;
    int32_t* ord[2] = {bufT<int32_t>(c, B_SP_ORD, N), bufT<int32_t>(c, B_SP_ORD2, N)};
    int32_t* seg[2] = {bufT<int32_t>(c, B_SP_SEG, N), bufT<int32_t>(c, B_SP_SEG2, N)};
    int32_t* shi[2] = {bufT<int32_t>(c, B_SP_HI, N), bufT<int32_t>(c, B_SP_HI2, N)};
    int32_t* snum[2] = {bufT<int32_t>(c, B_SP_NUM, N), bufT<int32_t>(c, B_SP_NUM2, N)};
    int4* sbb = bufT<int4>(c, B_SP_BB, N);
    unsigned long long* srep = bufT<unsigned long long>(c, B_SP_REPK, N);
    int32_t* srepn = bufT<int32_t>(c, B_SP_REPN, N);
    int64_t* flag = bufT<int64_t>(c, B_SP_FLAG, N);
    int64_t* rank = bufT<int64_t>(c, B_SP_RANK, N + 1);
    int32_t* left = bufT<int32_t>(c, B_T_LEFT, M);
    int32_t* right = bufT<int32_t>(c, B_T_RIGHT, M);
    int4* bb = bufT<int4>(c, B_T_BB, M);
    int32_t* rep = bufT<int32_t>(c, B_T_REP, M);
    int32_t* repn = bufT<int32_t>(c, B_T_VISIT, M);
    int32_t* X2 = bufT<int32_t>(c, B_SP_X, N);
    int32_t* Y2 = bufT<int32_t>(c, B_SP_Y, N);
    int64_t* cA2 = bufT<int64_t>(c, B_SP_CA, N);
    int64_t* cB2 = bufT<int64_t>(c, B_SP_CB, N);
    uint64_t* code2 = bufT<uint64_t>(c, B_SP_CODE, N);
    int32_t* pos = bufT<int32_t>(c, B_SP_POS, N);
    unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
    for (int q = 0; q < 2; q++)
        if (!ord[q] || !seg[q] || !shi[q] || !snum[q]) return PD_ENOMEM;
    if (!sbb || !srep || !srepn || !flag || !rank || !left || !right || !bb || !rep || !repn || !X2 || !Y2 ||
        !cA2 || !cB2 || !code2 || !pos || !sm)
        return PD_ENOMEM;
    if (N > 0) {
        k_sp_init<<<grid_for(N, 256), 256, 0, st>>>(N, ord[0], seg[0], shi[0], snum[0]);
        pd::count_launch();
    }
    int cur = 0;
    int64_t active = N >= 2 ? 1 : 0;
    for (int level = 0; active > 0; level++) {
        if (level >= 200) return fail(c, PD_EINVAL, "split tree deeper than 200 levels (duplicate points?)");
        const int nx = cur ^ 1;
        PD_TRY_CUDA(c, cudaMemsetAsync(sm + 14, 0, 2 * sizeof(unsigned long long), st));
        k_sp_reset<<<grid_for(N, 256), 256, 0, st>>>(N, seg[cur], shi[cur], sbb, srep);
        pd::count_launch();
        k_sp_box<<<grid_for(N, 256), 256, 0, st>>>(N, ord[cur], seg[cur], shi[cur], nodes->X, nodes->Y, sbb, srep);
        pd::count_launch();
        k_sp_flag<<<grid_for(N, 256), 256, 0, st>>>(N, ord[cur], seg[cur], shi[cur], nodes->X, nodes->Y, sbb, srep,
                                                     srepn, flag);
        pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY(scan_i64(c, flag, rank, N, rank + N, st));
        k_sp_scatter<<<grid_for(N, 256), 256, 0, st>>>(N, ord[cur], seg[cur], shi[cur], snum[cur], flag, rank, sbb,
                                                        srepn, ord[nx], seg[nx], shi[nx], snum[nx], left, right, bb,
                                                        repn, sm + 14, sm + 15);
        pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small + 14, sm + 14, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        if (c->h_small[15]) return fail(c, PD_EINVAL, "split tree: a cut left one side empty (duplicate points)");
        active = c->h_small[14];
        cur = nx;
    }
    if (N > 0) {
        k_sp_gather<<<grid_for(N, 256), 256, 0, st>>>(N, ord[cur], nodes->X, nodes->Y, nodes->cntA, nodes->cntB,
                                                       nodes->morton, X2, Y2, cA2, cB2, code2, pos);
        pd::count_launch();
    }
    if (N > 1) {
        k_sp_rep_pos<<<grid_for(N - 1, 256), 256, 0, st>>>(N - 1, repn, pos, rep);
        pd::count_launch();
    }
    PD_TRY_CUDA(c, cudaGetLastError());
    *nodes = pd_nodes{N, X2, Y2, cA2, cB2, code2};
    *tree = WsTree{N, X2, Y2, left, right, bb, rep};
    if (perm_out) *perm_out = ord[cur];
    return PD_OK;
}

}  // namespace pd
