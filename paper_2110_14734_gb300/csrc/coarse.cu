// Potentials for a warm start from a coarse solve of the same pair (no
// counterpart in the paper).  The optimal potentials of the transportation
// form are, up to a constant, the values of one 1-Lipschitz function at the
// nodes (Kantorovich duality of W1 with the diagonal as a point), so a solve
// of the pair condensed onto a coarser lattice (Algorithm 2's snapping with a
// cell of G_c >= 2 G) gives that function at the coarse nodes, and the fine
// nodes take the c-transforms of the coarse optimum (k_ctransform_potential);
// the error per node is of the order of the coarse cell.  The coarse problem
// has a few thousand nodes at most (G_c >= the node box / warm_cells, 64 by
// default), so its simplex is short; its buffers belong to a helper context, so the fine instance, its
// nodes and its WSPD tree stay in place.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "mlp.cuh"
#include "netsimplex.cuh"
#include "prims.cuh"

namespace pd {

constexpr int64_t COARSE_CELLS = 64;  // default coarse cells along the node box's longer side

__global__ void k_node_box(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t n,
                           int* __restrict__ box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicMin(&box[0], X[i]);
    atomicMax(&box[1], X[i]);
    atomicMin(&box[2], Y[i]);
    atomicMax(&box[3], Y[i]);
}

// Fine potentials from the coarse optimum by its c-transforms: the largest
// potential the coarse sinks allow a node at the fine position, min over
// coarse sinks w of pi(w) + c(u, w), and the smallest the coarse sources
// allow, max over coarse sources w of pi(w) - c(w, u), with c the
// transportation cost min(l2, c_make(u) + c_make(w)) and the coarse diagonal
// node among the coarse sinks (sources) when it is one; the fine node takes
// the midpoint of the two envelopes (the Lipschitz potential lies between
// them).  Unlike copying the nearest coarse node's potential, this respects
// the dual constraints of every coarse node, whatever offsets the coarse
// tree's components carry.  The fine diagonal node takes the coarse diagonal
// node's potential.  gap: half the distance between the envelopes (0 where
// one of them is missing), a feature of the learned correction.  cpi: the
// coarse instance's potentials (its sources, sinks, diagonal node); dsup:
// supply of the diagonal node (|B| - |A|).
__global__ void k_ctransform_potential(const int32_t* __restrict__ S, const int32_t* __restrict__ T, int64_t nS,
                                       int64_t nT, const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                                       const int32_t* __restrict__ cS, const int32_t* __restrict__ cT, int64_t cnS,
                                       int64_t cnT, const int32_t* __restrict__ cX, const int32_t* __restrict__ cY,
                                       const int64_t* __restrict__ cpi, int64_t dsup, DiagCost dc,
                                       double* __restrict__ p, double* __restrict__ gap) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > nS + nT) return;
    const int64_t D = cnS + cnT;  // the coarse diagonal node
    if (v == nS + nT) {
        p[v] = (double)cpi[D];
        gap[v] = 0.0;
        return;
    }
    const bool src = v < nS;
    const int32_t u = src ? S[v] : T[v - nS];
    const int32_t x = X[u], y = Y[u];
    const int64_t du = cost_make(x, y, dc);
    // upper envelope over the coarse sinks, lower envelope over the coarse sources
    int64_t up = INT64_MAX, lo = INT64_MIN;
    for (int64_t q = 0; q < cnS + cnT; q++) {
        const int32_t w = q < cnS ? cS[q] : cT[q - cnS];
        const int64_t l2 = cost_l2(x, y, cX[w], cY[w]);
        const int64_t g = du + cost_make(cX[w], cY[w], dc);
        const int64_t c = l2 < g ? l2 : g;
        if (q >= cnS) {
            const int64_t t = cpi[q] + c;
            up = t < up ? t : up;
        } else {
            const int64_t t = cpi[q] - c;
            lo = t > lo ? t : lo;
        }
    }
    // the diagonal node's arcs: sources -> D when D demands (dsup < 0), D -> sinks when it supplies
    if (dsup < 0) up = min(up, cpi[D] + du);
    if (dsup > 0) lo = max(lo, cpi[D] - du);
    double best, half = 0.0;
    if (up == INT64_MAX && lo == INT64_MIN) best = (double)cpi[D];
    else if (up == INT64_MAX) best = (double)lo;
    else if (lo == INT64_MIN) best = (double)up;
    else {
        best = 0.5 * ((double)up + (double)lo);
        half = 0.5 * ((double)up - (double)lo);
    }
    p[v] = best;
    gap[v] = half;
}

static Ctx* coarse_ctx(Ctx* c) {
    if (!c->coarse) {
        c->coarse = ctx_new(c->device, c->cap);
        if (c->coarse) {
            c->coarse->parent = c->parent ? c->parent : c;
            c->coarse->defer_free = c->defer_free;
        }
    }
    return c->coarse;
}

pd_status ws_coarse_potentials(Ctx* c, const Front& f, const W1Prep& w, const pd_opts& o, std::vector<double>* p,
                               cudaStream_t st) {
    p->clear();
    c->last_coarse_cell = 0;
    if (o.warm_cells < 0 || o.warm_cells > 4096) return fail(c, PD_EINVAL, "warm_cells must be 0 .. 4096");
    if (!w.ns.ready || f.nodes.n_nodes == 0) return PD_OK;
    const int64_t cells = o.warm_cells > 0 ? o.warm_cells : COARSE_CELLS;
    int* box = bufT<int>(c, B_CO_BOX, 4);
    if (!box) return PD_ENOMEM;
    const int init[4] = {INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN};
    memcpy(c->h_small + 28, init, sizeof(init));
    PD_TRY_CUDA(c, cudaMemcpyAsync(box, c->h_small + 28, sizeof(init), cudaMemcpyHostToDevice, st));
    k_node_box<<<grid_for(f.nodes.n_nodes, 256), 256, 0, st>>>(f.nodes.X, f.nodes.Y, f.nodes.n_nodes, box);
    pd::count_launch();
    int hb[4];
    PD_TRY_CUDA(c, cudaMemcpyAsync(hb, box, sizeof(hb), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    const int64_t side = std::max<int64_t>((int64_t)hb[1] - hb[0], (int64_t)hb[3] - hb[2]);
    const int64_t Gc = std::min<int64_t>(int64_t(1) << 28,
                                         std::max<int64_t>(2 * f.G, (side + cells - 1) / cells));
    Ctx* cc = coarse_ctx(c);
    if (!cc) return fail(c, PD_ENOMEM, "cannot create the coarse solve's context");
    cc->err.clear();
    pd_nodes cn;
    pd_status e = stage_condense_delta(cc, f.h, Gc, 0, 0, &cn, st);
    pd_opts oc = o;
    oc.warm_start = 0;
    oc.ns_block = 0;
    W1Prep wc;
    if (e == PD_OK) e = ns_prepare_w1(cc, cn, int64_t(1) << 40, f.h.FB - f.h.FA, oc, &wc, st);
    if (e != PD_OK) return fail(c, e, "coarse solve: " + cc->err);
    if (!wc.ns.ready) return PD_OK;  // nothing to solve at the coarse level: start cold
    NSInst* d = bufT<NSInst>(cc, B_NS_INST, 1);
    if (!d) return fail(c, PD_ENOMEM, "coarse solve: " + cc->err);
    NSInst r{};
    e = ns_run(cc, &wc.ns.h, 1, wc.ns.smem, d, &r, st);
    if (e == PD_OK) e = ns_status(cc, r);
    if (e != PD_OK) return fail(c, e, "coarse solve: " + cc->err);
    const int64_t nt = w.nt;
    double* dp = bufT<double>(c, B_CO_P, nt);
    double* dg = bufT<double>(c, B_CO_GAP, nt);
    if (!dp || !dg) return PD_ENOMEM;
    k_ctransform_potential<<<grid_for(nt, 128), 128, 0, st>>>(w.S, w.T, w.nS, w.nT, f.nodes.X, f.nodes.Y, wc.S,
                                                               wc.T, wc.nS, wc.nT, cn.X, cn.Y, r.pi,
                                                               f.h.FB - f.h.FA, w.dc, dp, dg);
    pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    p->resize((size_t)nt);
    PD_TRY_CUDA(c, cudaMemcpyAsync(p->data(), dp, sizeof(double) * nt, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    c->last_coarse_pivots = r.pivots;
    c->last_coarse_cell = Gc;
    return PD_OK;
}

}  // namespace pd
