// Warm start of the network simplex on the transportation form from
// predicted node potentials (the paper has no counterpart: it always starts
// the solver cold).  Only the starting tree changes; the simplex still runs
// to optimality, so the optimum is the cold start's.
//
// From potentials p (one per transportation node), the reduced costs
// r(i, j) = c(i, j) - p(i) + p(j) rank the arcs.  Every source keeps its
// WS_K best sinks, every sink its WS_K best sources, plus all arcs of the
// diagonal node; a greedy pass over these candidates in ascending r sends
// min(remaining supply, remaining demand) along each arc, and a second greedy
// rounds of the same over the nodes still unbalanced, a greedy pass over all
// their arcs once few are left, and the north-west corner rule over what is
// still unbalanced when the rounds stop making progress finish the flow.
// Each greedy assignment exhausts one end, so the arcs used form a forest;
// each of its trees hangs from the root by the artificial arc of one of its
// supply nodes (flow 0, pointing to the root), which makes the start strongly
// feasible; its cost big + art[r0] places the component's potentials at the
// predicted ones.  Potentials of the start follow from the tree.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mlp.cuh"

namespace pd {

constexpr int WS_K = 8;  // candidate arcs per source and per sink

// Top WS_K reduced costs of each listed source row rs[a] over the listed sink
// columns rt[0..nrt) (one warp per row).  outj: column indices into rt.
__global__ void k_topk_rows(const int32_t* __restrict__ cmat, int64_t nS, int64_t nT, const float* __restrict__ p,
                            const int32_t* __restrict__ rs, int64_t nrs, const int32_t* __restrict__ rt, int64_t nrt,
                            int32_t* __restrict__ outj) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= nrs) return;  // whole warps leave together
    const int64_t row = rs[a];
    float bv[WS_K];
    int32_t bj[WS_K];
#pragma unroll
    for (int q = 0; q < WS_K; q++) {
        bv[q] = INFINITY;
        bj[q] = -1;
    }
    const float pi = p[row];
    for (int64_t b = lane; b < nrt; b += 32) {
        const int32_t j = rt[b];
        float r = (float)cmat[row * nT + j] - pi + p[nS + j];
        if (r < bv[WS_K - 1]) {
            int q = WS_K - 1;
            while (q > 0 && bv[q - 1] > r) {
                bv[q] = bv[q - 1];
                bj[q] = bj[q - 1];
                q--;
            }
            bv[q] = r;
            bj[q] = (int32_t)b;
        }
    }
    // merge the 32 sorted lists: WS_K rounds of a warp arg-min over the heads
    int head = 0;
    for (int k = 0; k < WS_K; k++) {
        float v = INFINITY;
        int32_t jj = INT32_MAX;
#pragma unroll
        for (int q = 0; q < WS_K; q++)
            if (q == head) {
                v = bv[q];
                jj = bj[q] < 0 ? INT32_MAX : bj[q];
            }
        float mv = v;
        int32_t mj = jj;
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, mv, o);
            int32_t oj = __shfl_xor_sync(0xffffffffu, mj, o);
            if (ov < mv || (ov == mv && oj < mj)) {
                mv = ov;
                mj = oj;
            }
        }
        if (lane == 0) outj[a * WS_K + k] = mj == INT32_MAX ? -1 : mj;
        if (jj == mj && mj != INT32_MAX) head++;
    }
}

// Top WS_K reduced costs of each listed sink column rt[b] over the listed
// source rows (one thread per column; the listed columns ascend, so a warp's
// loads of one row are close together).  outi: row indices into rs.
__global__ void k_topk_cols(const int32_t* __restrict__ cmat, int64_t nS, int64_t nT, const float* __restrict__ p,
                            const int32_t* __restrict__ rs, int64_t nrs, const int32_t* __restrict__ rt, int64_t nrt,
                            int32_t* __restrict__ outi) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrt) return;
    const int32_t j = rt[b];
    float bv[WS_K];
    int32_t bi[WS_K];
#pragma unroll
    for (int q = 0; q < WS_K; q++) {
        bv[q] = INFINITY;
        bi[q] = -1;
    }
    const float pj = p[nS + j];
    for (int64_t a = 0; a < nrs; a++) {
        const int32_t i = rs[a];
        float r = (float)cmat[(int64_t)i * nT + j] - p[i] + pj;
        if (r < bv[WS_K - 1]) {
            int q = WS_K - 1;
            while (q > 0 && bv[q - 1] > r) {
                bv[q] = bv[q - 1];
                bi[q] = bi[q - 1];
                q--;
            }
            bv[q] = r;
            bi[q] = (int32_t)a;
        }
    }
#pragma unroll
    for (int q = 0; q < WS_K; q++) outi[b * WS_K + q] = bi[q];
}

// Reduced costs of the arcs between residual sources rs and residual sinks rt.
__global__ void k_residual_costs(const int32_t* __restrict__ cmat, int64_t nS, int64_t nT,
                                 const int32_t* __restrict__ rs, int64_t ns, const int32_t* __restrict__ rt, int64_t nt,
                                 int32_t* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * nt) return;
    const int64_t a = t / nt, b = t - a * nt;
    out[t] = cmat[(int64_t)rs[a] * nT + rt[b]];
}

// Costs of given implicit arcs.
__global__ void k_gather_costs(const int32_t* __restrict__ cmat, const int64_t* __restrict__ arcs, int64_t n,
                               int32_t* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = cmat[arcs[t]];
}

namespace {

struct Arc {
    int32_t t, h;  // transportation node ids
    int64_t id;    // arc id of the instance
    int32_t f;     // flow
};

}  // namespace

pd_status ns_warm_tree(Ctx* c, NSPrep* prep, const double* p, int64_t max_residual, bool* used, cudaStream_t st) {
    *used = false;
    NSInst& h = prep->h;
    if (!prep->ready) return PD_OK;
    const int64_t nS = h.nS, nT = h.nT, mst = h.mst, m = h.m, nt = h.n, N1 = nt + 1;
    if (mst != nS * nT || nt != nS + nT + 1) return PD_OK;  // not a transportation instance
    const int64_t mx = m - mst;
    // supplies and the diagonal node's arcs
    std::vector<int64_t> sup((size_t)nt);
    std::vector<int32_t> xt((size_t)std::max<int64_t>(mx, 1)), xh((size_t)std::max<int64_t>(mx, 1)),
        xc((size_t)std::max<int64_t>(mx, 1));
    PD_TRY_CUDA(c, cudaMemcpyAsync(sup.data(), h.supply, sizeof(int64_t) * nt, cudaMemcpyDeviceToHost, st));
    if (mx > 0) {
        PD_TRY_CUDA(c, cudaMemcpyAsync(xt.data(), h.tail, sizeof(int32_t) * mx, cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaMemcpyAsync(xh.data(), h.head, sizeof(int32_t) * mx, cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaMemcpyAsync(xc.data(), h.cost, sizeof(int32_t) * mx, cudaMemcpyDeviceToHost, st));
    }
    std::vector<int64_t> rem((size_t)nt);
    for (int64_t v = 0; v < nt; v++) rem[(size_t)v] = sup[(size_t)v] < 0 ? -sup[(size_t)v] : sup[(size_t)v];
    std::vector<Arc> used_arcs;
    std::vector<int64_t> arc_cost_used;
    auto take = [&](int64_t a, int32_t t, int32_t hh, int64_t cost) -> bool {
        if (sup[(size_t)t] < 0 || sup[(size_t)hh] > 0) return false;  // arcs run from supply to demand
        const int64_t f = std::min(rem[(size_t)t], rem[(size_t)hh]);
        if (f <= 0) return false;
        rem[(size_t)t] -= f;
        rem[(size_t)hh] -= f;
        used_arcs.push_back(Arc{t, hh, a, (int32_t)f});
        arc_cost_used.push_back(cost);
        return true;
    };
    float* dp = bufT<float>(c, B_WS_P, nt);
    if (!dp) return PD_ENOMEM;
    std::vector<float> pf((size_t)nt);
    for (int64_t v = 0; v < nt; v++) pf[(size_t)v] = (float)p[v];  // the device top-k ranks in float
    PD_TRY_CUDA(c, cudaMemcpyAsync(dp, pf.data(), sizeof(float) * nt, cudaMemcpyHostToDevice, st));
    // rounds over the still unbalanced sources x sinks: each source keeps its
    // WS_K best sinks and each sink its WS_K best sources (device), then a
    // greedy pass over these candidates in ascending reduced cost (host); when
    // few pairs are left, one greedy pass over all of them
    std::vector<int32_t> rs, rt, hr, hc;
    std::vector<int64_t> cand;
    std::vector<int32_t> cc;
    std::vector<std::pair<double, int64_t>> order;
    int64_t last_left = INT64_MAX;
    auto residual_lists = [&]() {
        rs.clear();
        rt.clear();
        for (int64_t i = 0; i < nS; i++)
            if (rem[(size_t)i] > 0) rs.push_back((int32_t)i);
        for (int64_t j = 0; j < nT; j++)
            if (rem[(size_t)(nS + j)] > 0) rt.push_back((int32_t)j);
    };
    for (int round = 0; round < 16; round++) {
        residual_lists();
        const int64_t nrs = (int64_t)rs.size(), nrt = (int64_t)rt.size();
        if (nrs == 0 || nrt == 0) break;
        if (nrs + nrt > last_left - last_left / 10) break;  // under 10 % progress: finish below
        last_left = nrs + nrt;
        const bool full = nrs * nrt <= max_residual;
        int32_t* drs = bufT<int32_t>(c, B_WS_RS, nrs);
        int32_t* drt = bufT<int32_t>(c, B_WS_RT, nrt);
        if (!drs || !drt) return PD_ENOMEM;
        PD_TRY_CUDA(c, cudaMemcpyAsync(drs, rs.data(), sizeof(int32_t) * nrs, cudaMemcpyHostToDevice, st));
        PD_TRY_CUDA(c, cudaMemcpyAsync(drt, rt.data(), sizeof(int32_t) * nrt, cudaMemcpyHostToDevice, st));
        cand.clear();
        if (full) {
            int32_t* dcost = bufT<int32_t>(c, B_WS_RC, nrs * nrt);
            if (!dcost) return PD_ENOMEM;
            k_residual_costs<<<grid_for(nrs * nrt, 256), 256, 0, st>>>(h.cmat, nS, nT, drs, nrs, drt, nrt, dcost); pd::count_launch();
            PD_TRY_CUDA(c, cudaGetLastError());
            cc.resize((size_t)(nrs * nrt));
            PD_TRY_CUDA(c, cudaMemcpyAsync(cc.data(), dcost, sizeof(int32_t) * nrs * nrt, cudaMemcpyDeviceToHost, st));
            PD_TRY_CUDA(c, cudaStreamSynchronize(st));
            for (int64_t a = 0; a < nrs; a++)
                for (int64_t b = 0; b < nrt; b++) cand.push_back((int64_t)rs[(size_t)a] * nT + rt[(size_t)b]);
        } else {
            int32_t* rj = bufT<int32_t>(c, B_WS_ROWK, nrs * WS_K);
            int32_t* ci = bufT<int32_t>(c, B_WS_COLK, nrt * WS_K);
            if (!rj || !ci) return PD_ENOMEM;
            k_topk_rows<<<grid_for(nrs * 32, 256), 256, 0, st>>>(h.cmat, nS, nT, dp, drs, nrs, drt, nrt, rj); pd::count_launch();
            k_topk_cols<<<grid_for(nrt, 128), 128, 0, st>>>(h.cmat, nS, nT, dp, drs, nrs, drt, nrt, ci); pd::count_launch();
            PD_TRY_CUDA(c, cudaGetLastError());
            hr.resize((size_t)(nrs * WS_K));
            hc.resize((size_t)(nrt * WS_K));
            PD_TRY_CUDA(c, cudaMemcpyAsync(hr.data(), rj, sizeof(int32_t) * nrs * WS_K, cudaMemcpyDeviceToHost, st));
            PD_TRY_CUDA(c, cudaMemcpyAsync(hc.data(), ci, sizeof(int32_t) * nrt * WS_K, cudaMemcpyDeviceToHost, st));
            PD_TRY_CUDA(c, cudaStreamSynchronize(st));
            for (int64_t a = 0; a < nrs; a++)
                for (int q = 0; q < WS_K; q++) {
                    const int32_t b = hr[(size_t)(a * WS_K + q)];
                    if (b >= 0) cand.push_back((int64_t)rs[(size_t)a] * nT + rt[(size_t)b]);
                }
            for (int64_t b = 0; b < nrt; b++)
                for (int q = 0; q < WS_K; q++) {
                    const int32_t a = hc[(size_t)(b * WS_K + q)];
                    if (a >= 0) cand.push_back((int64_t)rs[(size_t)a] * nT + rt[(size_t)b]);
                }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            // their costs
            const int64_t nc = (int64_t)cand.size();
            int64_t* da = bufT<int64_t>(c, B_WS_ARCS, std::max<int64_t>(nc, 1));
            int32_t* dc = bufT<int32_t>(c, B_WS_COST, std::max<int64_t>(nc, 1));
            if (!da || !dc) return PD_ENOMEM;
            cc.resize((size_t)std::max<int64_t>(nc, 1));
            PD_TRY_CUDA(c, cudaMemcpyAsync(da, cand.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, st));
            k_gather_costs<<<grid_for(nc, 256), 256, 0, st>>>(h.cmat, da, nc, dc); pd::count_launch();
            PD_TRY_CUDA(c, cudaGetLastError());
            PD_TRY_CUDA(c, cudaMemcpyAsync(cc.data(), dc, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, st));
            PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        }
        order.resize(cand.size());
        for (size_t q = 0; q < cand.size(); q++) {
            const int64_t a = cand[q];
            const int32_t t = (int32_t)(a / nT), hh = (int32_t)(nS + a % nT);
            order[q] = {(double)cc[q] - p[t] + p[hh], (int64_t)q};
        }
        std::sort(order.begin(), order.end());
        bool moved = false;
        for (auto& o : order) {
            const int64_t a = cand[(size_t)o.second];
            moved |= take(a, (int32_t)(a / nT), (int32_t)(nS + a % nT), cc[(size_t)o.second]);
        }
        if (full || !moved) break;
    }
    // whatever is still unbalanced: north-west corner over the residual lists
    // (each step exhausts a source or a sink, so the forest stays a forest)
    residual_lists();
    if (!rs.empty() && !rt.empty()) {
        std::vector<int64_t> sim(rem);
        cand.clear();
        size_t a = 0, b = 0;
        while (a < rs.size() && b < rt.size()) {
            const int32_t i = rs[a], j = rt[b];
            const int64_t f = std::min(sim[(size_t)i], sim[(size_t)(nS + j)]);
            cand.push_back((int64_t)i * nT + j);
            sim[(size_t)i] -= f;
            sim[(size_t)(nS + j)] -= f;
            if (sim[(size_t)i] == 0) a++;
            else b++;
        }
        const int64_t nc = (int64_t)cand.size();
        int64_t* da = bufT<int64_t>(c, B_WS_ARCS, std::max<int64_t>(nc, 1));
        int32_t* dc = bufT<int32_t>(c, B_WS_COST, std::max<int64_t>(nc, 1));
        if (!da || !dc) return PD_ENOMEM;
        cc.resize((size_t)std::max<int64_t>(nc, 1));
        PD_TRY_CUDA(c, cudaMemcpyAsync(da, cand.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, st));
        k_gather_costs<<<grid_for(nc, 256), 256, 0, st>>>(h.cmat, da, nc, dc); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        PD_TRY_CUDA(c, cudaMemcpyAsync(cc.data(), dc, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        for (int64_t q = 0; q < nc; q++)
            take(cand[(size_t)q], (int32_t)(cand[(size_t)q] / nT), (int32_t)(nS + cand[(size_t)q] % nT), cc[(size_t)q]);
    }
    // the diagonal node's arcs, in ascending reduced cost, for what is left
    std::vector<std::pair<double, int64_t>> dorder((size_t)mx);
    for (int64_t x = 0; x < mx; x++) dorder[(size_t)x] = {(double)xc[(size_t)x] - p[xt[(size_t)x]] + p[xh[(size_t)x]], x};
    std::sort(dorder.begin(), dorder.end());
    for (auto& o : dorder) {
        const int64_t x = o.second;
        take(mst + x, xt[(size_t)x], xh[(size_t)x], xc[(size_t)x]);
    }
    for (int64_t v = 0; v < nt; v++)
        if (rem[(size_t)v] != 0) return PD_OK;  // not balanced: start cold
    // forest -> tree: every component hangs from the root by one supply node
    std::vector<std::vector<int32_t>> adj((size_t)nt);
    for (size_t e = 0; e < used_arcs.size(); e++) {
        adj[(size_t)used_arcs[e].t].push_back((int32_t)e);
        adj[(size_t)used_arcs[e].h].push_back((int32_t)e);
    }
    std::vector<int64_t> pi((size_t)N1, 0);
    std::vector<int32_t> pred((size_t)N1, -1), parent((size_t)N1, -1), flow((size_t)N1, 0), ord, pos((size_t)N1, 0),
        size((size_t)N1, 1);
    std::vector<uint8_t> up((size_t)N1, 0);
    std::vector<uint8_t> seen((size_t)nt, 0);
    const int64_t big = h.big;
    ord.reserve((size_t)N1);
    ord.push_back((int32_t)nt);  // the root
    std::vector<int32_t> stack;
    std::vector<int32_t> comp_order;
    // Every component hangs from the root by the artificial arc of its root
    // node r0, whose cost big + art[r0] sets pi(r0): art[r0] = p(r0) - min p
    // over the component roots keeps the predicted offsets between components
    // (one common big would erase them).  The other supply nodes' artificial
    // arcs cost 2 big - 1, far above their potentials, so they never enter.
    // Every artificial cost is >= big: still a valid big-M start.
    std::vector<int64_t> art((size_t)nt, 0);
    double pmin = INFINITY;
    for (int64_t v = 0; v < nt; v++)
        if (sup[(size_t)v] >= 0 && p[v] < pmin) pmin = p[v];
    auto offset = [&](int64_t v) -> int64_t {
        const double o = p[v] - pmin;
        return o <= 0.0 ? 0 : (o >= (double)(big - 1) ? big - 1 : (int64_t)std::llround(o));
    };
    for (int64_t v = 0; v < nt; v++)
        if (sup[(size_t)v] >= 0) art[(size_t)v] = big - 1;
    for (int pass = 0; pass < 2; pass++) {
        // components are rooted at a supply node (first pass) or, for a node
        // of supply 0 on its own, at that node (second pass)
        for (int64_t r0 = 0; r0 < nt; r0++) {
            if (seen[(size_t)r0] || (pass == 0 && sup[(size_t)r0] <= 0) || (pass == 1 && sup[(size_t)r0] < 0))
                continue;
            seen[(size_t)r0] = 1;
            parent[(size_t)r0] = (int32_t)nt;
            pred[(size_t)r0] = (int32_t)(m + r0);
            up[(size_t)r0] = 1;
            flow[(size_t)r0] = 0;
            art[(size_t)r0] = offset(r0);
            pi[(size_t)r0] = big + art[(size_t)r0];
            stack.assign(1, (int32_t)r0);
            while (!stack.empty()) {  // preorder DFS
                const int32_t v = stack.back();
                stack.pop_back();
                ord.push_back(v);
                for (int32_t e : adj[(size_t)v]) {
                    const Arc& A = used_arcs[(size_t)e];
                    const int32_t w = A.t == v ? A.h : A.t;
                    if (seen[(size_t)w]) continue;
                    seen[(size_t)w] = 1;
                    parent[(size_t)w] = v;
                    pred[(size_t)w] = (int32_t)A.id;
                    flow[(size_t)w] = A.f;
                    const int64_t cst = arc_cost_used[(size_t)e];
                    if (A.t == w) {  // w -> v: the arc points to the parent
                        up[(size_t)w] = 1;
                        pi[(size_t)w] = pi[(size_t)v] + cst;
                    } else {
                        up[(size_t)w] = 0;
                        pi[(size_t)w] = pi[(size_t)v] - cst;
                    }
                    stack.push_back(w);
                }
            }
        }
    }
    if ((int64_t)ord.size() != N1) return PD_OK;  // a node of demand without supply in its component
    for (int64_t x = 0; x < N1; x++) pos[(size_t)ord[(size_t)x]] = (int32_t)x;
    for (int64_t x = N1 - 1; x >= 1; x--) {
        const int32_t v = ord[(size_t)x];
        size[(size_t)parent[(size_t)v]] += size[(size_t)v];
    }
    pi[(size_t)nt] = 0;
    pred[(size_t)nt] = -1;
    parent[(size_t)nt] = -1;
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.pi, pi.data(), sizeof(int64_t) * N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.pred, pred.data(), sizeof(int32_t) * N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.parent, parent.data(), sizeof(int32_t) * N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.flow, flow.data(), sizeof(int32_t) * N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.up, up.data(), N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.ord, ord.data(), sizeof(int32_t) * N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.pos, pos.data(), sizeof(int32_t) * N1, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(h.size, size.data(), sizeof(int32_t) * N1, cudaMemcpyHostToDevice, st));
    int64_t* dart = bufT<int64_t>(c, B_NS_ART, nt);
    if (!dart) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemcpyAsync(dart, art.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    h.art = dart;
    h.init_tree = 1;
    *used = true;
    return PD_OK;
}

}  // namespace pd
