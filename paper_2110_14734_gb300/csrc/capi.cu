// C ABI entry points (include/pdw1.h): context, buffers, and the pipeline of
// Algorithm 4 on one stream.
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "internal.h"
#include "prims.cuh"

using namespace pd;

struct pd_ctx : public pd::Ctx {};

namespace pd {

long long& launch_count_ref() {
    static thread_local long long n = 0;
    return n;
}

__global__ void k_fill_i64(int64_t* p, int64_t n, int64_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

pd_status fail(Ctx* c, pd_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

pd_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") at " + where;
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    return fail(c, e == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA, m);
}

void* buf(Ctx* c, Buf id, size_t bytes) {
    if (bytes == 0) bytes = 1;
    if (c->bytes[id] >= bytes) return c->ptr[id];
    size_t want = bytes + bytes / 8;
    if (c->cap && c->held - c->bytes[id] + want > c->cap) {
        want = bytes;
        if (c->held - c->bytes[id] + want > c->cap) {
            c->err = "device memory cap of the context reached";
            return nullptr;
        }
    }
    if (c->ptr[id]) {
        cudaFree(c->ptr[id]);
        c->held -= c->bytes[id];
        c->ptr[id] = nullptr;
        c->bytes[id] = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("cudaMalloc of ") + std::to_string(want) + " bytes failed";
        return nullptr;
    }
    c->ptr[id] = p;
    c->bytes[id] = want;
    c->held += want;
    return p;
}

pd_status sort_u64(Ctx* c, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n,
                   int bits, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return PD_OK;
    RadixScratch<uint64_t> s;
    s.k_alt = keys_alt;
    s.v_alt = vals_alt;
    int64_t nc = (int64_t)radix_counts_elems<uint64_t>(n);
    s.counts = bufT<int64_t>(c, B_RS_COUNTS, nc);
    s.part = bufT<int64_t>(c, B_RS_PART, scan_tiles(nc) + 1);
    if (!s.counts || !s.part) return PD_ENOMEM;
    PD_TRY_CUDA(c, radix_sort<uint64_t>(keys, vals, n, bits, s, st));
    return PD_OK;
}

pd_status scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, cudaStream_t st) {
    int64_t* part = bufT<int64_t>(c, B_SCAN_PART, scan_tiles(n) + 1);
    if (!part) return PD_ENOMEM;
    PD_TRY_CUDA(c, exclusive_scan<int64_t>(in, out, n, part, total_dev, st));
    return PD_OK;
}

// ---- eps -> s, delta (host; the same double expressions, no FMA contraction)

static double s_bound(int64_t s) {
    double sd = (double)s;
    double a = 1.0 + 4.0 / sd;
    a = a + 4.0 / (sd - 2.0);
    double b = 1.0 + 8.0 / (sd - 4.0);
    return a * b;
}

static int64_t s_for_eps(double eps) {
    if (!(eps > 0.0)) return -1;
    for (int64_t s = 13; s < (int64_t(1) << 40); s++)
        if (s_bound(s) <= 1.0 + eps) return s;
    return -1;
}

static void delta_for(int64_t LA, int64_t LB, int64_t FA, int64_t FB, int64_t s, double* delta, int64_t* G,
                      int64_t* P) {
    int64_t Llo = LA - FA;
    if (LB - FB > Llo) Llo = LB - FB;
    if (Llo < 0) Llo = 0;
    double ec = s >= 12 ? 8.0 / (double)(s - 4) : 1.0;
    double d = 0.0;
    if (FA + FB > 0) {
        double num = 2.0 * ec;
        num = num * (double)Llo;
        double den = sqrt(2.0) * (double)(FA + FB);
        d = num / den;
    }
    const int64_t gmax = int64_t(1) << 28;
    double g = floor(0.99 * d);
    int64_t Gv = g >= (double)gmax ? gmax : (int64_t)g;
    if (Gv < 1) Gv = 1;
    double p = floor(0.005 * d);
    int64_t Pv = p >= (double)gmax ? gmax : (int64_t)p;
    if (2 * Pv >= Gv) Pv = (Gv - 1) / 2;
    *delta = d;
    *G = Gv;
    *P = Pv;
}

}  // namespace pd

// ---------------------------------------------------------------------------

static int default_shift(int dtype) { return dtype == PD_U8 ? 12 : 20; }

extern "C" void pd_opts_default(pd_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->coord_shift = -1;
    o->s_override = 0;
    o->condense = 1;
    o->perturb = 1;
    o->seed = 0;
    o->alpha = 8;
    o->verify = 0;
    o->max_rounds = 0;
    o->time_limit_ms = 0;
    o->update_every = 0;
    o->seq_threshold = -1;
    o->solver = 0;
    o->ns_block = 0;
    o->ns_transport = 1;
    o->ns_smem = 1;
}

extern "C" pd_status pd_create(pd_ctx** out, int device, size_t arena_bytes) {
    if (!out) return PD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PD_EINVAL;
    }
    pd_ctx* c = new (std::nothrow) pd_ctx();
    if (!c) return PD_ENOMEM;
    c->device = device;
    c->cap = arena_bytes;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_small, 64 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PD_ECUDA;
    }
    *out = c;
    return PD_OK;
}

extern "C" void pd_destroy(pd_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    for (int i = 0; i < B_COUNT; i++)
        if (c->ptr[i]) cudaFree(c->ptr[i]);
    if (c->h_small) cudaFreeHost(c->h_small);
    delete c;
}

extern "C" const char* pd_last_error(const pd_ctx* c) { return c ? c->err.c_str() : "no context"; }

static pd_status check_diag(pd_ctx* c, const pd_diagram& d) {
    if (d.n < 0) return fail(c, PD_EINVAL, "negative diagram size");
    if (d.n > 0 && !d.bd) return fail(c, PD_EINVAL, "NULL diagram data");
    if (d.dtype != PD_F32 && d.dtype != PD_U8) return fail(c, PD_EINVAL, "unknown dtype");
    if (d.n >= (int64_t(1) << 31)) return fail(c, PD_ECAPACITY, "more than 2^31 - 1 points in a diagram");
    if (d.n > 0 && !d.on_host && ((uintptr_t)d.bd % (d.dtype == PD_F32 ? 8 : 2)) != 0)
        return fail(c, PD_EINVAL, "device diagram pointer not aligned to one (b, d) pair");
    return PD_OK;
}

static pd_status stage_inputs(pd_ctx* c, const pd_diagram& A, const pd_diagram& B, DevDiag* a, DevDiag* b,
                              cudaStream_t st) {
    PD_TRY(check_diag(c, A));
    PD_TRY(check_diag(c, B));
    const pd_diagram* src[2] = {&A, &B};
    DevDiag* dst[2] = {a, b};
    Buf ids[2] = {B_IN_A, B_IN_B};
    for (int q = 0; q < 2; q++) {
        const pd_diagram& d = *src[q];
        size_t bytes = (size_t)d.n * (d.dtype == PD_F32 ? 8 : 2);
        dst[q]->n = d.n;
        dst[q]->dtype = d.dtype;
        if (d.on_host && d.n > 0) {
            void* p = buf(c, ids[q], bytes);
            if (!p) return PD_ENOMEM;
            PD_TRY_CUDA(c, cudaMemcpyAsync(p, d.bd, bytes, cudaMemcpyHostToDevice, st));
            dst[q]->bd = p;
        } else {
            dst[q]->bd = d.bd;
        }
    }
    return PD_OK;
}

static pd_opts resolve_opts(const pd_opts* o) {
    pd_opts r;
    pd_opts_default(&r);
    if (o) r = *o;
    return r;
}

extern "C" pd_status pd_condense(pd_ctx* c, pd_diagram A, pd_diagram B, int64_t cell_quanta, int64_t shift_quanta,
                                 const pd_opts* opts, pd_nodes* out, void* stream) {
    if (!c || !out) return PD_EINVAL;
    c->err.clear();
    if (cell_quanta < 1 || shift_quanta < 0 || 2 * shift_quanta >= cell_quanta || cell_quanta > (int64_t(1) << 28))
        return fail(c, PD_EINVAL, "need 1 <= cell_quanta <= 2^28 and 0 <= 2 * shift_quanta < cell_quanta");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    pd_opts o = resolve_opts(opts);
    DevDiag a, b;
    PD_TRY(stage_inputs(c, A, B, &a, &b, st));
    int k = o.coord_shift >= 0 ? o.coord_shift : default_shift(A.dtype);
    Hats h;
    PD_TRY(stage_condense0(c, a, b, k, &h, st));
    pd_nodes nodes;
    PD_TRY(stage_condense_delta(c, h, cell_quanta, shift_quanta, o.seed, &nodes, st));
    c->nodes = nodes;
    *out = nodes;
    return PD_OK;
}

extern "C" pd_status pd_rwmd_lower_bound(pd_ctx* c, pd_diagram A, pd_diagram B, const pd_opts* opts, int64_t* out3,
                                         void* stream) {
    if (!c || !out3) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    pd_opts o = resolve_opts(opts);
    DevDiag a, b;
    PD_TRY(stage_inputs(c, A, B, &a, &b, st));
    int k = o.coord_shift >= 0 ? o.coord_shift : default_shift(A.dtype);
    Hats h;
    PD_TRY(stage_condense0(c, a, b, k, &h, st));
    int64_t L[3];
    PD_TRY(stage_rwmd(c, h, L, st));
    out3[0] = L[0];
    out3[1] = L[1];
    out3[2] = L[2];
    return PD_OK;
}

extern "C" pd_status pd_wspd_sparsify(pd_ctx* c, const pd_nodes* nodes, int32_t s, pd_network* out, void* stream) {
    if (!c || !nodes || !out) return PD_EINVAL;
    c->err.clear();
    if (nodes->n_nodes < 0 || (nodes->n_nodes > 0 && (!nodes->X || !nodes->Y || !nodes->cntA || !nodes->cntB ||
                                                      !nodes->morton)))
        return fail(c, PD_EINVAL, "bad pd_nodes");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    PD_TRY(validate_nodes(c, *nodes, (cudaStream_t)stream));
    pd_network net;
    PD_TRY(stage_network(c, *nodes, s, &net, nullptr, nullptr, nullptr, (cudaStream_t)stream));
    c->net = net;
    *out = net;
    return PD_OK;
}

extern "C" pd_status pd_mcf_solve(pd_ctx* c, const pd_network* net, const pd_opts* opts, int64_t* opt_out,
                                  pd_result* stats, void* stream) {
    if (!c || !net || !opt_out) return PD_EINVAL;
    c->err.clear();
    if (net->n_nodes < 0 || net->n_arcs < 0) return fail(c, PD_EINVAL, "bad pd_network");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    pd_opts o = resolve_opts(opts);
    PD_TRY(validate_network(c, *net, (cudaStream_t)stream));
    c->last_ns_ms = 0.f;
    const long long launches0 = launch_count_ref();
    SolveStats ss;
    if (o.solver == 1)
        PD_TRY(stage_solve(c, *net, o, &ss, (cudaStream_t)stream));
    else
        PD_TRY(ns_solve_network(c, *net, o, &ss, (cudaStream_t)stream));
    *opt_out = ss.opt;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->opt_quanta = ss.opt;
        stats->slack_quanta = ss.slack;
        stats->phases = ss.phases;
        stats->rounds = ss.rounds;
        stats->pushes = ss.pushes;
        stats->relabels = ss.relabels;
        stats->repair_passes = ss.repairs;
        stats->price_updates = ss.updates;
        stats->update_passes = ss.update_passes;
        stats->pivots = ss.pivots;
        stats->degenerate = ss.degenerate;
        stats->arcs_priced = ss.scanned;
        stats->solve_method = ss.method;
        stats->cert_failures = (int32_t)ss.cert_failures;
        stats->verified = ss.verified;
        stats->n_nodes = net->n_nodes;
        stats->n_arcs = net->n_arcs;
        stats->kernel_launches = launch_count_ref() - launches0;
        stats->ns_kernel_ms = c->last_ns_ms;
    }
    return PD_OK;
}

extern "C" pd_status pd_w1_approx(pd_ctx* c, pd_diagram A, pd_diagram B, double eps, const pd_opts* opts,
                                  pd_result* out, void* stream) {
    if (!c || !out) return PD_EINVAL;
    c->err.clear();
    pd_opts o = resolve_opts(opts);
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    c->last_ns_ms = 0.f;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    pd_result r;
    memset(&r, 0, sizeof(r));
    const long long launches0 = launch_count_ref();
    cudaEvent_t ev[5];
    for (int q = 0; q < 5; q++) PD_TRY_CUDA(c, cudaEventCreate(&ev[q]));
    PD_TRY_CUDA(c, cudaEventRecord(ev[0], st));
    DevDiag a, b;
    PD_TRY(stage_inputs(c, A, B, &a, &b, st));
    int k = o.coord_shift >= 0 ? o.coord_shift : default_shift(A.dtype);
    Hats h;
    PD_TRY(stage_condense0(c, a, b, k, &h, st));
    PD_TRY_CUDA(c, cudaEventRecord(ev[1], st));
    int64_t L[3];
    PD_TRY(stage_rwmd(c, h, L, st));
    PD_TRY_CUDA(c, cudaEventRecord(ev[2], st));
    int64_t s = o.s_override > 0 ? o.s_override : s_for_eps(eps);
    if (s < 1) return fail(c, PD_EINVAL, "no WSPD parameter s for this eps");
    double delta = 0.0;
    int64_t G = 1, P = 0;
    if (o.condense) delta_for(L[0], L[1], h.FA, h.FB, s, &delta, &G, &P);
    if (!o.perturb) P = 0;
    pd_nodes nodes;
    PD_TRY(stage_condense_delta(c, h, G, P, o.seed, &nodes, st));
    c->nodes = nodes;
    PD_TRY_CUDA(c, cudaEventRecord(ev[3], st));
    pd_network net;
    float mt = 0, mw = 0, mc = 0;
    PD_TRY(stage_network(c, nodes, s, &net, &mt, &mw, &mc, st));
    c->net = net;
    cudaEvent_t e5, e6;
    PD_TRY_CUDA(c, cudaEventCreate(&e5));
    PD_TRY_CUDA(c, cudaEventCreate(&e6));
    PD_TRY_CUDA(c, cudaEventRecord(e5, st));
    // The solver sees ā and b̄ merged into one diagonal node (the zero-cost
    // arc b̄ -> ā contracted): every flow of the paper's network maps to one of
    // the same cost, and an optimal acyclic flow of the merged network sends at
    // most |A| units into and |B| units out of the diagonal, so it maps back.
    pd_network mnet;
    PD_TRY(merge_diagonal(c, net, nodes.n_nodes, &mnet, st));
    SolveStats ss;
    if (o.solver == 1)
        PD_TRY(stage_solve(c, mnet, o, &ss, st));
    else
        PD_TRY(ns_solve_w1(c, nodes, net, mnet, o, &ss, st));
    PD_TRY_CUDA(c, cudaEventRecord(e6, st));
    PD_TRY_CUDA(c, cudaEventSynchronize(e6));
    float ms[4];
    cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
    cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
    cudaEventElapsedTime(&ms[2], ev[2], ev[3]);
    cudaEventElapsedTime(&ms[3], e5, e6);
    float tot = 0;
    cudaEventElapsedTime(&tot, ev[0], e6);
    for (int q = 0; q < 5; q++) cudaEventDestroy(ev[q]);
    cudaEventDestroy(e5);
    cudaEventDestroy(e6);
    r.opt_quanta = ss.opt;
    r.w1 = ldexp((double)ss.opt, -k);
    r.rwmd_A = L[0];
    r.rwmd_B = L[1];
    r.rwmd_quanta = L[2];
    r.slack_quanta = ss.slack;
    r.mass_A = h.FA;
    r.mass_B = h.FB;
    r.s = (int32_t)s;
    r.coord_shift = k;
    r.delta = delta;
    r.cell_quanta = G;
    r.shift_quanta = P;
    r.n_nodes = nodes.n_nodes;
    r.n_arcs = net.n_arcs;
    r.phases = ss.phases;
    r.verified = ss.verified;
    r.rounds = ss.rounds;
    r.pushes = ss.pushes;
    r.relabels = ss.relabels;
    r.repair_passes = ss.repairs;
    r.price_updates = ss.updates;
    r.update_passes = ss.update_passes;
    r.pivots = ss.pivots;
    r.degenerate = ss.degenerate;
    r.arcs_priced = ss.scanned;
    r.solve_method = ss.method;
    r.cert_failures = (int32_t)ss.cert_failures;
    r.stage_ms[0] = ms[0];
    r.stage_ms[1] = ms[1];
    r.stage_ms[2] = ms[2];
    r.stage_ms[3] = mt;
    r.stage_ms[4] = mw;
    r.stage_ms[5] = mc;
    r.stage_ms[6] = ms[3];
    r.stage_ms[7] = tot;
    r.kernel_launches = launch_count_ref() - launches0;
    r.ns_kernel_ms = c->last_ns_ms;
    *out = r;
    return PD_OK;
}
