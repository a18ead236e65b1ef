// C ABI entry points (include/pdw1.h): context, buffers, and the pipeline of
// Algorithm 4 on one stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <atomic>
#include <chrono>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "mlp.cuh"
#include "netsimplex.cuh"
#include "prims.cuh"

using namespace pd;


namespace pd {

long long& launch_count_ref() {
    static thread_local long long n = 0;
    return n;
}

static std::atomic<long long> g_launches{0};
void count_launch_total() { g_launches.fetch_add(1, std::memory_order_relaxed); }

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
    // growth slack: an eighth, or a half where a grow would be deferred
    size_t want = bytes + (c->defer_free ? bytes / 2 : bytes / 8);
    if (c->cap && c->held + c->retired_bytes - c->bytes[id] + want > c->cap) {
        want = bytes;
        if (c->held + c->retired_bytes - c->bytes[id] + want > c->cap) {
            c->err = "device memory cap of the context reached";
            return nullptr;
        }
    }
    if (c->ptr[id]) {
        if (c->defer_free) {
            // cudaFree waits for the whole device: a context that works beside
            // other threads' kernels keeps the old block until ctx_release
            c->retired.push_back(c->ptr[id]);
            c->retired_bytes += c->bytes[id];
        } else {
            cudaFree(c->ptr[id]);
        }
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

int64_t s_for_eps(double eps) {
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

namespace pd {
int default_shift(int dtype) { return dtype == PD_U8 ? 12 : 20; }
}  // namespace pd

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
    o->nn_prune = 1;
    o->warm_start = -1;
    o->ns_walk = -1;
    o->diag_kappa = 1;
    o->diag_tau = 0;
    o->warm_cells = 0;
    o->nn_wave0 = 0;
}

namespace pd {

static bool ctx_init(Ctx* c, int device, size_t cap) {
    c->device = device;
    c->cap = cap;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_small, 64 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

Ctx* ctx_new(int device, size_t cap) {
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return nullptr;
    if (!ctx_init(c, device, cap)) {
        ctx_free(c);
        return nullptr;
    }
    return c;
}

static void wave_free(Ctx* c) {
    if (c->wave_exec) cudaGraphExecDestroy(c->wave_exec);
    if (c->wave_stream) cudaStreamDestroy(c->wave_stream);
    for (cudaEvent_t& e : c->wave_ev)
        if (e) cudaEventDestroy(e);
    if (c->wave_pin) cudaFreeHost(c->wave_pin);
    c->wave_exec = nullptr;
    c->wave_stream = nullptr;
    c->wave_pin = nullptr;
}

// Frees the blocks a deferring context retired (and its helpers' ones).
void ctx_release(Ctx* c) {
    if (!c) return;
    for (void* p : c->retired) cudaFree(p);
    c->retired.clear();
    c->retired_bytes = 0;
    ctx_release(c->coarse);
}

void ctx_free(Ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    ctx_release(c);
    wave_free(c);
    ctx_free(c->coarse);
    c->coarse = nullptr;
    for (Ctx* sl : c->slots) ctx_free(sl);
    c->slots.clear();
    for (Ctx* wk : c->workers) ctx_free(wk);
    c->workers.clear();
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    for (int i = 0; i < B_COUNT; i++)
        if (c->ptr[i]) cudaFree(c->ptr[i]);
    if (c->h_small) cudaFreeHost(c->h_small);
    c->h_small = nullptr;
    delete c;
}

}  // namespace pd

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
    if (!ctx_init(c, device, arena_bytes)) {
        if (c->h_small) cudaFreeHost(c->h_small);
        delete c;
        return PD_ECUDA;
    }
    *out = c;
    return PD_OK;
}

extern "C" void pd_destroy(pd_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    wave_free(c);
    ctx_free(c->coarse);
    c->coarse = nullptr;
    for (Ctx* sl : c->slots) ctx_free(sl);
    c->slots.clear();
    for (Ctx* wk : c->workers) ctx_free(wk);
    c->workers.clear();
    for (int i = 0; i < B_COUNT; i++)
        if (c->ptr[i]) cudaFree(c->ptr[i]);
    if (c->h_small) cudaFreeHost(c->h_small);
    delete c;
}

extern "C" const char* pd_last_error(const pd_ctx* c) { return c ? c->err.c_str() : "no context"; }

extern "C" int64_t pd_kernel_launches(void) { return g_launches.load(); }

pd_status pd::check_diag_cost(Ctx* c, const pd_opts& o) {
    if ((o.diag_kappa != 0 && o.diag_kappa != 1) || o.diag_tau < 0 || o.diag_tau >= (int64_t(1) << 30))
        return fail(c, PD_EINVAL, "need diag_kappa in {0, 1} and 0 <= diag_tau < 2^30");
    return PD_OK;
}

pd_status pd::check_diag(Ctx* c, const pd_diagram& d) {
    if (d.n < 0) return fail(c, PD_EINVAL, "negative diagram size");
    if (d.n > 0 && !d.bd) return fail(c, PD_EINVAL, "NULL diagram data");
    if (d.dtype != PD_F32 && d.dtype != PD_U8) return fail(c, PD_EINVAL, "unknown dtype");
    if (d.n >= (int64_t(1) << 31)) return fail(c, PD_ECAPACITY, "more than 2^31 - 1 points in a diagram");
    if (d.n > 0 && !d.on_host && ((uintptr_t)d.bd % (d.dtype == PD_F32 ? 8 : 2)) != 0)
        return fail(c, PD_EINVAL, "device diagram pointer not aligned to one (b, d) pair");
    return PD_OK;
}

pd_status pd::stage_inputs(Ctx* c, const pd_diagram& A, const pd_diagram& B, DevDiag* a, DevDiag* b,
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
    PD_TRY(check_diag_cost(c, o));
    PD_TRY(stage_rwmd(c, h, L, diag_cost(o), st));
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

extern "C" pd_status pd_wspd_sparsify_tree(pd_ctx* c, const pd_nodes* nodes, int32_t s, int32_t tree,
                                           pd_nodes* ordered_out, pd_network* out, void* stream) {
    if (!c || !nodes || !out) return PD_EINVAL;
    c->err.clear();
    if (tree != 0 && tree != 1) return fail(c, PD_EINVAL, "tree must be 0 (radix tree) or 1 (split tree)");
    if (nodes->n_nodes < 0 || (nodes->n_nodes > 0 && (!nodes->X || !nodes->Y || !nodes->cntA || !nodes->cntB ||
                                                      !nodes->morton)))
        return fail(c, PD_EINVAL, "bad pd_nodes");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    PD_TRY(validate_nodes(c, *nodes, st));
    pd_nodes nd = *nodes;
    WsTree split{};
    if (tree == 1) PD_TRY(stage_split_tree(c, &nd, &split, nullptr, st));
    pd_network net;
    PD_TRY(stage_network(c, nd, s, &net, nullptr, nullptr, nullptr, st, false, nullptr, tree == 1 ? &split : nullptr));
    c->net = net;
    *out = net;
    if (ordered_out) *ordered_out = nd;
    return PD_OK;
}

extern "C" pd_status pd_wspd_count(pd_ctx* c, const pd_nodes* nodes, int32_t s, int32_t tree, int64_t* n_arcs_out,
                                   void* stream) {
    if (!c || !nodes || !n_arcs_out) return PD_EINVAL;
    c->err.clear();
    if (tree != 0 && tree != 1) return fail(c, PD_EINVAL, "tree must be 0 (radix tree) or 1 (split tree)");
    if (nodes->n_nodes < 0 || (nodes->n_nodes > 0 && (!nodes->X || !nodes->Y || !nodes->cntA || !nodes->cntB ||
                                                      !nodes->morton)))
        return fail(c, PD_EINVAL, "bad pd_nodes");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    PD_TRY(validate_nodes(c, *nodes, st));
    pd_nodes nd = *nodes;
    WsTree split{};
    if (tree == 1) PD_TRY(stage_split_tree(c, &nd, &split, nullptr, st));
    pd_network net;
    PD_TRY(stage_network(c, nd, s, &net, nullptr, nullptr, nullptr, st, true, nullptr, tree == 1 ? &split : nullptr));
    *n_arcs_out = net.n_arcs;
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

namespace pd {

pd_status front_half(Ctx* c, const pd_diagram& A, const pd_diagram& B, double eps, const pd_opts& o, Front* f,
                     cudaStream_t st, bool count_only) {
    cudaEvent_t ev[4];
    for (int q = 0; q < 4; q++) PD_TRY_CUDA(c, cudaEventCreate(&ev[q]));
    struct Guard {
        cudaEvent_t* e;
        ~Guard() {
            for (int q = 0; q < 4; q++) cudaEventDestroy(e[q]);
        }
    } guard{ev};
    PD_TRY(check_diag_cost(c, o));
    PD_TRY_CUDA(c, cudaEventRecord(ev[0], st));
    DevDiag a, b;
    PD_TRY(stage_inputs(c, A, B, &a, &b, st));
    f->k = o.coord_shift >= 0 ? o.coord_shift : default_shift(A.dtype);
    PD_TRY(stage_condense0(c, a, b, f->k, &f->h, st));
    PD_TRY_CUDA(c, cudaEventRecord(ev[1], st));
    PD_TRY(stage_rwmd(c, f->h, f->L, diag_cost(o), st));
    PD_TRY_CUDA(c, cudaEventRecord(ev[2], st));
    f->s = o.s_override > 0 ? o.s_override : s_for_eps(eps);
    if (f->s < 1) return fail(c, PD_EINVAL, "no WSPD parameter s for this eps");
    f->delta = 0.0;
    f->G = 1;
    f->P = 0;
    if (o.condense) delta_for(f->L[0], f->L[1], f->h.FA, f->h.FB, f->s, &f->delta, &f->G, &f->P);
    if (!o.perturb) f->P = 0;
    PD_TRY(stage_condense_delta(c, f->h, f->G, f->P, o.seed, &f->nodes, st));
    PD_TRY_CUDA(c, cudaEventRecord(ev[3], st));
    WsTree split{};
    if (o.tree == 1) PD_TRY(stage_split_tree(c, &f->nodes, &split, nullptr, st));  // nodes renumbered by leaf order
    c->nodes = f->nodes;
    PD_TRY(stage_network(c, f->nodes, f->s, &f->net, &f->ms[3], &f->ms[4], &f->ms[5], st, count_only, &f->tree,
                         o.tree == 1 ? &split : nullptr, diag_cost(o)));
    f->counted = count_only;
    c->net = f->net;
    if (count_only) {
        PD_TRY_CUDA(c, cudaEventSynchronize(ev[3]));
        cudaEventElapsedTime(&f->ms[0], ev[0], ev[1]);
        cudaEventElapsedTime(&f->ms[1], ev[1], ev[2]);
        cudaEventElapsedTime(&f->ms[2], ev[2], ev[3]);
        return PD_OK;
    }
    // The solver sees ā and b̄ merged into one diagonal node (the zero-cost
    // arc b̄ -> ā contracted): every flow of the paper's network maps to one of
    // the same cost, and an optimal acyclic flow of the merged network sends at
    // most |A| units into and |B| units out of the diagonal, so it maps back.
    PD_TRY(merge_diagonal(c, f->net, f->nodes.n_nodes, &f->mnet, st));
    PD_TRY_CUDA(c, cudaEventSynchronize(ev[3]));
    cudaEventElapsedTime(&f->ms[0], ev[0], ev[1]);
    cudaEventElapsedTime(&f->ms[1], ev[1], ev[2]);
    cudaEventElapsedTime(&f->ms[2], ev[2], ev[3]);
    return PD_OK;
}

}  // namespace pd

static void fill_result(const Front& f, const SolveStats& ss, pd_result* out) {
    pd_result r;
    memset(&r, 0, sizeof(r));
    r.opt_quanta = ss.opt;
    r.w1 = ldexp((double)ss.opt, -f.k);
    r.rwmd_A = f.L[0];
    r.rwmd_B = f.L[1];
    r.rwmd_quanta = f.L[2];
    r.slack_quanta = ss.slack;
    r.mass_A = f.h.FA;
    r.mass_B = f.h.FB;
    r.s = (int32_t)f.s;
    r.coord_shift = f.k;
    r.delta = f.delta;
    r.cell_quanta = f.G;
    r.shift_quanta = f.P;
    r.n_nodes = f.nodes.n_nodes;
    r.n_arcs = f.net.n_arcs;
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
    for (int q = 0; q < 6; q++) r.stage_ms[q] = f.ms[q];
    *out = r;
}

// The warm start's greedy takes all arcs between the still unbalanced nodes
// at once when there are at most this many (before that, rounds of top-k).
constexpr int64_t WARM_MAX_RESIDUAL = int64_t(1) << 18;
// warm_start -1: transportation instances of at least this many nodes start
// from the coarse solve (below it the cold start is about as fast)
constexpr int64_t WARM_AUTO_NODES = 4096;

static float elapsed_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// What a warm start cost (pd_result.warm_ms, warm_pivots).
struct WarmStats {
    float ms[2] = {0.f, 0.f};  // potentials, start tree (host wall time)
    int64_t coarse_pivots = 0;
};

// Warm start of a prepared transportation instance (opts.warm_start): the
// potentials from a coarse solve (4), corrected by the network (1), from the
// exact potentials of a cold solve (2) or from the distances to the diagonal
// (3), then the start tree.  `c` does the work; the instance's buffers
// belong to `tc` (the same context on the one-pair path, the pair's slot in a
// batch).  *used: the start tree was installed.
static pd_status warm_start(Ctx* c, Ctx* tc, const Front& f, W1Prep* w, const pd_opts& oi, bool* used,
                            WarmStats* ws, cudaStream_t st) {
    *used = false;
    if (!w->ns.ready || oi.warm_start == 0) return PD_OK;
    pd_opts o = oi;
    if (o.warm_start == -1) {  // automatic: the coarse solve's start for large instances
        if (w->nt < WARM_AUTO_NODES) return PD_OK;
        o.warm_start = 4;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<float> pf;
    std::vector<double> p;
    c->last_coarse_pivots = 0;
    if (o.warm_start == 1) {  // the coarse solve's potentials corrected by the network
        PD_TRY(ws_coarse_potentials(c, f, *w, o, &p, st));
        PD_TRY(ws_predict(c, f.nodes, *w, &pf, st));
        if (!p.empty())
            for (size_t v = 0; v < p.size() && v < pf.size(); v++) p[v] += pf[v];
    } else if (o.warm_start == 2) {
        NSInst* d = bufT<NSInst>(c, B_NS_INST, 1);
        if (!d) return PD_ENOMEM;
        NSInst r{};
        PD_TRY(ns_run(c, &w->ns.h, 1, w->ns.smem, d, &r, st));
        PD_TRY(ns_status(c, r));
        const int64_t nt = w->nt;
        std::vector<int64_t> pi((size_t)nt);
        PD_TRY_CUDA(c, cudaMemcpyAsync(pi.data(), r.pi, sizeof(int64_t) * nt, cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        p.resize((size_t)nt);
        for (int64_t v = 0; v < nt; v++) p[(size_t)v] = (double)(pi[(size_t)v] - pi[(size_t)(nt - 1)]);
    } else if (o.warm_start == 3) {
        PD_TRY(ws_diag_potentials(c, f.nodes, *w, &pf, st));  // the greedy ranks arcs by their saving
    } else if (o.warm_start == 4) {
        PD_TRY(ws_coarse_potentials(c, f, *w, o, &p, st));
        if (p.empty()) return PD_OK;  // nothing to solve at the coarse level: cold start
    } else {
        return fail(c, PD_EINVAL, "warm_start must be -1 .. 4");
    }
    if (p.empty()) p.assign(pf.begin(), pf.end());
    ws->coarse_pivots = c->last_coarse_pivots;
    ws->ms[0] = elapsed_ms(t0);
    const auto t1 = std::chrono::steady_clock::now();
    PD_TRY(ns_warm_tree(tc, &w->ns, p.data(), WARM_MAX_RESIDUAL, used, st));
    ws->ms[1] = elapsed_ms(t1);
    return PD_OK;
}

extern "C" pd_status pd_w1_approx(pd_ctx* c, pd_diagram A, pd_diagram B, double eps, const pd_opts* opts,
                                  pd_result* out, void* stream) {
    if (!c || !out) return PD_EINVAL;
    c->err.clear();
    pd_opts o = resolve_opts(opts);
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    if (o.tree != 0 && o.tree != 1) return fail(c, PD_EINVAL, "tree must be 0 (radix tree) or 1 (split tree)");
    c->last_ns_ms = 0.f;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const long long launches0 = launch_count_ref();
    const auto t0 = std::chrono::steady_clock::now();
    Front f;
    bool warm_used = false;
    WarmStats wst;
    const bool transport = o.solver != 1 && o.ns_transport != 0;
    PD_TRY(front_half(c, A, B, eps, o, &f, st, transport));
    const auto t1 = std::chrono::steady_clock::now();
    SolveStats ss;
    if (o.solver == 1) {
        PD_TRY(stage_solve(c, f.mnet, o, &ss, st));
    } else {
        W1Prep w;
        if (transport) PD_TRY(ns_prepare_w1(c, f.nodes, f.net.n_arcs, f.h.FB - f.h.FA, o, &w, st));
        if (w.ns.ready) {
            bool used = false;
            PD_TRY(warm_start(c, c, f, &w, o, &used, &wst, st));
            warm_used = used;
            NSInst* d = bufT<NSInst>(c, B_NS_INST, 1);
            if (!d) return PD_ENOMEM;
            NSInst r{};
            if (o.warm_start == 2) c->last_ns_ms = 0.f;  // report the warm solve only
            PD_TRY(ns_run(c, &w.ns.h, 1, w.ns.smem, d, &r, st));
            PD_TRY(ns_finish_w1(c, f.tree, f.s, nullptr, o, w, d, r, &ss, st));
        }
        if (!w.ns.ready || ss.method == -1) {
            // the sparse network itself: build it (the nodes are still in place) and solve it
            const SolveStats first = ss;
            pd_network mnet = f.mnet;
            if (f.counted) {
                // on the same tree: with the split tree the nodes are in its leaf order, not Morton order
                pd_network net;
                const WsTree given = f.tree;
                PD_TRY(stage_network(c, f.nodes, f.s, &net, nullptr, nullptr, nullptr, st, false, nullptr,
                                     o.tree == 1 ? &given : nullptr, diag_cost(o)));
                PD_TRY(merge_diagonal(c, net, f.nodes.n_nodes, &mnet, st));
            }
            PD_TRY(ns_solve_network(c, mnet, o, &ss, st));
            ss.pivots += first.pivots;
            ss.degenerate += first.degenerate;
            ss.scanned += first.scanned;
            ss.cert_failures = first.cert_failures;
        }
    }
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    fill_result(f, ss, out);
    out->stage_ms[6] = elapsed_ms(t1);
    out->stage_ms[7] = elapsed_ms(t0);
    out->kernel_launches = launch_count_ref() - launches0;
    out->ns_kernel_ms = c->last_ns_ms;
    out->warm_used = warm_used ? 1 : 0;
    out->warm_ms[0] = wst.ms[0];
    out->warm_ms[1] = wst.ms[1];
    out->warm_pivots = wst.coarse_pivots;
    return PD_OK;
}

extern "C" pd_status pd_w1_sparsify_count(pd_ctx* c, pd_diagram A, pd_diagram B, double eps, const pd_opts* opts,
                                          pd_result* out, void* stream) {
    if (!c || !out) return PD_EINVAL;
    c->err.clear();
    pd_opts o = resolve_opts(opts);
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    if (o.tree != 0 && o.tree != 1) return fail(c, PD_EINVAL, "tree must be 0 (radix tree) or 1 (split tree)");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const long long launches0 = launch_count_ref();
    const auto t0 = std::chrono::steady_clock::now();
    Front f;
    PD_TRY(front_half(c, A, B, eps, o, &f, st, true));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    fill_result(f, SolveStats{}, out);
    out->solve_method = -1;
    out->stage_ms[7] = elapsed_ms(t0);
    out->kernel_launches = launch_count_ref() - launches0;
    return PD_OK;
}

// A pair of a batch between its preprocessing and its certificate: the
// transportation instance lives in the pair's slot, with copies of what the
// certificate reads (node coordinates, sparse network rows and heads).
struct BatchPair {
    Front f;
    W1Prep w;
    WsTree tree{};      // slot copies of the node coordinates and the WSPD tree
    bool done = false;  // solved during preprocessing (no transportation form)
    bool warm = false;  // starts from a warm-start tree
    WarmStats wst;
    SolveStats ss;
    float front_ms = 0.f, solve_ms = 0.f;
    long long launches = 0;
    int inst = -1;      // index in the wave's launch
};

// What the certificate reads, copied from the worker into the pair's slot:
// node coordinates and the WSPD tree (about 36 bytes per node).
static pd_status persist_for_certificate(Ctx* slot, const Front& f, BatchPair* bp, cudaStream_t st) {
    const int64_t N = f.nodes.n_nodes, M = N > 1 ? N - 1 : 1;
    int32_t* X = bufT<int32_t>(slot, B_NX, N);
    int32_t* Y = bufT<int32_t>(slot, B_NY, N);
    int32_t* l = bufT<int32_t>(slot, B_T_LEFT, M);
    int32_t* r = bufT<int32_t>(slot, B_T_RIGHT, M);
    int4* bb = bufT<int4>(slot, B_T_BB, M);
    int32_t* rep = bufT<int32_t>(slot, B_T_REP, M);
    if (!X || !Y || !l || !r || !bb || !rep) return PD_ENOMEM;
    if (N > 0) {
        PD_TRY_CUDA(slot, cudaMemcpyAsync(X, f.nodes.X, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
        PD_TRY_CUDA(slot, cudaMemcpyAsync(Y, f.nodes.Y, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
    }
    if (N > 1) {
        PD_TRY_CUDA(slot, cudaMemcpyAsync(l, f.tree.left, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
        PD_TRY_CUDA(slot, cudaMemcpyAsync(r, f.tree.right, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
        PD_TRY_CUDA(slot, cudaMemcpyAsync(bb, f.tree.bb, sizeof(int4) * M, cudaMemcpyDeviceToDevice, st));
        PD_TRY_CUDA(slot, cudaMemcpyAsync(rep, f.tree.rep, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, st));
    }
    bp->tree = WsTree{N, X, Y, l, r, bb, rep};
    return PD_OK;
}

// The sparse network of a pair, built in full and solved (no transportation
// form, or its certificate failed).
static pd_status solve_sparse(Ctx* c, const pd_diagram& A, const pd_diagram& B, double eps, const pd_opts& o,
                              SolveStats* ss, cudaStream_t st) {
    Front f;
    PD_TRY(front_half(c, A, B, eps, o, &f, st, false));
    PD_TRY(ns_solve_network(c, f.mnet, o, ss, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    return PD_OK;
}

// Preprocessing of one pair on a worker context: front half, then the
// transportation instance in the pair's slot (or, without one, the solve of
// the sparse network right here).
static pd_status batch_prepare(Ctx* work, Ctx* slot, const pd_diagram& A, const pd_diagram& B, double eps,
                               const pd_opts& o, BatchPair* bp) {
    cudaStream_t st = work->own_stream;
    const long long l0 = launch_count_ref();
    const auto t0 = std::chrono::steady_clock::now();
    work->last_ns_ms = 0.f;
    slot->last_ns_ms = 0.f;
    const bool transport = o.ns_transport != 0;
    PD_TRY(front_half(work, A, B, eps, o, &bp->f, st, transport));
    if (transport)
        PD_TRY(ns_prepare_w1(slot, bp->f.nodes, bp->f.net.n_arcs, bp->f.h.FB - bp->f.h.FA, o, &bp->w, st));
    if (bp->w.ns.ready) {
        if (o.warm_start != 0 && o.warm_start != 1 && o.warm_start != 4 && o.warm_start != -1)
            return fail(work, PD_EINVAL, "the batched solve takes warm_start -1, 0, 1 or 4");
        PD_TRY(warm_start(work, slot, bp->f, &bp->w, o, &bp->warm, &bp->wst, st));
        PD_TRY(persist_for_certificate(slot, bp->f, bp, st));
    } else {
        const auto t1 = std::chrono::steady_clock::now();
        PD_TRY(solve_sparse(work, A, B, eps, o, &bp->ss, st));
        bp->solve_ms = elapsed_ms(t1);
        bp->done = true;
    }
    PD_TRY_CUDA(work, cudaStreamSynchronize(st));
    bp->front_ms = elapsed_ms(t0) - bp->solve_ms;
    bp->launches = launch_count_ref() - l0;
    if (bp->done) slot->last_ns_ms = work->last_ns_ms;
    return PD_OK;
}

extern "C" pd_status pd_w1_approx_batch(pd_ctx* c, const pd_diagram* A, const pd_diagram* B, int64_t count,
                                        double eps, const pd_opts* opts, pd_result* out, void* stream) {
    if (!c) return PD_EINVAL;
    c->err.clear();
    if (count < 0 || (count > 0 && (!A || !B || !out))) return fail(c, PD_EINVAL, "bad batch arguments");
    if (count == 0) return PD_OK;
    pd_opts o = resolve_opts(opts);
    // automatic warm start: cold here -- with a wave of pairs per launch the
    // per-pair coarse solves and start trees on the host cost more than the
    // pivots they save
    if (o.warm_start == -1) o.warm_start = 0;
    return pd::batch_solve(c, A, B, count, eps, o, out, (cudaStream_t)stream);
}

namespace pd {

pd_status batch_solve(Ctx* c, const pd_diagram* A, const pd_diagram* B, int64_t count, double eps,
                      const pd_opts& o, pd_result* out, cudaStream_t st) {
    if (count <= 0) return PD_OK;
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    if (o.solver == 1) return fail(c, PD_EINVAL, "the batched solve runs the network simplex only");
    if (o.batch_slots < 0 || o.batch_threads < 0) return fail(c, PD_EINVAL, "batch_slots and batch_threads must be >= 0");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    const int64_t W = std::min<int64_t>(count, o.batch_slots > 0 ? o.batch_slots : 2 * std::max(c->sm_count, 1));
    const int nthr = (int)std::min<int64_t>(W, o.batch_threads > 0 ? o.batch_threads : 8);
    while ((int64_t)c->slots.size() < W) {
        Ctx* sl = ctx_new(c->device, c->cap);
        if (!sl) return fail(c, PD_ECUDA, "cannot create the buffers of a batch slot");
        sl->parent = c;
        sl->defer_free = true;
        c->slots.push_back(sl);
    }
    while ((int)c->workers.size() < nthr) {
        Ctx* wk = ctx_new(c->device, c->cap);
        if (!wk) return fail(c, PD_ECUDA, "cannot create a batch worker");
        if (cudaStreamCreateWithFlags(&wk->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ctx_free(wk);
            return fail(c, PD_ECUDA, "cannot create a batch worker stream");
        }
        wk->parent = c;
        wk->defer_free = true;
        c->workers.push_back(wk);
    }
    for (Ctx* wk : c->workers) wk->mlp_owner = c;  // predictions use this context's network
    if (o.warm_start == 1 && !c->mlp_ready) return fail(c, PD_EINVAL, "warm_start = 1 needs a trained network");
    // the workers start after everything already queued on the caller's stream
    cudaEvent_t ready;
    PD_TRY_CUDA(c, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    std::vector<BatchPair> bp((size_t)W);
    std::vector<NSInst> hin, hout;
    std::vector<CertJob> jobs;
    std::vector<unsigned long long> cert;
    pd_status status = PD_OK;
    for (int64_t base = 0; base < count && status == PD_OK; base += W) {
        const int64_t nw = std::min<int64_t>(W, count - base);
        for (int64_t j = 0; j < nw; j++) bp[(size_t)j] = BatchPair{};
        // ---- preprocessing: host threads, one worker context and stream each
        cudaEventRecord(ready, st);
        std::atomic<int64_t> next{0};
        std::mutex mu;
        pd_status first = PD_OK;
        std::string first_msg;
        auto run = [&](int t) {
            Ctx* wk = c->workers[(size_t)t];
            cudaSetDevice(c->device);
            cudaStreamWaitEvent(wk->own_stream, ready, 0);
            for (;;) {
                const int64_t j = next.fetch_add(1);
                if (j >= nw) break;
                {
                    std::lock_guard<std::mutex> g(mu);
                    if (first != PD_OK) break;
                }
                Ctx* sl = c->slots[(size_t)j];
                wk->err.clear();
                sl->err.clear();
                pd_status e = batch_prepare(wk, sl, A[base + j], B[base + j], eps, o, &bp[(size_t)j]);
                if (e != PD_OK) {
                    std::lock_guard<std::mutex> g(mu);
                    if (first == PD_OK) {
                        first = e;
                        first_msg = "pair " + std::to_string(base + j) + ": " + (wk->err.empty() ? sl->err : wk->err);
                    }
                    break;
                }
            }
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nthr; t++) th.emplace_back(run, t);
        run(0);
        for (auto& x : th) x.join();
        if (first != PD_OK) {
            status = fail(c, first, first_msg);
            break;
        }
        // ---- the wave as one CUDA graph: records up, one persistent simplex
        // launch (one CTA per SM takes the pairs, largest first), every pair's
        // certificate in one launch, records and certificate counts down
        hin.clear();
        jobs.clear();
        size_t smem = 0;
        for (int64_t j = 0; j < nw; j++) {
            BatchPair& p = bp[(size_t)j];
            if (p.done) continue;
            p.inst = (int)hin.size();
            hin.push_back(p.w.ns.h);
            CertJob J{};
            J.rec = p.inst;
            J.S = p.w.S;
            J.T = p.w.T;
            J.nS = p.w.nS;
            J.nT = p.w.nT;
            J.s = p.f.s;
            J.tree = p.tree;
            J.dc = diag_cost(o);
            jobs.push_back(J);
            smem = std::max(smem, p.w.ns.smem);
        }
        hout.assign(hin.size(), NSInst{});
        cert.assign(2 * hin.size(), 0ull);
        c->last_ns_ms = 0.f;
        const auto tl = std::chrono::steady_clock::now();
        const long long lw = launch_count_ref();
        if (!hin.empty()) {
            status = ns_run_wave(c, hin.data(), (int)hin.size(), smem, jobs.data(), hout.data(), cert.data(), st);
            if (status != PD_OK) break;
        }
        const float wave_ms = elapsed_ms(tl), wave_ns = c->last_ns_ms;
        const long long wave_launches = launch_count_ref() - lw;
        // ---- results; a pair whose certificate failed is preprocessed again
        // and solved on its sparse network
        for (int64_t j = 0; j < nw && status == PD_OK; j++) {
            BatchPair& p = bp[(size_t)j];
            Ctx* sl = c->slots[(size_t)j];
            sl->last_ns_ms = 0.f;
            if (!p.done) {
                const long long l0 = launch_count_ref();
                const auto t0 = std::chrono::steady_clock::now();
                const NSInst& r = hout[(size_t)p.inst];
                status = ns_status(sl, r);
                if (status != PD_OK) {
                    status = fail(c, status, "pair " + std::to_string(base + j) + ": " + sl->err);
                    break;
                }
                p.ss = SolveStats{};
                p.ss.pivots = r.pivots;
                p.ss.degenerate = r.degenerate;
                p.ss.scanned = r.scanned;
                if (cert[2 * (size_t)p.inst] == 0) {
                    p.ss.opt = r.opt;
                    p.ss.slack = (int64_t)cert[2 * (size_t)p.inst + 1];
                    p.ss.verified = 1;
                    p.ss.method = 2;
                } else {
                    Ctx* wk = c->workers[0];
                    const SolveStats first_try = p.ss;
                    wk->last_ns_ms = 0.f;
                    status = solve_sparse(wk, A[base + j], B[base + j], eps, o, &p.ss, wk->own_stream);
                    if (status != PD_OK) {
                        status = fail(c, status, "pair " + std::to_string(base + j) + ": " + wk->err);
                        break;
                    }
                    p.ss.pivots += first_try.pivots;
                    p.ss.degenerate += first_try.degenerate;
                    p.ss.scanned += first_try.scanned;
                    p.ss.cert_failures = (int64_t)cert[2 * (size_t)p.inst];
                    sl->last_ns_ms += wk->last_ns_ms;
                }
                p.solve_ms = wave_ms + elapsed_ms(t0);
                p.launches += wave_launches + (launch_count_ref() - l0);
            }
            pd_result& res = out[base + j];
            fill_result(p.f, p.ss, &res);
            res.stage_ms[6] = p.solve_ms;
            res.stage_ms[7] = p.front_ms + p.solve_ms;
            res.kernel_launches = p.launches;
            res.ns_kernel_ms = (p.done ? 0.f : wave_ns) + sl->last_ns_ms;
            res.warm_used = p.warm ? 1 : 0;
            res.warm_ms[0] = p.wst.ms[0];
            res.warm_ms[1] = p.wst.ms[1];
            res.warm_pivots = p.wst.coarse_pivots;
        }
    }
    cudaEventDestroy(ready);
    // the blocks the slots and workers outgrew: freed now that their work is done
    cudaStreamSynchronize(st);
    for (Ctx* sl : c->slots) ctx_release(sl);
    for (Ctx* wk : c->workers) ctx_release(wk);
    return status;
}

}  // namespace pd

extern "C" pd_status pd_ws_train(pd_ctx* c, const pd_diagram* A, const pd_diagram* B, int64_t n_pairs, double eps,
                                 const pd_opts* opts, int32_t epochs, float lr, uint64_t seed, pd_ws_stats* out,
                                 void* stream) {
    if (!c || !out || n_pairs < 0 || (n_pairs > 0 && (!A || !B)) || epochs < 0 || !(lr > 0.f)) return PD_EINVAL;
    c->err.clear();
    pd_opts o = resolve_opts(opts);
    o.warm_start = 0;
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    pd_ws_stats r;
    memset(&r, 0, sizeof(r));
    PD_TRY(mlp_init(c, seed, false, st));
    // the data set: at most one row per point of every pair
    int64_t cap = 0;
    for (int64_t i = 0; i < n_pairs; i++) cap += std::max<int64_t>(A[i].n, 0) + std::max<int64_t>(B[i].n, 0);
    cap = std::max<int64_t>(cap, 1);
    if (!bufT<__nv_bfloat16>(c, B_WS_DF, cap * WS_IN) || !bufT<float>(c, B_WS_DT, cap) ||
        !bufT<float>(c, B_WS_DM, cap))
        return PD_ENOMEM;
    c->ws_cap = cap;
    c->ws_rows = 0;
    // the last eighth of the pairs (at least one, with four or more pairs)
    // is held out: its rows pick the epoch whose weights are kept
    const int64_t n_val = n_pairs >= 4 ? std::max<int64_t>(1, n_pairs / 8) : 0;
    int64_t r_train = 0;
    const auto t0 = std::chrono::steady_clock::now();
    for (int64_t i = 0; i < n_pairs; i++) {
        if (i == n_pairs - n_val) r_train = c->ws_rows;
        Front f;
        PD_TRY(front_half(c, A[i], B[i], eps, o, &f, st, true));
        W1Prep w;
        PD_TRY(ns_prepare_w1(c, f.nodes, f.net.n_arcs, f.h.FB - f.h.FA, o, &w, st));
        if (!w.ns.ready) continue;
        NSInst* d = bufT<NSInst>(c, B_NS_INST, 1);
        if (!d) return PD_ENOMEM;
        // the network learns the correction to the coarse solve's potentials
        std::vector<double> base;
        PD_TRY(ws_coarse_potentials(c, f, w, o, &base, st));
        NSInst rec{};
        PD_TRY(ns_run(c, &w.ns.h, 1, w.ns.smem, d, &rec, st));
        PD_TRY(ns_status(c, rec));
        const int64_t cmax = (rec.big - 1) / (int64_t)(rec.n + 1) - 1;
        PD_TRY(ws_collect(c, f.nodes, w, d, rec, cmax, base.empty() ? nullptr : &base, st));
        r.pairs++;
        r.cold_pivots += rec.pivots;
    }
    if (n_val == 0) r_train = c->ws_rows;
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    r.collect_ms = elapsed_ms(t0);
    r.rows = c->ws_rows;
    r.val_rows = c->ws_rows - r_train;
    r.val_pairs = (int32_t)n_val;
    const auto t1 = std::chrono::steady_clock::now();
    float* g = bufT<float>(c, B_MLP_G, WS_PART);
    int32_t* didx = bufT<int32_t>(c, B_WS_IDX, std::max<int64_t>(r_train, 1));
    if (!g || !didx) return PD_ENOMEM;
    const int64_t R = r_train, bs = 2048;
    // held-out loss of predicting no correction (the coarse start itself)
    if (r.val_rows > 0) {
        std::vector<float> ht((size_t)r.val_rows), hm((size_t)r.val_rows);
        PD_TRY_CUDA(c, cudaMemcpyAsync(ht.data(), (const float*)c->ptr[B_WS_DT] + r_train, sizeof(float) * r.val_rows,
                                       cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaMemcpyAsync(hm.data(), (const float*)c->ptr[B_WS_DM] + r_train, sizeof(float) * r.val_rows,
                                       cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        double ls = 0.0, ms = 0.0;
        for (size_t q = 0; q < ht.size(); q++) {
            ls += (double)hm[q] * (double)ht[q] * (double)ht[q];
            ms += hm[q];
        }
        r.val_loss_zero = (float)(ms > 0.0 ? ls / ms : 0.0);
        double l0 = 0.0;
        PD_TRY(mlp_loss(c, r_train, c->ws_rows, &l0, st));
        r.val_loss = (float)l0;
        PD_TRY(mlp_snapshot(c, false, st));
    }
    std::mt19937_64 rng(seed ^ 0x5DEECE66Dull);
    std::vector<int32_t> perm((size_t)R);
    for (int64_t q = 0; q < R; q++) perm[(size_t)q] = (int32_t)q;
    for (int32_t e = 0; e < epochs && R > 0; e++) {
        std::shuffle(perm.begin(), perm.end(), rng);
        PD_TRY_CUDA(c, cudaMemcpyAsync(didx, perm.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, st));
        for (int64_t r0 = 0; r0 < R; r0 += bs) {
            const int64_t nb = std::min<int64_t>(bs, R - r0);
            __nv_bfloat16* F;
            float *T, *M;
            PD_TRY(mlp_gather_rows(c, didx + r0, nb, &F, &T, &M, st));
            PD_TRY(mlp_grad(c, F, T, M, nb, 1.f / (float)nb, g, st));
            const bool first = r.steps == 0, last = e == epochs - 1 && r0 + bs >= R;
            if (first || last) {
                float lm[2];
                PD_TRY_CUDA(c, cudaMemcpyAsync(lm, g + WS_NPARAMS, sizeof(lm), cudaMemcpyDeviceToHost, st));
                PD_TRY_CUDA(c, cudaStreamSynchronize(st));
                const float l = lm[1] > 0.f ? lm[0] / lm[1] : 0.f;
                if (first) r.loss_first = l;
                if (last) r.loss_last = l;
            }
            PD_TRY(mlp_adam(c, g, lr, st));
            r.steps++;
        }
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));  // perm is rewritten next epoch
        if (r.val_rows > 0) {
            double lv = 0.0;
            PD_TRY(mlp_loss(c, r_train, c->ws_rows, &lv, st));
            if (lv < (double)r.val_loss) {
                r.val_loss = (float)lv;
                r.best_epoch = e + 1;
                PD_TRY(mlp_snapshot(c, false, st));
            }
        }
    }
    if (r.val_rows > 0) PD_TRY(mlp_snapshot(c, true, st));  // the held-out best (epoch 0: no correction)
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    r.train_ms = elapsed_ms(t1);
    *out = r;
    return PD_OK;
}
