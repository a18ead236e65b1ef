// Autotuner of the network simplex's launch parameters (no counterpart in the
// paper, whose block search uses a block of sqrt(arcs)): the pricing block,
// which trades pricing work per pivot against the quality of the entering
// arc, and the walk limit, below which the two half-cycles of a pivot are
// followed by two lanes instead of scanned by the whole CTA.  The best values
// depend on the instance's size and on the GPU, so they are measured: the
// transportation instances of sample pairs are solved once per candidate
// (block, walk), each launch timed by CUDA events, and the fastest is kept per
// size class (floor(log2(arcs + nodes))) in the context -- every later solve
// of that class whose pd_opts.ns_block is 0 (ns_walk -1) uses it -- and in an
// optional cache file, one line per (GPU name, SM count, class):
// "name sms class block walk".
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "netsimplex.cuh"

using namespace pd;

namespace {

const int64_t kBlocks[] = {4096, 8192, 16384, 32768};
const int32_t kWalks[] = {0, 8, 32};
constexpr int kDefaultWalk = 0;
struct Choice {
    int64_t block;
    int32_t walk;
};

std::string device_key(int device, int sms) {
    cudaDeviceProp p;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&p, device) == cudaSuccess) name = p.name;
    else cudaGetLastError();
    for (char& ch : name)
        if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
    return name + " " + std::to_string(sms);
}

// Lines "name sms class block walk" of the cache file that match this GPU.
std::map<int, Choice> read_cache(const char* path, const std::string& key) {
    std::map<int, Choice> m;
    FILE* f = path ? fopen(path, "r") : nullptr;
    if (!f) return m;
    char name[256];
    int sms = 0, cls = 0, walk = 0;
    long long blk = 0;
    while (fscanf(f, "%255s %d %d %lld %d", name, &sms, &cls, &blk, &walk) == 5)
        if (std::string(name) + " " + std::to_string(sms) == key && blk > 0 && walk >= 0)
            m[cls] = Choice{(int64_t)blk, walk};
    fclose(f);
    return m;
}

bool write_cache(const char* path, const std::string& key, const std::map<int, Choice>& mine) {
    // keep other GPUs' lines, replace this GPU's
    std::vector<std::string> keep;
    if (FILE* f = fopen(path, "r")) {
        char name[256];
        int sms = 0, cls = 0, walk = 0;
        long long blk = 0;
        while (fscanf(f, "%255s %d %d %lld %d", name, &sms, &cls, &blk, &walk) == 5) {
            const std::string k = std::string(name) + " " + std::to_string(sms);
            if (k != key)
                keep.push_back(k + " " + std::to_string(cls) + " " + std::to_string(blk) + " " + std::to_string(walk));
        }
        fclose(f);
    }
    FILE* f = fopen(path, "w");
    if (!f) return false;
    for (auto& l : keep) fprintf(f, "%s\n", l.c_str());
    for (auto& e : mine) fprintf(f, "%s %d %lld %d\n", key.c_str(), e.first, (long long)e.second.block, e.second.walk);
    return fclose(f) == 0;
}

}  // namespace

namespace pd {

int tune_class(int64_t M) { return M > 0 ? (int)floor(log2((double)M)) : 0; }

int64_t tuned_block(const Ctx* c, int64_t M) {
    const Ctx* o = c->parent ? c->parent : c;
    auto it = o->tuned_block.find(tune_class(M));
    return it == o->tuned_block.end() ? 0 : it->second;
}

int32_t tuned_walk(const Ctx* c, int64_t M) {
    const Ctx* o = c->parent ? c->parent : c;
    auto it = o->tuned_walk.find(tune_class(M));
    return it == o->tuned_walk.end() ? kDefaultWalk : it->second;
}

}  // namespace pd

extern "C" pd_status pd_autotune(pd_ctx* cx, const pd_diagram* A, const pd_diagram* B, int64_t count, double eps,
                                 const pd_opts* opts, const char* cache_path, pd_tune_result* out, void* stream) {
    Ctx* c = cx;
    if (!c || !out || count < 0 || (count > 0 && (!A || !B))) return PD_EINVAL;
    c->err.clear();
    pd_opts o;
    pd_opts_default(&o);
    if (opts) o = *opts;
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    if (o.solver == 1) return fail(c, PD_EINVAL, "the tuner times the network simplex");
    o.warm_start = 0;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    pd_tune_result r;
    memset(&r, 0, sizeof(r));
    r.size_class = -1;
    const std::string key = device_key(c->device, c->sm_count);
    const std::map<int, Choice> cached = read_cache(cache_path, key);
    NSInst* d = bufT<NSInst>(c, B_NS_INST, 1);
    if (!d) return PD_ENOMEM;
    const int NB = (int)(sizeof(kBlocks) / sizeof(kBlocks[0])), NW = (int)(sizeof(kWalks) / sizeof(kWalks[0]));
    // per size class: total device time of every candidate over the pairs timed
    std::map<int, std::vector<double>> total;
    std::map<int, double> dflt;
    for (int64_t i = 0; i < count; i++) {
        Front f;
        PD_TRY(front_half(c, A[i], B[i], eps, o, &f, st, true));
        W1Prep w;
        PD_TRY(ns_prepare_w1(c, f.nodes, f.net.n_arcs, f.h.FB - f.h.FA, o, &w, st));
        if (!w.ns.ready) continue;
        const int64_t M = w.ns.h.m + w.ns.h.n;
        const int cls = tune_class(M);
        if (r.size_class < 0) r.size_class = cls;
        if (cached.count(cls)) {
            c->tuned_block[cls] = cached.at(cls).block;
            c->tuned_walk[cls] = cached.at(cls).walk;
            continue;
        }
        std::vector<double>& t = total[cls];
        t.resize((size_t)(NB * NW), 0.0);
        int64_t opt = -1;
        for (int q = 0; q <= NB * NW; q++) {  // the candidates, then the defaults
            NSInst h = w.ns.h;
            if (q < NB * NW) {
                h.block = kBlocks[q / NW];
                h.walk = kWalks[q % NW];
                if (h.block > 4 * M) continue;
            } else {
                h.block = std::max<int64_t>(8 * NS_THREADS, (int64_t)sqrt((double)M));
                h.walk = kDefaultWalk;
            }
            NSInst res{};
            c->last_ns_ms = 0.f;
            PD_TRY(ns_run(c, &h, 1, w.ns.smem, d, &res, st));
            PD_TRY(ns_status(c, res));
            if (opt >= 0 && res.opt != opt) return fail(c, PD_ECUDA, "tuner: the optimum changed with the parameters");
            opt = res.opt;
            if (q < NB * NW) t[(size_t)q] += c->last_ns_ms;
            else dflt[cls] += c->last_ns_ms;
        }
        r.pairs++;
    }
    std::map<int, Choice> mine = cached;
    for (auto& e : total) {
        size_t best = 0;
        for (size_t q = 1; q < e.second.size(); q++)
            if (e.second[q] > 0.0 && (e.second[best] <= 0.0 || e.second[q] < e.second[best])) best = q;
        const Choice ch{kBlocks[best / NW], kWalks[best % NW]};
        c->tuned_block[e.first] = ch.block;
        c->tuned_walk[e.first] = ch.walk;
        mine[e.first] = ch;
        if (e.first == r.size_class) {
            r.best_ms = (float)e.second[best];
            r.default_ms = (float)dflt[e.first];
        }
    }
    r.candidates = NB * NW;
    r.from_cache = (r.size_class >= 0 && total.count(r.size_class) == 0) ? 1 : 0;
    if (r.size_class >= 0 && c->tuned_block.count(r.size_class)) {
        r.ns_block = c->tuned_block[r.size_class];
        r.ns_walk = c->tuned_walk[r.size_class];
    }
    if (cache_path && !total.empty() && !write_cache(cache_path, key, mine))
        return fail(c, PD_EINVAL, std::string("cannot write the tuning cache ") + cache_path);
    *out = r;
    return PD_OK;
}

extern "C" pd_status pd_tuned_block(const pd_ctx* cx, int64_t arcs_and_nodes, int64_t* block_out) {
    if (!cx || !block_out) return PD_EINVAL;
    *block_out = tuned_block(cx, arcs_and_nodes);
    return PD_OK;
}
