// Instance record of the single-CTA network simplex kernel (netsimplex.cu).
#pragma once
#include <stddef.h>
#include <stdint.h>

#include "internal.h"

namespace pd {

constexpr int NS_THREADS = 1024;

struct NSInst {
    int32_t n;         // real nodes (root = n)
    int64_t m;         // real arcs
    // arcs a < mst are implicit: tail a / nT, head nS + a % nT, cost cmat[a];
    // arcs mst <= a < m are explicit: tail/head/cost[a - mst]
    int64_t mst;
    int64_t nT;
    int64_t nS;
    const int32_t* cmat;
    const int32_t* tail;
    const int32_t* head;
    const int32_t* cost;
    const int64_t* supply;
    const int64_t* art;  // n or null: the artificial arc of node i costs big + art[i] (art[i] >= 0; null = 0)
    int64_t* pi;       // n + 1
    int32_t* parent;   // n + 1
    int32_t* pred;     // n + 1 (arc id; artificial arc of node i is m + i; m + n < 2^31)
    int32_t* flow;     // n + 1: flow on the pred arc (total supply < 2^31; bit 31 = up while solving in global mode)
    uint8_t* up;       // n + 1: pred arc points from the node to its parent
    int32_t* ord;      // n + 1 preorder
    int32_t* pos;      // n + 1
    int32_t* size;     // n + 1
    int32_t* tmp;      // n + 1 scratch (re-hang buffer of the global layout)
    int32_t* path;     // 2 (n + 1) scratch: the two half-cycles past the shared-memory part
    int32_t* seg;      // 3 * (2n + 3) scratch: segment start, length, output offset
    int64_t block;     // pricing block (arcs)
    int64_t big;       // cost of the artificial arcs (more than any path cost)
    int32_t smem_nodes; // node arrays: 1 all in shared memory, 2 all but pred / flow, 3 the 16-bit ones, 0 global
    int32_t walk;      // shared-memory layout: longest half-cycle side followed by the two-lane walk (longer: the scan)
    int32_t init_tree;  // 1: pi, pred, parent, flow, up, ord, pos, size hold a strongly feasible start
    int32_t pad1;
    int64_t scanned;   // result: arcs priced
    int64_t max_pivots;
    uint64_t time_limit_ns;
    // results
    int64_t opt;
    int64_t pivots;
    int64_t degenerate;
    int32_t status;    // 0 ok, 1 infeasible, 2 pivot cap / time, 3 unbounded, 4 path too long
    int32_t pad;
};

// Persistent over `count` instance records taken in `order` (next = a zeroed
// device counter); results are written back into the records.
__global__ void k_netsimplex(NSInst* insts, const int32_t* __restrict__ order, int32_t count,
                             int32_t* __restrict__ next);
// Dynamic shared memory of N1 nodes in shared-memory layout 1, 2 or 3.
size_t ns_smem_bytes(int64_t N1, int layout);
// Raises the kernel's dynamic shared memory limit on the current device once,
// to the most any instance can use (thread-safe; never lowers it).
cudaError_t ns_kernel_setup();
// The layout N1 nodes get beside the kernel's static shared memory
// (max_optin: the device's opt-in limit per CTA): 1 all node arrays in shared
// memory, 2 all but pred and the packed flow, 3 only the four 16-bit arrays,
// 0 none (global memory).
int ns_smem_layout(int64_t N1, int max_optin);
__global__ void k_i64_to_i32_cost(const int64_t* __restrict__ c, int64_t m, int32_t* __restrict__ o,
                                  unsigned long long* __restrict__ bad);
__global__ void k_abs_sum(const int64_t* __restrict__ s, int64_t n, unsigned long long* __restrict__ out);
__global__ void k_check_network(const int64_t* __restrict__ rp, const int32_t* __restrict__ hd, int64_t n, int64_t m,
                                unsigned long long* __restrict__ bad);

// An instance ready to launch (buffers of the context that prepared it).
struct NSPrep {
    NSInst h{};
    size_t smem = 0;     // dynamic shared memory it needs
    bool ready = false;  // false: nothing to solve
};

// The transportation form of one W1 network, prepared for the simplex.
struct W1Prep {
    NSPrep ns;           // ns.ready false: solve the sparse network instead
    DiagCost dc{1, 0, 0};  // creation / destruction costs of the diagonal node's routes
    const int32_t* S = nullptr;
    const int32_t* T = nullptr;
    int64_t nS = 0, nT = 0, nt = 0;
};

pd_status ns_prepare_arcs(Ctx* c, int32_t n, int64_t m, int64_t mst, int64_t nS, int64_t nT, const int32_t* cmat,
                          const int32_t* tail, const int32_t* head, const int32_t* cost, const int64_t* supply,
                          int64_t cmax, const pd_opts& o, NSPrep* p, cudaStream_t st);
// Runs `count` prepared instances in one launch (one CTA each): h -> device
// records d -> results r (host), synchronising the stream; smem = the largest
// dynamic shared memory of the instances.
pd_status ns_run(Ctx* c, const NSInst* h, int count, size_t smem, NSInst* d, NSInst* r, cudaStream_t st);
pd_status ns_status(Ctx* c, const NSInst& r);
pd_status ns_prepare_w1(Ctx* c, const pd_nodes& nodes, int64_t n_arcs, int64_t dsup, const pd_opts& o, W1Prep* w,
                        cudaStream_t st);
// Certificate (on the WSPD tree of s) and fallback after the launch; d_res =
// the device record of the solved instance, r = its host copy.  merged ==
// nullptr: no fallback here -- out->method = -1 tells the caller to solve the
// sparse network itself.
pd_status ns_finish_w1(Ctx* c, const WsTree& tr, int64_t s, const pd_network* merged, const pd_opts& o,
                       const W1Prep& w, const NSInst* d_res, const NSInst& r, SolveStats* out, cudaStream_t st);
__global__ void k_certify_tree(const NSInst* __restrict__ I, const int32_t* __restrict__ S,
                               const int32_t* __restrict__ T, int64_t nS, int64_t nT, WsTree tr, int64_t s,
                               DiagCost dc, unsigned long long* __restrict__ out);

// One pair's certificate in a batched launch: its solved record, its
// transportation lists and its WSPD tree.
struct CertJob {
    const NSInst* inst;  // device record (set by ns_run_wave from rec)
    int64_t rec;         // index of the pair's record in the wave
    const int32_t* S;
    const int32_t* T;
    int64_t nS, nT, s;
    WsTree tree;
    DiagCost dc;
};
// k_certify_tree for every job: blockIdx.y = job, out[2 job .. 2 job + 1].
__global__ void k_certify_batch(const CertJob* __restrict__ jobs, unsigned long long* __restrict__ out);

// One wave of a batch as a CUDA graph: upload of the records, the persistent
// simplex over all of them, every pair's certificate, download of records and
// certificate counts.  Captured once per configuration, replayed per wave.
pd_status ns_run_wave(Ctx* c, const NSInst* h, int count, size_t smem, const CertJob* jobs, NSInst* r,
                      unsigned long long* cert, cudaStream_t st);

}  // namespace pd
