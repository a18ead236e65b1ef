// Internal (C++) interface between the entry points and the stages.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/pdw1.h"
#include "common.cuh"

namespace pd {

// Named device buffers held by a context; each grows on demand.
enum Buf : int {
    B_IN_A, B_IN_B,                 // staged host diagrams
    B_QX, B_QY, B_QKEY, B_QKEY2, B_QVAL, B_QVAL2, B_FLAG, B_IDX,
    B_HAT_X, B_HAT_Y, B_HAT_C,      // 0-condensed nodes of A then B
    B_CKEY, B_CKEY2, B_CVAL, B_CVAL2, B_CIDX, B_CX, B_CY, B_CA, B_CB,
    B_NX, B_NY, B_NCA, B_NCB, B_NCODE,  // output nodes
    B_T_LEFT, B_T_RIGHT, B_T_BB, B_T_REP, B_T_PARENT, B_T_LPARENT, B_T_VISIT,
    B_F0, B_F1, B_WSFLAG, B_WSOFF,  // WSPD frontier
    B_ARCKEY, B_ARCKEY2,            // arc keys (tail << hb | head)
    B_ROWPTR, B_HEAD, B_COST, B_SUPPLY,
    B_S_ROWPTR, B_S_HEAD, B_S_CW, B_S_TWIN, B_S_X, B_S_PAIR, B_S_XKEY, B_S_XKEY2, B_S_XVAL,
    B_S_XVAL2, B_S_XPTR, B_S_XPOS, B_S_TAIL,
    B_S_E, B_S_P, B_S_D, B_S_CUR, B_S_RELAB, B_S_CTL, B_S_Q,
    B_RS_COUNTS, B_RS_PART, B_SCAN_PART,
    B_M_ROWPTR, B_M_SUPPLY,
    B_NS_PI, B_NS_PARENT, B_NS_PRED, B_NS_FLOW, B_NS_UP, B_NS_ORD, B_NS_POS, B_NS_SIZE, B_NS_TMP,
    B_NS_PATH, B_NS_SEG, B_NS_INST, B_NS_ORDER, B_NS_COST, B_NS_ART, B_TR_S, B_TR_T, B_TR_SUP, B_TR_XCOST,
    B_DB_SXY, B_DB_SCNT, B_DB_SID,  // nearest-neighbour database: staging
    B_DB_XY, B_DB_CNT, B_DB_ID, B_DB_OFF, B_DB_ROFF, B_Q_XY, B_Q_CNT, B_DB_LA, B_DB_BIG, B_DB_VAL, B_DB_PERS,
    B_MLP_P, B_MLP_M, B_MLP_V, B_MLP_WB, B_MLP_PART, B_MLP_G,  // warm-start network
    B_WS_GRID, B_WS_FEAT, B_WS_Y, B_WS_PS, B_WS_BOX, B_WS_DF, B_WS_DT, B_WS_DM, B_WS_IN, B_WS_TIN, B_WS_MIN,
    B_WS_P, B_WS_ROWK, B_WS_COLK, B_WS_ARCS, B_WS_COST, B_WS_RS, B_WS_RT, B_WS_RC, B_WS_COMP, B_WS_CSIZE, B_WS_CSUM,
    B_SP_ORD, B_SP_ORD2, B_SP_SEG, B_SP_SEG2, B_SP_HI, B_SP_HI2, B_SP_NUM, B_SP_NUM2,  // split tree
    B_SP_BB, B_SP_REPK, B_SP_REPN, B_SP_FLAG, B_SP_RANK, B_SP_X, B_SP_Y, B_SP_CA, B_SP_CB, B_SP_CODE, B_SP_POS,
    B_CO_BOX, B_CO_P, B_CO_P2, B_CO_GAP,  // coarse-solve warm start
    B_MLP_BEST, B_WS_BF, B_WS_BT, B_WS_BM, B_WS_IDX,  // network training: best weights, shuffled batch
    B_NS_JOBS, B_NS_CERT,           // batched certificate
    B_RW_BOX, B_RW_START, B_RW_CUR, B_RW_PTS, B_RW_LIST, B_RW_NL,  // RWMD grid
    B_SMALL,                        // small device scalars
    B_COUNT
};

struct Ctx {
    int device = 0;
    size_t cap = 0;
    size_t held = 0;
    bool defer_free = false;         // retire grown-out blocks instead of freeing them (batch threads)
    std::vector<void*> retired;      // blocks waiting for ctx_release
    size_t retired_bytes = 0;
    std::string err;
    void* ptr[B_COUNT] = {};
    size_t bytes[B_COUNT] = {};
    int64_t* h_small = nullptr;  // pinned host mirror of small scalars
    pd_nodes nodes{};
    pd_network net{};
    int sm_count = 0;
    float last_ns_ms = 0.f;  // device time of the network simplex kernels since it was last reset
    std::vector<Ctx*> slots;    // pd_w1_approx_batch: per-pair buffers kept from preprocessing to solve
    std::vector<Ctx*> workers;  // pd_w1_approx_batch: preprocessing contexts, one per host thread
    cudaStream_t own_stream = nullptr;  // stream of a worker context
    // nearest-neighbour database (pd_db_build): caller-owned diagrams and
    // their 0-condensed nodes packed in B_DB_XY / B_DB_CNT / B_DB_ID / B_DB_OFF
    std::vector<pd_diagram> db;
    std::vector<int64_t> db_hats;
    int64_t db_total = 0;
    int db_k = 0, db_dtype = 0;
    bool db_big = false;  // a database coordinate is not exact in float32
    std::vector<int64_t> db_pers;  // total persistence sum cnt * (Y - X) of every database diagram (quanta)
    // warm-start network: parameters in B_MLP_* (of mlp_owner when set, as
    // for the batch workers), training rows in B_WS_DF / DT / DM
    bool mlp_ready = false;
    int64_t mlp_steps = 0;
    int64_t ws_rows = 0, ws_cap = 0;
    Ctx* mlp_owner = nullptr;
    // pricing blocks chosen by pd_autotune, per size class (of the context that
    // ran it: slots and workers of a batch look theirs up in `parent`)
    std::map<int, int64_t> tuned_block;
    std::map<int, int32_t> tuned_walk;
    Ctx* parent = nullptr;
    Ctx* coarse = nullptr;            // helper context of the coarse solve (warm_start 4)
    int64_t last_coarse_pivots = 0;   // pivots of the last coarse solve
    int64_t last_coarse_cell = 0;     // its lattice cell (quanta; 0: no coarse solve)
    // the batch's wave as a CUDA graph (ns_run_wave): pinned staging, the
    // captured executable and what it was captured with
    void* wave_pin = nullptr;
    size_t wave_pin_bytes = 0;
    cudaGraphExec_t wave_exec = nullptr;
    cudaStream_t wave_stream = nullptr;
    cudaEvent_t wave_ev[3] = {nullptr, nullptr, nullptr};
    uint64_t wave_key = 0;
    int64_t wave_launches = 0;        // graph launches (each replays the wave's kernels)
};

Ctx* ctx_new(int device, size_t cap);  // nullptr on failure
void ctx_free(Ctx* c);
void ctx_release(Ctx* c);  // frees the blocks a deferring context retired

// Returns a device buffer of at least `bytes` bytes (contents undefined), or
// nullptr (ctx->err set) when allocation fails or the cap is reached.
void* buf(Ctx* c, Buf id, size_t bytes);

template <typename T>
T* bufT(Ctx* c, Buf id, int64_t n) {
    return (T*)buf(c, id, sizeof(T) * (size_t)(n > 0 ? n : 1));
}

pd_status fail(Ctx* c, pd_status st, const std::string& msg);
pd_status cuda_fail(Ctx* c, cudaError_t e, const char* where);

#define PD_TRY_CUDA(c, expr)                                    \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return cuda_fail((c), _e, #expr); \
    } while (0)

#define PD_TRY(expr)                       \
    do {                                   \
        pd_status _s = (expr);             \
        if (_s != PD_OK) return _s;        \
    } while (0)

// Quantised diagram points already on the device.
struct DevDiag {
    const void* bd;
    int64_t n;
    int dtype;
};

// 0-condensed nodes of A (first nA) and B (next nB): device X, Y, cnt.
struct Hats {
    int32_t* X;
    int32_t* Y;
    int64_t* cnt;
    int64_t nA, nB;  // node counts
    int64_t FA, FB;  // masses (points kept)
};

struct SolveStats {
    int64_t opt = 0, slack = 0, rounds = 0, pushes = 0, relabels = 0, repairs = 0, updates = 0, update_passes = 0;
    int64_t pivots = 0, degenerate = 0, cert_failures = 0, scanned = 0;
    int32_t phases = 0, verified = 0, method = 0;  // method: 0 cost scaling, 1 simplex on the network, 2 transport form
};

pd_status stage_condense0(Ctx* c, const DevDiag& A, const DevDiag& B, int k, Hats* out, cudaStream_t st);
pd_status stage_rwmd(Ctx* c, const Hats& h, int64_t L[3], DiagCost dc, cudaStream_t st);
pd_status stage_condense_delta(Ctx* c, const Hats& h, int64_t G, int64_t P, uint64_t seed, pd_nodes* out,
                               cudaStream_t st);
// Hierarchical tree of the WSPD (device arrays of the context that built it):
// internal nodes 0..N-2 with children (c >= 0 internal, c < 0 leaf ~c), tight
// boxes (min x, max x, min y, max y) and leftmost representatives.
struct WsTree {
    int64_t N;
    const int32_t* X;
    const int32_t* Y;
    const int32_t* left;
    const int32_t* right;
    const int4* bb;
    const int32_t* rep;
};

// count_only: the WSPD is enumerated and its arcs counted (out->n_arcs,
// n_nodes), but no arc is stored and out's arrays are null.  tree (may be
// null) receives the hierarchical tree.  given (may be null): a tree already
// built over `nodes` (the split tree), used instead of the radix tree.
pd_status stage_network(Ctx* c, const pd_nodes& nodes, int64_t s, pd_network* out, float* ms_tree,
                        float* ms_wspd, float* ms_csr, cudaStream_t st, bool count_only = false,
                        WsTree* tree = nullptr, const WsTree* given = nullptr, DiagCost dc = DiagCost{1, 0, 0});
// The paper's split tree over `nodes` (splittree.cu): *nodes is replaced by
// the nodes in the tree's leaf order (context buffers), *tree receives the
// tree over those positions, *perm_out (may be null) position -> input index.
pd_status stage_split_tree(Ctx* c, pd_nodes* nodes, WsTree* tree, int32_t** perm_out, cudaStream_t st);
pd_status merge_diagonal(Ctx* c, const pd_network& net, int64_t N, pd_network* out, cudaStream_t st);

// Algorithm 4 up to the network handed to the solver: quantise, 0-condense,
// RWMD, delta-condense, (split tree,) sparse network, diagonal merge.
struct Front {
    Hats h{};
    int64_t L[3] = {0, 0, 0};
    int64_t s = 0, G = 1, P = 0;
    double delta = 0.0;
    int k = 0;
    pd_nodes nodes{};
    pd_network net{}, mnet{};  // count-only front half: net holds only the counts, mnet is empty
    WsTree tree{};
    bool counted = false;
    float ms[6] = {};  // quantise+0-condense, RWMD, delta-condense, tree, WSPD, CSR
};

// count_only: the sparse network is enumerated and counted but not stored
// (enough for the transportation form and its certificate).
pd_status front_half(Ctx* c, const pd_diagram& A, const pd_diagram& B, double eps, const pd_opts& o, Front* f,
                     cudaStream_t st, bool count_only);

struct W1Prep;
// Potentials of the fine transportation instance w from an exact solve of the
// same pair condensed onto a coarser lattice (coarse.cu); empty if there is
// nothing to solve at the coarse level.
pd_status ws_coarse_potentials(Ctx* c, const Front& f, const W1Prep& w, const pd_opts& o, std::vector<double>* p,
                               cudaStream_t st);
pd_status stage_solve(Ctx* c, const pd_network& net, const pd_opts& o, SolveStats* out, cudaStream_t st);

pd_status validate_nodes(Ctx* c, const pd_nodes& nodes, cudaStream_t st);
pd_status validate_network(Ctx* c, const pd_network& net, cudaStream_t st);

pd_status ns_solve_network(Ctx* c, const pd_network& net, const pd_opts& o, SolveStats* out, cudaStream_t st);
__global__ void k_arc_tails(const int64_t* __restrict__ rp, int64_t n, int64_t m, int32_t* __restrict__ tail);
__global__ void k_max_cost(const int64_t* __restrict__ cost, int64_t m, unsigned long long* __restrict__ out);
__global__ void k_max_cost32(const int32_t* __restrict__ cost, int64_t m, unsigned long long* __restrict__ out);

__global__ void k_row_ptr(const uint64_t* key, int64_t m, int hb, int64_t nrows, int64_t* row_ptr);

// creation / destruction costs of the options (validated by check_diag_cost)
inline DiagCost diag_cost(const pd_opts& o) { return DiagCost{o.diag_kappa, 0, o.diag_tau}; }
pd_status check_diag_cost(Ctx* c, const pd_opts& o);

// entry-point helpers shared by the C ABI files
int default_shift(int dtype);                // k of the quantum for a dtype
int64_t s_for_eps(double eps);               // WSPD parameter s from eps (-1 if none)
pd_status check_diag(Ctx* c, const pd_diagram& d);
pd_status stage_inputs(Ctx* c, const pd_diagram& A, const pd_diagram& B, DevDiag* a, DevDiag* b, cudaStream_t st);
// pd_w1_approx_batch after argument checks (opts resolved)
pd_status batch_solve(Ctx* c, const pd_diagram* A, const pd_diagram* B, int64_t count, double eps,
                      const pd_opts& o, pd_result* out, cudaStream_t st);

// Size class of a simplex instance with M arcs + nodes, and the pricing block
// pd_autotune chose for it (0 = none: the default block).
int tune_class(int64_t M);
int64_t tuned_block(const Ctx* c, int64_t M);
int32_t tuned_walk(const Ctx* c, int64_t M);  // the walk limit (16 when none was tuned)

// radix sort / scan with context scratch
pd_status sort_u64(Ctx* c, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t n,
                   int bits, cudaStream_t st);
pd_status scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, cudaStream_t st);

}  // namespace pd

// The opaque context of the C ABI.
struct pd_ctx : public pd::Ctx {};
