/*
 * pdw1.h -- C ABI of the GB300 (sm_103a) library for the approximate
 * 1-Wasserstein distance between persistence diagrams by graph
 * sparsification (Dey & Zhang, arXiv 2110.14734).
 *
 * Every step runs in hand-written CUDA kernels on one GPU.  Plain C types
 * only: pointers, sizes, a CUDA stream as an opaque pointer.
 *
 * Conventions (all entry points):
 *   - Device pointers are on the context's device.  Diagram inputs may also be
 *     host pointers (pd_diagram.on_host = 1); the library then copies them to
 *     the device on the given stream.
 *   - Device outputs (pd_nodes, pd_network) are owned by the context and stay
 *     valid until the next call on the same context.  The caller never frees
 *     them.
 *   - Host outputs are written only when the call returns PD_OK.  Entry points
 *     with host outputs synchronise their stream before returning.
 *   - Calls are ordered on the stream passed in (NULL = legacy default
 *     stream).  One context must not be used from two streams at once.
 *   - No C++ exception crosses the ABI.  On an error the context stays usable;
 *     pd_last_error() describes the error.
 *
 * Units: coordinates are quantised to q = 2^-k (k = coord_shift); every cost
 * is an integer number of quanta, rounded UP (so rounded costs keep the
 * triangle inequality); W1 ~= opt_quanta * q.
 */
#ifndef PDW1_H
#define PDW1_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PD_OK = 0,
    PD_EINVAL = 1,      /* bad argument or a non-finite / out-of-range coordinate */
    PD_ENOMEM = 2,      /* device allocation failed or the context's byte cap was reached */
    PD_ECUDA = 3,       /* a CUDA runtime call failed */
    PD_ETIMEOUT = 4,    /* the solver's round cap or a bounded device wait ran out */
    PD_ECAPACITY = 5,   /* a size limit of the library was exceeded (stated in the message) */
    PD_EOVERFLOW = 6,   /* an integer quantity left its 64-bit range */
    PD_EINFEASIBLE = 7  /* the network has no feasible flow */
} pd_status;

typedef struct pd_ctx pd_ctx;

/* Create a context on CUDA device `device`.  arena_bytes caps the device
 * memory the context may hold at once (0 = no cap).  Allocates lazily. */
pd_status pd_create(pd_ctx** out, int device, size_t arena_bytes);
void pd_destroy(pd_ctx* ctx);
/* Message of the last error on this context ("" after success). */
const char* pd_last_error(const pd_ctx* ctx);

/* Kernels launched by this library in this process so far, over all contexts
 * and threads (a utility for measurement; no counterpart in the paper). */
int64_t pd_kernel_launches(void);

typedef enum { PD_F32 = 0, PD_U8 = 1 } pd_dtype;

/* A persistence diagram: n points stored as interleaved (birth, death) pairs,
 * float32 (PD_F32) or uint8 (PD_U8).  Points with birth == death (after
 * quantisation) lie on the diagonal and are ignored (Problem Formulation). */
typedef struct {
    const void* bd;
    int64_t n;
    int32_t dtype;
    int32_t on_host; /* 1: bd is host memory (pinned or pageable) */
} pd_diagram;

/* Options.  pd_opts_default() fills the defaults; a NULL pd_opts* means
 * defaults everywhere. */
typedef struct {
    int32_t coord_shift; /* k of the quantum 2^-k; -1 = 20 for PD_F32, 12 for PD_U8 */
    int32_t s_override;  /* WSPD parameter s; 0 = derived from eps (see pd_w1_approx) */
    int32_t condense;    /* 1 = delta-condensation (Algorithm 2); 0 = only merge coincident points */
    int32_t perturb;     /* 1 = random shift of condensed nodes (Algorithm 2); 0 = none */
    uint64_t seed;       /* seed of the shift (a pure function of seed and lattice cell) */
    int32_t alpha;       /* cost-scaling divisor of the solver, >= 2 (default 8) */
    int32_t verify;      /* 1 = certify optimality of the final flow on the device */
    int64_t max_rounds;  /* solver watchdog: push/relabel rounds over all phases (0 = default) */
    int64_t time_limit_ms;  /* solver watchdog: device wall-clock limit of one solve (0 = 60000) */
    int64_t update_every;   /* relabels between global price updates (0 = number of nodes, -1 = never) */
    int32_t seq_threshold;  /* cost scaling: at most this many active nodes, one block finishes them (-1 = 64) */
    int32_t solver;         /* 0 = network simplex (default), 1 = cost scaling with push/relabel */
    int64_t ns_block;       /* network simplex pricing block in arcs (0 = max(8192, sqrt(arcs))) */
    int32_t ns_transport;   /* W1 only: 1 = try the transportation form with its certificate first when it
                               has at most twice the sparse network's arcs (default); 2 = whenever its
                               arcs fit the simplex (< 2^31); 0 = solve the sparse network itself */
    int32_t ns_smem;        /* network simplex: 1 = hot node arrays in shared memory when they fit (default) */
    int32_t batch_slots;    /* pairs per simplex launch of pd_w1_approx_batch and pd_nn_search
                               (0 = twice the number of SMs) */
    int32_t batch_threads;  /* pd_w1_approx_batch: host threads preprocessing pairs (0 = 8) */
    int32_t nn_prune;       /* pd_nn_search: 1 = skip pairs whose lower bound exceeds the best optimum
                               (default); 0 = solve every pair */
    int32_t warm_start;     /* network simplex on the transportation form: -1 = automatic (default):
                               4 for instances of at least 4,096 transportation nodes in pd_w1_approx
                               and pd_nn_search, else 0; pd_w1_approx_batch starts cold;
                               0 = cold start;
                               1 = start from the coarse solve's potentials (as 4) corrected by the
                               context's network (pd_ws_train / pd_ws_load); 2 = start from the exact
                               potentials of a
                               cold solve of the same pair (diagnostic: the best a prediction can do);
                               3 = start from the potentials +d(u) for sources, -d(v) for sinks (d: the
                               distance to the diagonal), i.e. the greedy by the saving
                               d(u) + d(v) - c(u, v) of pairing u with v (no network);
                               4 = start from the potentials of an exact solve of the same pair
                               condensed onto a coarser lattice (cell max(2 G, node box / warm_cells)),
                               mapped to the fine nodes by the coarse optimum's c-transforms
                               (the midpoint of the upper and lower envelope) */
    int32_t ns_walk;        /* network simplex, trees in shared memory: the two half-cycles of a pivot are
                               followed up the tree by two lanes when neither side is longer than this
                               many nodes, else found by a scan of the whole preorder by the CTA
                               (-1 = the autotuned value, else 0; 0 = always the scan; at most 512) */
    int32_t tree;           /* hierarchical tree of the WSPD: 0 = binary radix tree over the Morton order
                               of the nodes (a compressed quadtree; default), 1 = the paper's split tree
                               (WSPD section: the longest side of a bounding box cut in the middle) */
    int32_t diag_kappa;     /* unbalanced transport (the Conclusion: ā and b̄ as destructor / creator):
                               a unit at p is destroyed (arc p -> ā) or created (b̄ -> p) at cost
                               diag_kappa * d_diag(p) + diag_tau quanta; 1 and 0 (default) give W1
                               between persistence diagrams, 0 a constant cost diag_tau */
    int64_t diag_tau;       /* >= 0 quanta, < 2^30 */
    int32_t warm_cells;     /* warm_start 1 and 4: coarse cells along the longer side of the nodes'
                               bounding box (0 = 64; at most 4096) */
    int32_t nn_wave0;       /* pd_nn_search: pairs of its first wave; later waves double up to
                               batch_slots (0 = 16 with pruning, batch_slots without) */
} pd_opts;

void pd_opts_default(pd_opts* opts);

/* Condensed nodes, device memory owned by the context, ordered by the 64-bit
 * Morton code of (X - min X, Y - min Y) (bit i of x -> bit 2i, of y -> 2i+1). */
typedef struct {
    int64_t n_nodes;
    int32_t* X;
    int32_t* Y;
    int64_t* cntA; /* multiplicity of diagram A at the node */
    int64_t* cntB; /* multiplicity of diagram B at the node */
    uint64_t* morton;
} pd_nodes;

/* Sparse transshipment network in CSR form, device memory owned by the
 * context.  Node ids: 0..N-1 the condensed nodes (Morton rank), N = ā (A's
 * diagonal node), N+1 = b̄ (B's diagonal node); n_nodes = N + 2.  Rows are
 * sorted by head.  cost in quanta; supply[u] = cntA - cntB, supply[ā] = -|A|,
 * supply[b̄] = |B|. */
typedef struct {
    int64_t n_nodes;
    int64_t n_arcs;
    int64_t* row_ptr; /* n_nodes + 1 entries */
    int32_t* head;    /* n_arcs */
    int64_t* cost;    /* n_arcs */
    int64_t* supply;  /* n_nodes */
} pd_network;

typedef struct {
    double w1;              /* opt_quanta * 2^-coord_shift */
    int64_t opt_quanta;     /* optimum of the sparse network (exact, integer) */
    int64_t rwmd_quanta;    /* RWMD of the 0-condensed diagrams, max(L_A, L_B) */
    int64_t rwmd_A;         /* L_A */
    int64_t rwmd_B;         /* L_B */
    int64_t slack_quanta;   /* total flow: bound on the cost rounding, W1 <= w1 + slack*q */
    int64_t mass_A;         /* |A| after dropping diagonal points */
    int64_t mass_B;         /* |B| */
    int32_t s;              /* WSPD parameter used */
    int32_t coord_shift;    /* k used */
    double delta;           /* delta of Algorithm 2, in quanta */
    int64_t cell_quanta;    /* lattice spacing G = max(1, floor(0.99 delta)) */
    int64_t shift_quanta;   /* shift bound P = floor(0.005 delta) */
    int64_t n_nodes;        /* condensed nodes N (without ā, b̄) */
    int64_t n_arcs;         /* arcs of the sparse network */
    int32_t phases;         /* solver: cost-scaling phases */
    int32_t verified;       /* 1 if the device optimality certificate passed */
    int64_t rounds;         /* solver: push/relabel rounds */
    int64_t pushes;         /* solver: push operations */
    int64_t relabels;       /* solver: relabel operations */
    int64_t repair_passes;  /* solver: price-repair passes */
    int64_t price_updates;  /* solver: global price updates */
    int64_t update_passes;  /* solver: relaxation passes of the global price updates */
    int64_t pivots;         /* network simplex: pivots (all attempts) */
    int64_t degenerate;     /* network simplex: pivots that moved no flow */
    int64_t arcs_priced;    /* network simplex: arcs whose reduced cost was evaluated */
    int32_t solve_method;   /* 0 cost scaling, 1 simplex on the sparse network, 2 transportation form + certificate */
    int32_t cert_failures;  /* pairs of the transportation optimum missing from the sparse network */
    int64_t kernel_launches; /* kernels this call launched */
    float ns_kernel_ms;     /* device time of the network simplex kernel(s) of this call */
    int32_t warm_used;      /* 1 if the simplex started from a warm-start tree */
    float stage_ms[8];      /* device time of quantize+0-condense, RWMD, delta-condense, tree, WSPD, CSR;
                               host wall time of the solve (incl. certificate) and of the whole call */
    float warm_ms[2];       /* warm start, host wall time: the potentials (coarse solve and mapping,
                               network inference), then the start tree; 0 for a cold start */
    int64_t warm_pivots;    /* pivots of the coarse solve behind the warm start (0 if none) */
} pd_result;

/*
 * delta-condensation (Algorithm 2, snapping and aggregation): quantise A and B,
 * merge coincident points, snap every node to the common lattice
 * cell_quanta * Z^2 (nearest lattice point, ties up), aggregate the
 * multiplicities per cell, shift each cell's node by a pseudo-random offset
 * in [-shift_quanta, shift_quanta]^2 (a pure function of opts->seed and the
 * cell), and order the nodes by Morton code.  cell_quanta = 1 and
 * shift_quanta = 0 give the 0-condensation of A united with B.
 * Requires cell_quanta >= 1, 0 <= 2 * shift_quanta < cell_quanta.
 */
pd_status pd_condense(pd_ctx* ctx, pd_diagram A, pd_diagram B, int64_t cell_quanta,
                      int64_t shift_quanta, const pd_opts* opts, pd_nodes* out, void* stream);

/*
 * RWMD lower bound (Algorithm 1) of the 0-condensed diagrams with rounded-up
 * costs: L_A = sum_u cntA(u) * min(d_diag(u), min_v c(u, v)) over A's nodes,
 * v over B's nodes (the relaxed min-cost flow also lets a unit go to its
 * diagonal node), L_B symmetric.  out3[0] = L_A, out3[1] = L_B,
 * out3[2] = max(L_A, L_B), host memory, in quanta.
 */
pd_status pd_rwmd_lower_bound(pd_ctx* ctx, pd_diagram A, pd_diagram B, const pd_opts* opts,
                              int64_t* out3, void* stream);

/*
 * Sparse network WS_s^PD (WSPD section, Algorithms 6-9): a binary radix tree
 * (compressed quadtree) over the Morton-ordered nodes, every s-well-separated
 * pair of the s-WSPD as the biarc between the leftmost points of the two sets,
 * the diagonal arcs u -> ā (u holds A mass), b̄ -> v (v holds B mass) and
 * b̄ -> ā at cost 0, assembled into CSR.  `nodes` is device memory laid out as
 * pd_nodes (unique coordinates, ascending Morton code, |X|,|Y| < 2^30).
 */
pd_status pd_wspd_sparsify(pd_ctx* ctx, const pd_nodes* nodes, int32_t s, pd_network* out,
                           void* stream);

/*
 * The sparse network of pd_wspd_sparsify built on a chosen tree: tree = 0 the
 * radix tree (exactly pd_wspd_sparsify), tree = 1 the paper's split tree (WSPD
 * section: a set's tight bounding box is cut at the middle of its longest
 * side, the x side on ties, a point going to the lower half when twice its
 * coordinate is below min + max; recursion to single points).  With the split
 * tree the network's node ids 0..N-1 are the positions of the nodes in the
 * tree's leaf order (the recursion's order, lower half first, the input order
 * kept within each half); ordered_out (may be NULL) receives the nodes in that
 * order (context-owned device memory, valid until the next call).  `nodes` as
 * for pd_wspd_sparsify.
 */
pd_status pd_wspd_sparsify_tree(pd_ctx* ctx, const pd_nodes* nodes, int32_t s, int32_t tree,
                                pd_nodes* ordered_out, pd_network* out, void* stream);

/*
 * Size of the sparse network of pd_wspd_sparsify_tree without building it:
 * the WSPD is enumerated level by level and its pairs counted, no arc is
 * stored.  *n_arcs_out (host) = WSPD biarcs + diagonal arcs + 1, exactly
 * pd_wspd_sparsify_tree's n_arcs.  Device memory: the pair frontier of one
 * level at a time (8 bytes per pair not yet separated).
 */
pd_status pd_wspd_count(pd_ctx* ctx, const pd_nodes* nodes, int32_t s, int32_t tree, int64_t* n_arcs_out,
                        void* stream);

/*
 * Exact integer min-cost flow on an uncapacitated network (the min-cost flow
 * of the transshipment network definition).  Default solver: primal network
 * simplex with block pricing in one CTA (network-simplex section, run to
 * optimality); opts->solver = 1 selects cost scaling with push/relabel rounds
 * in one persistent kernel.  `net` is device memory in pd_network layout:
 * unique (tail, head) arcs, rows sorted by head, costs in [0, 2^31),
 * supplies summing to 0.  *opt_out (host) receives the optimum; stats (host,
 * may be NULL) receives the solver counters.
 */
pd_status pd_mcf_solve(pd_ctx* ctx, const pd_network* net, const pd_opts* opts, int64_t* opt_out,
                       pd_result* stats, void* stream);

/*
 * Approximate W1 (Algorithm 4): delta-condensation with delta from the RWMD
 * (Algorithm 2), the sparse network (pd_wspd_sparsify) and its exact optimum
 * (pd_mcf_solve; the solver contracts the zero-cost arc b̄ -> ā into one
 * diagonal node of supply |B| - |A|, which leaves the optimum unchanged).  s is the smallest integer >= 13 with
 * (1 + 4/s + 4/(s-2)) (1 + 8/(s-4)) <= 1 + eps (the tighter bound of the
 * paper's experiments) unless opts->s_override is set; eps_c = 8/(s-4)
 * (1 for s < 12), delta = 2 eps_c L_lo / (sqrt(2) (|A| + |B|)) with
 * L_lo = max(L_A - |A|, L_B - |B|, 0).  Result (host) in *out.
 */
pd_status pd_w1_approx(pd_ctx* ctx, pd_diagram A, pd_diagram B, double eps, const pd_opts* opts,
                       pd_result* out, void* stream);

/*
 * Algorithm 4 up to the sparse network, without solving: quantise,
 * 0-condense, RWMD, delta-condense, tree and WSPD as pd_w1_approx runs them,
 * the network's arcs counted but not stored.  Fills *out (host) as
 * pd_w1_approx would except for the solver's fields (opt_quanta, w1, slack,
 * pivots ... are 0): s, delta, cell_quanta, shift_quanta, n_nodes, n_arcs, the
 * RWMD and the masses.  For sizing a problem before solving it.
 */
pd_status pd_w1_sparsify_count(pd_ctx* ctx, pd_diagram A, pd_diagram B, double eps, const pd_opts* opts,
                               pd_result* out, void* stream);

/*
 * Approximate W1 of `count` independent pairs (A[i], B[i]), each computed
 * exactly as pd_w1_approx computes it with the same eps and opts (so
 * out[i].opt_quanta equals what pd_w1_approx returns for that pair).  The
 * paper solves one pair at a time; this batched form has no counterpart
 * there.  Pairs are processed in waves of W = opts->batch_slots (0 = twice
 * the number of SMs) pairs: host worker threads (opts->batch_threads) run the
 * preprocessing of the wave's pairs, each on its own stream after the work
 * already queued on `stream`; then the network simplex solves of the wave
 * share one persistent launch (one CTA per SM takes the pairs, largest
 * first); then each pair's certificate runs.
 * A and B: host arrays of `count` descriptors; out: host array of `count`
 * results (ns_kernel_ms and stage_ms[6] include the wave's shared launch).
 * Device memory: one buffer set per slot, grown on demand and kept by the
 * context until pd_destroy (the context's arena cap applies to each slot).
 * opts->solver must be 0.  On an error the status of the first failing pair
 * is returned (its index in pd_last_error) and out is unspecified.
 */
pd_status pd_w1_approx_batch(pd_ctx* ctx, const pd_diagram* A, const pd_diagram* B, int64_t count,
                             double eps, const pd_opts* opts, pd_result* out, void* stream);

/* Result of pd_nn_search (host). */
typedef struct {
    int64_t nn_index;       /* argmin over the database of OPT_int(query, db[i]); ties -> lowest i; -1 if empty */
    int64_t nn_opt_quanta;  /* OPT_int of that pair (-1 if the database is empty) */
    double nn_w1;           /* nn_opt_quanta * 2^-coord_shift */
    int64_t solved;         /* pairs whose W1 was computed */
    int64_t pruned;         /* pairs skipped: lower bound above the best optimum */
    int32_t waves;          /* batched solves issued */
    int32_t coord_shift;    /* k used */
    float lb_ms;            /* device time of the query's condensation and all lower bounds */
    float solve_ms;         /* host wall time of the waves */
    float total_ms;         /* host wall time of the call */
    int32_t wcd_above;      /* diagrams whose WCD bound is above their RWMD bound */
} pd_nn_result;

/*
 * Database for nearest-neighbour search (the NN-search application of the
 * experiments section; the batched database form has no counterpart in the
 * paper).  Records the n_db descriptors -- the caller keeps their memory
 * valid until the database is rebuilt or the context destroyed -- and
 * 0-condenses each diagram once (quantum 2^-k, k from opts->coord_shift or the
 * dtype; all diagrams share one dtype).  Replaces any previous database.
 */
pd_status pd_db_build(pd_ctx* ctx, const pd_diagram* dbs, int64_t n_db, const pd_opts* opts, void* stream);

/*
 * Nearest neighbour of `query` in the database: the index i minimising the
 * approximate W1 of (query, db[i]) as pd_w1_approx computes it (OPT_int;
 * ties -> lowest i).  Two lower bounds, both scaled by (1 - eps_c) with
 * eps_c = 8 / (s - 4) (0 without condensation), because delta-condensation
 * moves the points by at most eps_c * W1 in total:
 *   - RWMD_i, the relaxed-flow bound (Algorithm 1, diagonal included) of the
 *     0-condensed diagrams, evaluated in float32 with every distance rounded
 *     down;
 *   - WCD_i / 2 (Appendix, WCD): the word centroid distance of
 *     query + db[i]'s diagonal projections against db[i] + the query's
 *     projections is at most twice W1; it equals |T_q - T_i| / sqrt(2) with
 *     T the total persistence sum (d - b) of a diagram (exact integers; each
 *     database diagram's T is summed once by pd_db_build).
 * LB_i = max of the two, rounded down, <= OPT_int(query, db[i]).  Pairs are
 * solved in ascending LB_i (ties by index), opts->batch_slots pairs
 * per batched solve (pd_w1_approx_batch); with opts->nn_prune (default) the
 * search stops at the first pair whose bound exceeds the best optimum found,
 * which leaves the answer unchanged.  opt_out (host, n_db entries, may be
 * NULL): OPT_int of every solved pair, -1 for pruned pairs; lb_out (host,
 * n_db, may be NULL): LB_i; wcd_out (host, n_db, may be NULL): the WCD bound
 * alone.  An empty database gives nn_index = -1.
 */
pd_status pd_nn_search(pd_ctx* ctx, pd_diagram query, double eps, const pd_opts* opts, pd_nn_result* out,
                       int64_t* opt_out, int64_t* lb_out, int64_t* wcd_out, void* stream);

/* ---- autotuner of the simplex's launch parameters (no counterpart in the paper)
 *
 * The paper's block search prices blocks of sqrt(arcs) arcs.  pd_autotune
 * measures instead: it prepares the transportation instance of each sample
 * pair (A[i], B[i]) at eps/opts exactly as pd_w1_approx does, solves it once
 * per candidate (pricing block of 4096 ... 32768 arcs) x (walk limit 0, 8,
 * 32, see pd_opts.ns_walk), and once with the defaults, each launch timed by
 * CUDA events, and keeps the fastest pair of values of each size class
 * floor(log2(arcs + nodes)) in the context: later solves of that class whose
 * opts->ns_block is 0 (and ns_walk -1) use them (pd_w1_approx,
 * pd_w1_approx_batch, pd_nn_search, pd_mcf_solve).  Every candidate reaches
 * the same optimum (checked).  cache_path (may be NULL): a text file of lines
 * "gpu-name sms class block walk"; classes it already holds for this GPU are
 * loaded instead of timed, and newly timed classes are written back (other
 * GPUs' lines kept).  Must not run concurrently with other calls on the same
 * context. */
typedef struct {
    int64_t ns_block;   /* block chosen for the first sample pair's size class (0 if none) */
    int32_t ns_walk;    /* walk limit chosen for that class (pd_opts.ns_walk) */
    int32_t size_class; /* that class, floor(log2(arcs + nodes)); -1 if no pair had a transportation form */
    int32_t candidates; /* candidate blocks */
    int32_t pairs;      /* pairs timed (not taken from the cache) */
    int32_t from_cache; /* 1: the first pair's class came from cache_path */
    float best_ms;      /* simplex device time of the timed pairs of that class with the chosen block */
    float default_ms;   /* ... with the default block max(8192, sqrt(arcs + nodes)) and walk 0 */
} pd_tune_result;

pd_status pd_autotune(pd_ctx* ctx, const pd_diagram* A, const pd_diagram* B, int64_t count, double eps,
                      const pd_opts* opts, const char* cache_path, pd_tune_result* out, void* stream);
/* The block the context uses for an instance of arcs + nodes = M (0: none tuned, the default applies). */
pd_status pd_tuned_block(const pd_ctx* ctx, int64_t arcs_and_nodes, int64_t* block_out);

/* ---- learned warm start (no counterpart in the paper) ----------------------
 *
 * A network of 72 -> 128 -> 128 -> 1 units (ReLU) predicts, per node of the
 * transportation form, the correction from the potentials of a coarse solve
 * of the same pair (pd_opts warm_start = 4) to its optimal potential (up to a
 * common offset); the simplex then starts from a greedy flow on the arcs of
 * smallest predicted reduced cost, each tree of that forest hung from the
 * root at its predicted potential, instead of the all-artificial tree
 * (pd_opts warm_start = 1).  Weights are stored in bf16, products accumulate in
 * float32; the float32 master parameters (PD_WS_NPARAMS floats) are laid out
 * as W1[72][128], b1[128], W2[128][128], b2[128], w3[128], b3 (W[k][j] is the
 * weight from input k to unit j); w3 and b3 start at 0, so an untrained
 * network gives the coarse start unchanged.  Features of a node (72): its
 * coordinates relative to the pair's node box and divided by the box's larger
 * side, log(1 + cntA), log(1 + cntB), an 8 x 8 window (offsets -4..3) of a
 * 64 x 64 grid over the box holding sign(s) log(1 + |s|) of the summed supply
 * s = cntA - cntB of the nodes in each cell, half the gap between the coarse
 * optimum's upper and lower c-transform envelopes at the node over the coarse
 * cell Gc (at most 16), +1 / -1 for a source / sink, and the node's offset
 * from its coarse lattice point over Gc.  Target: ((potential of the node in
 * the optimal tree - the mean potential of the tree's largest component below
 * the root) - (the same for the coarse solve's potentials)) / Gc, for the
 * nodes of that component.
 */
#define PD_WS_NFEAT 72
#define PD_WS_NPARAMS 25985

typedef struct {
    int64_t rows;        /* training rows (transportation nodes) collected */
    int32_t pairs;       /* pairs whose cold solve gave rows */
    int32_t steps;       /* optimiser steps */
    float loss_first;    /* mean squared error of the first step */
    float loss_last;     /* ... of the last step */
    float collect_ms;    /* host wall time of the cold solves and feature extraction */
    float train_ms;      /* host wall time of the optimisation */
    int64_t cold_pivots; /* pivots of the cold solves */
    int64_t val_rows;    /* rows of the held-out pairs */
    int32_t val_pairs;   /* held-out pairs: the last n_pairs / 8 (at least one) when n_pairs >= 4, else 0 */
    int32_t best_epoch;  /* epoch whose weights are kept (0: the initial ones, i.e. no correction) */
    float val_loss_zero; /* held-out mean squared error of predicting no correction */
    float val_loss;      /* held-out mean squared error of the kept weights */
} pd_ws_stats;

/* Trains the context's network (initialised from `seed` on first use) on the
 * potentials of cold solves of the n_pairs pairs (A[i], B[i]) at eps/opts:
 * `epochs` passes of Adam (lr) over minibatches of 2048 rows drawn in a
 * seeded random order, on the device.  The last pairs are held out (see
 * pd_ws_stats.val_pairs); the weights of the epoch with the smallest held-out
 * error are kept, the initial ones (no correction) when no epoch beats them. */
pd_status pd_ws_train(pd_ctx* ctx, const pd_diagram* A, const pd_diagram* B, int64_t n_pairs, double eps,
                      const pd_opts* opts, int32_t epochs, float lr, uint64_t seed, pd_ws_stats* out,
                      void* stream);
/* Master parameters (host, PD_WS_NPARAMS floats) out of / into the context. */
pd_status pd_ws_get_params(pd_ctx* ctx, float* params);
pd_status pd_ws_set_params(pd_ctx* ctx, const float* params);
/* Network output for n feature rows (host n x PD_WS_NFEAT floats, rounded to
 * bf16 on the way in) into y (host, n). */
pd_status pd_ws_forward(pd_ctx* ctx, const float* feats, int64_t n, float* y, void* stream);
/* Loss sum_i mask_i (y_i - t_i)^2 / n and its gradient with respect to the
 * master parameters (host, PD_WS_NPARAMS), as the training step computes it
 * (bf16 weights and features, float32 arithmetic).  mask may be NULL (all 1). */
pd_status pd_ws_grad(pd_ctx* ctx, const float* feats, const float* target, const float* mask, int64_t n,
                     float* grad, float* loss, void* stream);
/* Parameters to / from a file (a 16-byte header, then the floats). */
pd_status pd_ws_save(pd_ctx* ctx, const char* path);
pd_status pd_ws_load(pd_ctx* ctx, const char* path);

/*
 * Allocation-free min-cost flow (no counterpart in the paper).
 *
 * Some callers cannot allocate device memory when they solve: code running
 * under an allocator that forbids growth after start-up (a serving process
 * with a fixed memory budget, a framework that owns every device byte through
 * its own pool), or code that must not trigger the implicit synchronisation
 * and latency of cudaMalloc / cudaFree in the middle of its work.  For them
 * this entry point solves the same problem as pd_mcf_solve, with the same
 * network simplex kernel, but takes no context and allocates nothing: its
 * scratch is one fixed array of 12 MiB in the library's device memory, which
 * every GPU that loads the library holds until the process exits.
 *
 * `net`: device memory in pd_network layout, as for pd_mcf_solve, with at
 * most PD_NOALLOC_MAX_NODES - 1 nodes and PD_NOALLOC_MAX_ARCS arcs; larger
 * networks return PD_ECAPACITY (so do total supplies >= 2^31).  *opt_out
 * (host) receives the optimum.  The call synchronises `stream` and reads
 * results back to the host, so it must not be called while `stream` (or the
 * legacy default stream) is being captured into a CUDA graph.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  All calls share the one array and it keeps the last call's
 * contents: calls whose GPU work overlaps (other streams, other host threads
 * on the same device) race with each other and must be serialised by the
 * caller.  Errors are reported by the return code only.
 */
#define PD_NOALLOC_MAX_NODES 32768
#define PD_NOALLOC_MAX_ARCS (1 << 20)
pd_status pd_mcf_solve_noalloc(const pd_network* net, int64_t* opt_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PDW1_H */
