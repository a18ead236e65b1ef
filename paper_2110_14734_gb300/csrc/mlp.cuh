// The warm-start potential predictor (mlp.cu) and the warm start of the
// network simplex (warm.cu).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "internal.h"
#include "netsimplex.cuh"
#include "prims.cuh"

namespace pd {

constexpr int WS_IN = 72;    // features per node
constexpr int WS_H = 128;    // hidden width (both layers)
constexpr int WS_TILE = 32;  // nodes per block step
constexpr int WS_GRID = 64;  // density grid per axis
// parameter layout: W1 [WS_IN][WS_H], b1, W2 [WS_H][WS_H], b2, w3 [WS_H], b3
constexpr int WS_OFF_W1 = 0;
constexpr int WS_OFF_B1 = WS_OFF_W1 + WS_IN * WS_H;
constexpr int WS_OFF_W2 = WS_OFF_B1 + WS_H;
constexpr int WS_OFF_B2 = WS_OFF_W2 + WS_H * WS_H;
constexpr int WS_OFF_W3 = WS_OFF_B2 + WS_H;
constexpr int WS_OFF_B3 = WS_OFF_W3 + WS_H;
constexpr int WS_NPARAMS = WS_OFF_B3 + 1;
constexpr int WS_PART = WS_NPARAMS + 2;  // gradients, loss sum, mask sum

pd_status mlp_init(Ctx* c, uint64_t seed, bool force, cudaStream_t st);
pd_status mlp_set(Ctx* c, const float* host, cudaStream_t st);
pd_status mlp_get(Ctx* c, float* host, cudaStream_t st);
pd_status mlp_forward(Ctx* c, const __nv_bfloat16* F, int64_t n, float* y, cudaStream_t st);
pd_status mlp_grad(Ctx* c, const __nv_bfloat16* F, const float* t, const float* mask, int64_t n, float inv_norm,
                   float* g, cudaStream_t st);
pd_status mlp_adam(Ctx* c, const float* g, float lr, cudaStream_t st);
// Rows idx[0..n) (device) of the context's data set gathered into a batch
// (context-owned buffers, valid until the next gather).
pd_status mlp_gather_rows(Ctx* c, const int32_t* idx, int64_t n, __nv_bfloat16** F, float** T, float** M,
                          cudaStream_t st);
// Master parameters saved to (restore false) or restored from the snapshot.
pd_status mlp_snapshot(Ctx* c, bool restore, cudaStream_t st);
// Masked mean squared error of data-set rows [r0, r1).
pd_status mlp_loss(Ctx* c, int64_t r0, int64_t r1, double* loss, cudaStream_t st);
pd_status ws_features(Ctx* c, const pd_nodes& nodes, const W1Prep& w, __nv_bfloat16* F, long long* box,
                      cudaStream_t st);
pd_status ws_predict(Ctx* c, const pd_nodes& nodes, const W1Prep& w, std::vector<float>* p, cudaStream_t st);
// Potentials +d(u) / -d(v) from the distance to the diagonal (host, nS + nT + 1).
pd_status ws_diag_potentials(Ctx* c, const pd_nodes& nodes, const W1Prep& w, std::vector<float>* p, cudaStream_t st);
pd_status ws_collect(Ctx* c, const pd_nodes& nodes, const W1Prep& w, const NSInst* d_res, const NSInst& r,
                     int64_t cmax, const std::vector<double>* base, cudaStream_t st);

// Strongly feasible start of a prepared transportation instance from
// potentials p (host, one per transportation node, cost units); the greedy
// takes all arcs between the unbalanced nodes once at most max_residual are
// left.  *used = false (instance untouched) if the greedy does not balance.
pd_status ns_warm_tree(Ctx* c, NSPrep* prep, const double* p, int64_t max_residual, bool* used, cudaStream_t st);

}  // namespace pd
