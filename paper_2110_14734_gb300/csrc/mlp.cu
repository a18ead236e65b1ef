// The potential predictor of the warm start: per transportation node, 68
// features -> 128 -> 128 -> 1 (ReLU), weights stored in bf16 with float32
// master copies for the optimiser, every product accumulated in float32.
// Forward, backward and Adam are this file's kernels; the predictor and its
// training are not part of the paper (its solver always starts cold).
//
// Features of a node at (X, Y) of a pair whose condensed nodes span the box
// [x0, x0 + ext] x [y0, y0 + ext]:
//   0, 1   (X - x0) / ext, (Y - y0) / ext
//   2, 3   log(1 + cntA), log(1 + cntB)
//   4..67  an 8 x 8 window of a 64 x 64 grid over the box around the node's
//          grid cell (offsets -4..3 on each axis): per cell the signed supply
//          sum(cntA - cntB) of the nodes in it, as sign * log(1 + |sum|)
//   68     half the gap between the coarse optimum's two c-transform
//          envelopes at the node, over the coarse cell Gc (at most 16)
//   69     +1 for a source, -1 for a sink
//   70, 71 offset of the node from its coarse lattice point, over Gc
//          (in [-1/2, 1/2]); 68, 70, 71 are 0 without a coarse solve
// Target / output: the correction from the coarse solve's potential to the
// optimal one (each less its mean over the largest component of the optimal
// simplex tree), over Gc (the box's side without a coarse solve); nodes
// outside that component are left out of the loss.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "mlp.cuh"

namespace pd {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------

__global__ void k_box(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t N,
                      long long* __restrict__ box) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long mnx = LLONG_MAX, mny = LLONG_MAX, mxx = LLONG_MIN, mxy = LLONG_MIN;
    if (i < N) {
        mnx = mxx = X[i];
        mny = mxy = Y[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if ((threadIdx.x & 31) == 0 && mxx != LLONG_MIN) {
        atomicMin(&box[0], mnx);
        atomicMin(&box[1], mny);
        atomicMax(&box[2], mxx);
        atomicMax(&box[3], mxy);
    }
}

PD_D int grid_cell(int32_t v, long long v0, long long ext) {
    long long g = ((long long)v - v0) * WS_GRID / (ext + 1);
    return (int)(g < 0 ? 0 : (g >= WS_GRID ? WS_GRID - 1 : g));
}

__global__ void k_grid(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                       const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB, int64_t N,
                       const long long* __restrict__ box, float* __restrict__ grid) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long ext = max(box[2] - box[0], box[3] - box[1]);
    const int gx = grid_cell(X[i], box[0], ext), gy = grid_cell(Y[i], box[1], ext);
    atomicAdd(&grid[gx * WS_GRID + gy], (float)(cntA[i] - cntB[i]));
}

// Features of the transportation nodes: sources S, sinks T (condensed node
// ids); rows nS + nT (the diagonal node) get no row.
__global__ void k_features(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                           const int64_t* __restrict__ cntA, const int64_t* __restrict__ cntB,
                           const int32_t* __restrict__ S, const int32_t* __restrict__ T, int64_t nS, int64_t nT,
                           const long long* __restrict__ box, const float* __restrict__ grid,
                           const double* __restrict__ gap, int64_t Gc, __nv_bfloat16* __restrict__ F) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nS + nT) return;
    const int32_t u = r < nS ? S[r] : T[r - nS];
    const long long ext = max(max(box[2] - box[0], box[3] - box[1]), 1LL);
    __nv_bfloat16* f = F + r * WS_IN;
    f[0] = __float2bfloat16((float)((double)((long long)X[u] - box[0]) / (double)ext));
    f[1] = __float2bfloat16((float)((double)((long long)Y[u] - box[1]) / (double)ext));
    f[2] = __float2bfloat16(log1pf((float)cntA[u]));
    f[3] = __float2bfloat16(log1pf((float)cntB[u]));
    const int gx = grid_cell(X[u], box[0], ext), gy = grid_cell(Y[u], box[1], ext);
    for (int dx = 0; dx < 8; dx++)
        for (int dy = 0; dy < 8; dy++) {
            const int cx = gx + dx - 4, cy = gy + dy - 4;
            float v = 0.f;
            if (cx >= 0 && cx < WS_GRID && cy >= 0 && cy < WS_GRID) v = grid[cx * WS_GRID + cy];
            f[4 + dx * 8 + dy] = __float2bfloat16(v < 0.f ? -log1pf(-v) : log1pf(v));
        }
    float g = 0.f, ox = 0.f, oy = 0.f;
    if (Gc > 0) {
        g = gap ? (float)fmin(gap[r] / (double)Gc, 16.0) : 0.f;
        // the coarse lattice point of Algorithm 2's snapping: floor((2X + Gc) / (2 Gc)) Gc
        const int64_t cx = floor_div(2 * (int64_t)X[u] + Gc, 2 * Gc), cy = floor_div(2 * (int64_t)Y[u] + Gc, 2 * Gc);
        ox = (float)((double)((int64_t)X[u] - cx * Gc) / (double)Gc);
        oy = (float)((double)((int64_t)Y[u] - cy * Gc) / (double)Gc);
    }
    f[68] = __float2bfloat16(g);
    f[69] = __float2bfloat16(r < nS ? 1.f : -1.f);
    f[70] = __float2bfloat16(ox);
    f[71] = __float2bfloat16(oy);
}

// The child of the root above node v in the solved tree (its component).
PD_D int32_t tree_component(const int32_t* __restrict__ parent, int32_t v, int32_t root, int32_t limit) {
    for (int32_t k = 0; k < limit; k++) {
        const int32_t p = parent[v];
        if (p == root || p < 0) return v;
        v = p;
    }
    return -1;
}

// Component (child of the root) of every transportation node in the solved
// tree, and the component sizes.
__global__ void k_components(const int32_t* __restrict__ parent, int64_t n, int32_t root, int32_t* __restrict__ comp,
                             int32_t* __restrict__ size) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t c = tree_component(parent, (int32_t)r, root, root + 1);
    comp[r] = c;
    if (c >= 0) atomicAdd(&size[c], 1);
}

__global__ void k_component_sum(const int64_t* __restrict__ pi, const int32_t* __restrict__ comp, int64_t n,
                                int32_t anchor, unsigned long long* __restrict__ sum) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n && comp[r] == anchor) atomicAdd(sum, (unsigned long long)pi[r]);  // two's complement sum
}

// Targets: (pi(node) - mean pi of the largest component) / ext for the nodes
// of the largest component of the optimal tree (mask 1).  The other
// components hang from the root by artificial arcs, which fix their
// potentials only up to an offset of their own; a common offset does not
// matter to the start (only differences enter reduced costs).
// Target of row r: its optimal potential minus the anchor component's mean,
// less the same for the base potentials (a coarse solve's) when given, over
// `scale` (the coarse cell; the node box's side when 0); rows outside the
// anchor component are masked out.
__global__ void k_targets(const int64_t* __restrict__ pi, const int32_t* __restrict__ comp, int64_t n,
                          int32_t anchor, double mean, const double* __restrict__ base, double base_mean,
                          const long long* __restrict__ box, int64_t scale, float* __restrict__ t,
                          float* __restrict__ mask) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const long long ext = scale > 0 ? (long long)scale : max(max(box[2] - box[0], box[3] - box[1]), 1LL);
    const bool ok = comp[r] == anchor;
    const double b = base ? base[r] - base_mean : 0.0;
    t[r] = ok ? (float)(((double)pi[r] - mean - b) / (double)ext) : 0.f;
    mask[r] = ok ? 1.f : 0.f;
}

// Potentials from the distance to the diagonal: +d(u) for a source, -d(v)
// for a sink, 0 for the diagonal node, so that the reduced cost of an arc is
// c(u, v) - d(u) - d(v) <= 0: minus the saving of sending u to v instead of
// both to the diagonal.
__global__ void k_diag_potentials(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                                  const int32_t* __restrict__ S, const int32_t* __restrict__ T, int64_t nS, int64_t nT,
                                  float* __restrict__ p, DiagCost dc) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > nS + nT) return;
    if (r == nS + nT) {
        p[r] = 0.f;
        return;
    }
    const int32_t u = r < nS ? S[r] : T[r - nS];
    const float d = (float)cost_make(X[u], Y[u], dc);
    p[r] = r < nS ? d : -d;
}

pd_status ws_diag_potentials(Ctx* c, const pd_nodes& nodes, const W1Prep& w, std::vector<float>* p, cudaStream_t st) {
    const int64_t n = w.nS + w.nT;
    float* dp = bufT<float>(c, B_WS_PS, n + 1);
    if (!dp) return PD_ENOMEM;
    k_diag_potentials<<<grid_for(n + 1, 256), 256, 0, st>>>(nodes.X, nodes.Y, w.S, w.T, w.nS, w.nT, dp, w.dc); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    p->resize((size_t)(n + 1));
    PD_TRY_CUDA(c, cudaMemcpyAsync(p->data(), dp, sizeof(float) * (n + 1), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    return PD_OK;
}

// ---------------------------------------------------------------------------
// the network: tiles of WS_TILE nodes, thread j owns hidden unit j
// ---------------------------------------------------------------------------

struct MlpW {
    const __nv_bfloat16* W1;  // [WS_IN][WS_H]
    const float* b1;          // [WS_H]
    const __nv_bfloat16* W2;  // [WS_H][WS_H]
    const float* b2;
    const __nv_bfloat16* w3;  // [WS_H]
    const float* b3;          // [1]
};

// Forward of one tile: x (smem, [WS_TILE][WS_IN] float) -> h1, h2 (smem) and
// the outputs (smem, [WS_TILE]).
PD_D void tile_forward(const MlpW& w, const float* x, float* h1, float* h2, float* out, int nrow) {
    const int j = threadIdx.x;
    float acc[WS_TILE];
#pragma unroll
    for (int r = 0; r < WS_TILE; r++) acc[r] = 0.f;
    for (int k = 0; k < WS_IN; k++) {
        const float wk = __bfloat162float(w.W1[k * WS_H + j]);
#pragma unroll
        for (int r = 0; r < WS_TILE; r++) acc[r] = fmaf(x[r * WS_IN + k], wk, acc[r]);
    }
    const float bj = w.b1[j];
#pragma unroll
    for (int r = 0; r < WS_TILE; r++) h1[r * WS_H + j] = fmaxf(acc[r] + bj, 0.f);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < WS_TILE; r++) acc[r] = 0.f;
    for (int k = 0; k < WS_H; k++) {
        const float wk = __bfloat162float(w.W2[k * WS_H + j]);
#pragma unroll
        for (int r = 0; r < WS_TILE; r++) acc[r] = fmaf(h1[r * WS_H + k], wk, acc[r]);
    }
    const float b2j = w.b2[j];
#pragma unroll
    for (int r = 0; r < WS_TILE; r++) h2[r * WS_H + j] = fmaxf(acc[r] + b2j, 0.f);
    __syncthreads();
    // out[r] = sum_j h2[r][j] w3[j] + b3: warp r % 4 .. sums rows
    const int lane = j & 31, wid = j >> 5;
    for (int r = wid; r < nrow; r += WS_H / 32) {
        float s = 0.f;
        for (int k = lane; k < WS_H; k += 32) s = fmaf(h2[r * WS_H + k], __bfloat162float(w.w3[k]), s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[r] = s + w.b3[0];
    }
    __syncthreads();
}

PD_D void load_tile(const __nv_bfloat16* __restrict__ F, int64_t r0, int nrow, float* x) {
    for (int t = threadIdx.x; t < WS_TILE * WS_IN; t += WS_H) {
        const int r = t / WS_IN;
        x[t] = r < nrow ? __bfloat162float(F[(r0 + r) * WS_IN + (t - r * WS_IN)]) : 0.f;
    }
}

__global__ void __launch_bounds__(WS_H) k_mlp_forward(MlpW w, const __nv_bfloat16* __restrict__ F, int64_t n,
                                                      float* __restrict__ y) {
    __shared__ float x[WS_TILE * WS_IN];
    __shared__ float h1[WS_TILE * WS_H];
    __shared__ float h2[WS_TILE * WS_H];
    __shared__ float out[WS_TILE];
    for (int64_t r0 = (int64_t)blockIdx.x * WS_TILE; r0 < n; r0 += (int64_t)gridDim.x * WS_TILE) {
        const int nrow = (int)min((int64_t)WS_TILE, n - r0);
        __syncthreads();
        load_tile(F, r0, nrow, x);
        __syncthreads();
        tile_forward(w, x, h1, h2, out, nrow);
        if (threadIdx.x < nrow) y[r0 + threadIdx.x] = out[threadIdx.x];
    }
}

// Loss sum(mask * (y - t)^2) / sum(mask) and its gradients; every block sums
// its tiles' gradients into its own row of `part` (WS_NPARAMS floats + 2:
// loss sum, mask sum), reduced afterwards in a fixed order.
__global__ void __launch_bounds__(WS_H) k_mlp_backward(MlpW w, const __nv_bfloat16* __restrict__ F,
                                                       const float* __restrict__ tgt, const float* __restrict__ mask,
                                                       int64_t n, float inv_norm, float* __restrict__ part) {
    extern __shared__ float sm[];
    float* x = sm;                            // WS_TILE * WS_IN
    float* h1 = x + WS_TILE * WS_IN;          // WS_TILE * WS_H
    float* h2 = h1 + WS_TILE * WS_H;          // WS_TILE * WS_H (becomes delta2)
    float* out = h2 + WS_TILE * WS_H;         // WS_TILE (becomes delta3)
    float* gW1 = out + WS_TILE;               // WS_IN * WS_H
    float* gW2 = gW1 + WS_IN * WS_H;          // WS_H * WS_H
    float* gsm = gW2 + WS_H * WS_H;           // b1, b2, w3 (3 * WS_H), b3, loss, mask
    const int j = threadIdx.x;
    for (int t = j; t < WS_IN * WS_H; t += WS_H) gW1[t] = 0.f;
    for (int t = j; t < WS_H * WS_H; t += WS_H) gW2[t] = 0.f;
    for (int t = j; t < 3 * WS_H + 3; t += WS_H) gsm[t] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f;
    for (int64_t r0 = (int64_t)blockIdx.x * WS_TILE; r0 < n; r0 += (int64_t)gridDim.x * WS_TILE) {
        const int nrow = (int)min((int64_t)WS_TILE, n - r0);
        __syncthreads();
        load_tile(F, r0, nrow, x);
        __syncthreads();
        tile_forward(w, x, h1, h2, out, nrow);
        // delta3 = 2 mask (y - t) / norm
        if (j < WS_TILE) {
            float d = 0.f;
            if (j < nrow) {
                const float e = out[j] - tgt[r0 + j];
                const float mk = mask[r0 + j];
                d = 2.f * mk * e * inv_norm;
                atomicAdd(&gsm[3 * WS_H + 1], mk * e * e);
                atomicAdd(&gsm[3 * WS_H + 2], mk);
                atomicAdd(&gsm[3 * WS_H], d);
            }
            out[j] = d;
        }
        __syncthreads();
        // w3, then delta2 = delta3 * w3 * relu'(h2) (in place of h2)
        const float w3j = __bfloat162float(w.w3[j]);
#pragma unroll 4
        for (int r = 0; r < WS_TILE; r++) {
            const float hv = h2[r * WS_H + j];
            gw3 = fmaf(hv, out[r], gw3);
            const float d2 = hv > 0.f ? out[r] * w3j : 0.f;
            h2[r * WS_H + j] = d2;
            gb2 += d2;
        }
        __syncthreads();
        // gW2[k][j] += sum_r h1[r][k] delta2[r][j]; delta1[r][j] = sum_t delta2[r][t] W2[j][t] relu'(h1[r][j])
        for (int k = 0; k < WS_H; k++) {
            float s = 0.f;
#pragma unroll 4
            for (int r = 0; r < WS_TILE; r++) s = fmaf(h1[r * WS_H + k], h2[r * WS_H + j], s);
            gW2[k * WS_H + j] += s;
        }
        float d1[WS_TILE];
#pragma unroll
        for (int r = 0; r < WS_TILE; r++) d1[r] = 0.f;
        for (int t = 0; t < WS_H; t++) {
            const float wjt = __bfloat162float(w.W2[j * WS_H + t]);
#pragma unroll
            for (int r = 0; r < WS_TILE; r++) d1[r] = fmaf(h2[r * WS_H + t], wjt, d1[r]);
        }
        __syncthreads();  // h1 is overwritten by delta1 below
#pragma unroll
        for (int r = 0; r < WS_TILE; r++) {
            const float v = h1[r * WS_H + j] > 0.f ? d1[r] : 0.f;
            h1[r * WS_H + j] = v;
            gb1 += v;
        }
        __syncthreads();
        // gW1[k][j] += sum_r x[r][k] delta1[r][j]
        for (int k = 0; k < WS_IN; k++) {
            float s = 0.f;
#pragma unroll 4
            for (int r = 0; r < WS_TILE; r++) s = fmaf(x[r * WS_IN + k], h1[r * WS_H + j], s);
            gW1[k * WS_H + j] += s;
        }
    }
    gsm[j] = gb1;
    gsm[WS_H + j] = gb2;
    gsm[2 * WS_H + j] = gw3;
    __syncthreads();
    // layout of a gradient row: W1, b1, W2, b2, w3, b3, then loss sum, mask sum
    float* row = part + (int64_t)blockIdx.x * WS_PART;
    for (int t = j; t < WS_IN * WS_H; t += WS_H) row[WS_OFF_W1 + t] = gW1[t];
    for (int t = j; t < WS_H * WS_H; t += WS_H) row[WS_OFF_W2 + t] = gW2[t];
    row[WS_OFF_B1 + j] = gsm[j];
    row[WS_OFF_B2 + j] = gsm[WS_H + j];
    row[WS_OFF_W3 + j] = gsm[2 * WS_H + j];
    if (j == 0) {
        row[WS_OFF_B3] = gsm[3 * WS_H];
        row[WS_NPARAMS] = gsm[3 * WS_H + 1];
        row[WS_NPARAMS + 1] = gsm[3 * WS_H + 2];
    }
}

// Sum of the blocks' rows, in block order.
__global__ void k_reduce_parts(const float* __restrict__ part, int nb, float* __restrict__ g) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= WS_PART) return;
    float s = 0.f;
    for (int b = 0; b < nb; b++) s += part[(int64_t)b * WS_PART + t];
    g[t] = s;
}

// Adam on the float32 master weights; bf16 copies of the weight matrices.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ wb) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= WS_NPARAMS) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    const float pt = p[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    p[t] = pt;
    wb[t] = __float2bfloat16(pt);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < WS_NPARAMS) wb[t] = __float2bfloat16(p[t]);
}

// Rows idx[0..n) of the data set (features, targets, mask) into a batch.
__global__ void k_gather_rows(const __nv_bfloat16* __restrict__ F, const float* __restrict__ T,
                              const float* __restrict__ M, const int32_t* __restrict__ idx, int64_t n,
                              __nv_bfloat16* __restrict__ Fo, float* __restrict__ To, float* __restrict__ Mo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * WS_IN) return;
    const int64_t r = t / WS_IN, k = t - r * WS_IN;
    const int64_t src = idx[r];
    Fo[t] = F[src * WS_IN + k];
    if (k == 0) {
        To[r] = T[src];
        Mo[r] = M[src];
    }
}

// Outputs in cost units: times the coarse cell (scale > 0) or the box's side.
__global__ void k_scale_out(const float* __restrict__ y, int64_t n, const long long* __restrict__ box,
                            int64_t scale, float* __restrict__ p) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    const long long ext = scale > 0 ? (long long)scale : max(max(box[2] - box[0], box[3] - box[1]), 1LL);
    p[r] = r < n ? y[r] * (float)ext : 0.f;  // row n: the diagonal node, potential 0
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static Ctx* owner(Ctx* c) { return c->mlp_owner ? c->mlp_owner : c; }

static MlpW weights_of(Ctx* c) {
    c = owner(c);
    const __nv_bfloat16* wb = (const __nv_bfloat16*)c->ptr[B_MLP_WB];
    const float* p = (const float*)c->ptr[B_MLP_P];
    // biases are read in float32 from the master copy; matrices in bf16
    return MlpW{wb + WS_OFF_W1, p + WS_OFF_B1, wb + WS_OFF_W2, p + WS_OFF_B2, wb + WS_OFF_W3, p + WS_OFF_B3};
}

static size_t backward_smem() {
    return sizeof(float) * (WS_TILE * WS_IN + 2 * WS_TILE * WS_H + WS_TILE + WS_IN * WS_H + WS_H * WS_H + 3 * WS_H + 3);
}

// Parameters: allocated and initialised once per context (hidden layers
// He-uniform from a SplitMix64 stream of `seed`, output layer and biases 0).
pd_status mlp_init(Ctx* c, uint64_t seed, bool force, cudaStream_t st) {
    if (c->mlp_ready && !force) return PD_OK;
    float* p = bufT<float>(c, B_MLP_P, WS_NPARAMS);
    float* m = bufT<float>(c, B_MLP_M, WS_NPARAMS);
    float* v = bufT<float>(c, B_MLP_V, WS_NPARAMS);
    __nv_bfloat16* wb = bufT<__nv_bfloat16>(c, B_MLP_WB, WS_NPARAMS);
    if (!p || !m || !v || !wb) return PD_ENOMEM;
    std::vector<float> h(WS_NPARAMS, 0.f);
    uint64_t z = seed;
    auto unif = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    const double a1 = std::sqrt(6.0 / WS_IN), a2 = std::sqrt(6.0 / WS_H);
    for (int t = 0; t < WS_IN * WS_H; t++) h[WS_OFF_W1 + t] = (float)(a1 * unif());
    for (int t = 0; t < WS_H * WS_H; t++) h[WS_OFF_W2 + t] = (float)(a2 * unif());
    // the output layer starts at 0: the untrained network predicts no
    // correction, so the start is the coarse solve's until training moves it
    PD_TRY(mlp_set(c, h.data(), st));
    c->mlp_steps = 0;
    return PD_OK;
}

pd_status mlp_set(Ctx* c, const float* host, cudaStream_t st) {
    float* p = bufT<float>(c, B_MLP_P, WS_NPARAMS);
    float* m = bufT<float>(c, B_MLP_M, WS_NPARAMS);
    float* v = bufT<float>(c, B_MLP_V, WS_NPARAMS);
    __nv_bfloat16* wb = bufT<__nv_bfloat16>(c, B_MLP_WB, WS_NPARAMS);
    if (!p || !m || !v || !wb) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemcpyAsync(p, host, sizeof(float) * WS_NPARAMS, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(m, 0, sizeof(float) * WS_NPARAMS, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(v, 0, sizeof(float) * WS_NPARAMS, st));
    k_to_bf16<<<grid_for(WS_NPARAMS, 256), 256, 0, st>>>(p, wb); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    c->mlp_ready = true;
    c->mlp_steps = 0;
    return PD_OK;
}

pd_status mlp_get(Ctx* c, float* host, cudaStream_t st) {
    if (!c->mlp_ready) return fail(c, PD_EINVAL, "the warm-start network has no parameters yet");
    PD_TRY_CUDA(c, cudaMemcpyAsync(host, c->ptr[B_MLP_P], sizeof(float) * WS_NPARAMS, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    return PD_OK;
}

pd_status mlp_forward(Ctx* c, const __nv_bfloat16* F, int64_t n, float* y, cudaStream_t st) {
    if (!owner(c)->mlp_ready) return fail(c, PD_EINVAL, "the warm-start network has no parameters yet");
    if (n <= 0) return PD_OK;
    const int64_t tiles = (n + WS_TILE - 1) / WS_TILE;
    const int grid = (int)std::min<int64_t>(tiles, 4 * std::max(c->sm_count, 1));
    k_mlp_forward<<<grid, WS_H, 0, st>>>(weights_of(c), F, n, y); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    return PD_OK;
}

// Loss and gradients of rows [0, n) into g (device, WS_PART floats: the
// WS_NPARAMS gradients, loss sum, mask sum).
pd_status mlp_grad(Ctx* c, const __nv_bfloat16* F, const float* t, const float* mask, int64_t n, float inv_norm,
                   float* g, cudaStream_t st) {
    if (!c->mlp_ready) return fail(c, PD_EINVAL, "the warm-start network has no parameters yet");
    const int64_t tiles = std::max<int64_t>((n + WS_TILE - 1) / WS_TILE, 1);
    const int nb = (int)std::min<int64_t>(tiles, std::max(c->sm_count, 1));
    float* part = bufT<float>(c, B_MLP_PART, (int64_t)nb * WS_PART);
    if (!part) return PD_ENOMEM;
    const size_t smem = backward_smem();
    PD_TRY_CUDA(c, cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_backward<<<nb, WS_H, smem, st>>>(weights_of(c), F, t, mask, n, inv_norm, part); pd::count_launch();
    k_reduce_parts<<<grid_for(WS_PART, 256), 256, 0, st>>>(part, nb, g); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    return PD_OK;
}

pd_status mlp_adam(Ctx* c, const float* g, float lr, cudaStream_t st) {
    c->mlp_steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)c->mlp_steps), c2 = 1.f - std::pow(b2, (float)c->mlp_steps);
    k_adam<<<grid_for(WS_NPARAMS, 256), 256, 0, st>>>((float*)c->ptr[B_MLP_P], (float*)c->ptr[B_MLP_M],
                                                       (float*)c->ptr[B_MLP_V], g, lr, b1, b2, 1e-8f, c1, c2,
                                                       (__nv_bfloat16*)c->ptr[B_MLP_WB]); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    return PD_OK;
}

pd_status mlp_gather_rows(Ctx* c, const int32_t* idx, int64_t n, __nv_bfloat16** F, float** T, float** M,
                          cudaStream_t st) {
    __nv_bfloat16* Fo = bufT<__nv_bfloat16>(c, B_WS_BF, std::max<int64_t>(n, 1) * WS_IN);
    float* To = bufT<float>(c, B_WS_BT, std::max<int64_t>(n, 1));
    float* Mo = bufT<float>(c, B_WS_BM, std::max<int64_t>(n, 1));
    if (!Fo || !To || !Mo) return PD_ENOMEM;
    if (n > 0) {
        k_gather_rows<<<grid_for(n * WS_IN, 256), 256, 0, st>>>((const __nv_bfloat16*)c->ptr[B_WS_DF],
                                                                 (const float*)c->ptr[B_WS_DT],
                                                                 (const float*)c->ptr[B_WS_DM], idx, n, Fo, To, Mo); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
    }
    *F = Fo;
    *T = To;
    *M = Mo;
    return PD_OK;
}

// Master parameters to the snapshot (restore false) or back from it, with
// the bf16 copies and the optimiser state left as they are.
pd_status mlp_snapshot(Ctx* c, bool restore, cudaStream_t st) {
    float* p = (float*)c->ptr[B_MLP_P];
    float* b = bufT<float>(c, B_MLP_BEST, WS_NPARAMS);
    if (!p || !b) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemcpyAsync(restore ? p : b, restore ? b : p, sizeof(float) * WS_NPARAMS,
                                   cudaMemcpyDeviceToDevice, st));
    if (restore) {
        k_to_bf16<<<grid_for(WS_NPARAMS, 256), 256, 0, st>>>(p, (__nv_bfloat16*)c->ptr[B_MLP_WB]); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
    }
    return PD_OK;
}

// Mean squared error (over the masked rows) of data-set rows [r0, r1).
pd_status mlp_loss(Ctx* c, int64_t r0, int64_t r1, double* loss, cudaStream_t st) {
    float* g = bufT<float>(c, B_MLP_G, WS_PART);
    if (!g) return PD_ENOMEM;
    const __nv_bfloat16* F = (const __nv_bfloat16*)c->ptr[B_WS_DF];
    const float* T = (const float*)c->ptr[B_WS_DT];
    const float* M = (const float*)c->ptr[B_WS_DM];
    double ls = 0.0, ms = 0.0;
    for (int64_t a = r0; a < r1; a += 2048) {
        const int64_t nb = std::min<int64_t>(2048, r1 - a);
        PD_TRY(mlp_grad(c, F + a * WS_IN, T + a, M + a, nb, 1.f, g, st));
        float lm[2];
        PD_TRY_CUDA(c, cudaMemcpyAsync(lm, g + WS_NPARAMS, sizeof(lm), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        ls += lm[0];
        ms += lm[1];
    }
    *loss = ms > 0.0 ? ls / ms : 0.0;
    return PD_OK;
}

// Features of a prepared transportation instance (rows: its sources then its
// sinks), written to F (device, (nS + nT) x WS_IN bf16); box (device, 4).
pd_status ws_features(Ctx* c, const pd_nodes& nodes, const W1Prep& w, __nv_bfloat16* F, long long* box,
                      cudaStream_t st) {
    const int64_t N = nodes.n_nodes;
    float* grid = bufT<float>(c, B_WS_GRID, WS_GRID * WS_GRID);
    if (!grid) return PD_ENOMEM;
    const long long init[4] = {LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN};
    std::memcpy(c->h_small + 24, init, sizeof(init));
    PD_TRY_CUDA(c, cudaMemcpyAsync(box, c->h_small + 24, sizeof(init), cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(grid, 0, sizeof(float) * WS_GRID * WS_GRID, st));
    if (N > 0) {
        k_box<<<grid_for(N, 256), 256, 0, st>>>(nodes.X, nodes.Y, N, box); pd::count_launch();
        k_grid<<<grid_for(N, 256), 256, 0, st>>>(nodes.X, nodes.Y, nodes.cntA, nodes.cntB, N, box, grid); pd::count_launch();
    }
    // the coarse solve's envelope gaps and cell, when one ran on this context for this instance
    const int64_t Gc = c->last_coarse_cell;
    const double* gap = Gc > 0 ? (const double*)c->ptr[B_CO_GAP] : nullptr;
    if (w.nS + w.nT > 0)
        k_features<<<grid_for(w.nS + w.nT, 128), 128, 0, st>>>(nodes.X, nodes.Y, nodes.cntA, nodes.cntB, w.S, w.T,
                                                                w.nS, w.nT, box, grid, gap, Gc, F); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));  // h_small + 24 is reused
    return PD_OK;
}

// Predicted potentials (host, nS + nT + 1 floats, cost units, the diagonal
// node last at 0) of a prepared transportation instance.
pd_status ws_predict(Ctx* c, const pd_nodes& nodes, const W1Prep& w, std::vector<float>* p, cudaStream_t st) {
    const int64_t n = w.nS + w.nT;
    __nv_bfloat16* F = bufT<__nv_bfloat16>(c, B_WS_FEAT, std::max<int64_t>(n, 1) * WS_IN);
    float* y = bufT<float>(c, B_WS_Y, n + 1);
    float* ps = bufT<float>(c, B_WS_PS, n + 1);
    long long* box = bufT<long long>(c, B_WS_BOX, 4);
    if (!F || !y || !ps || !box) return PD_ENOMEM;
    PD_TRY(ws_features(c, nodes, w, F, box, st));
    PD_TRY(mlp_forward(c, F, n, y, st));
    k_scale_out<<<grid_for(n + 1, 256), 256, 0, st>>>(y, n, box, c->last_coarse_cell, ps); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    p->resize((size_t)(n + 1));
    PD_TRY_CUDA(c, cudaMemcpyAsync(p->data(), ps, sizeof(float) * (n + 1), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    return PD_OK;
}

// Training rows of one solved pair appended to the context's data set: the
// instance's features and the targets from the solved record d_res.
pd_status ws_collect(Ctx* c, const pd_nodes& nodes, const W1Prep& w, const NSInst* d_res, const NSInst& r,
                     int64_t cmax, const std::vector<double>* base, cudaStream_t st) {
    const int64_t n = w.nS + w.nT;
    if (n <= 0) return PD_OK;
    const int64_t have = c->ws_rows;
    if (have + n > c->ws_cap) return fail(c, PD_ECAPACITY, "training rows exceed the reserved data set");
    __nv_bfloat16* F = (__nv_bfloat16*)c->ptr[B_WS_DF];
    float* T = (float*)c->ptr[B_WS_DT];
    float* M = (float*)c->ptr[B_WS_DM];
    if (!F || !T || !M) return fail(c, PD_EINVAL, "no training data set reserved");
    long long* box = bufT<long long>(c, B_WS_BOX, 4);
    if (!box) return PD_ENOMEM;
    PD_TRY(ws_features(c, nodes, w, F + have * WS_IN, box, st));
    const int32_t root = (int32_t)(w.nt);  // the simplex root follows the transportation nodes
    int32_t* comp = bufT<int32_t>(c, B_WS_COMP, n);
    int32_t* csize = bufT<int32_t>(c, B_WS_CSIZE, root + 1);
    unsigned long long* sum = bufT<unsigned long long>(c, B_WS_CSUM, 1);
    if (!comp || !csize || !sum) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(csize, 0, sizeof(int32_t) * (root + 1), st));
    PD_TRY_CUDA(c, cudaMemsetAsync(sum, 0, sizeof(unsigned long long), st));
    k_components<<<grid_for(n, 256), 256, 0, st>>>(r.parent, n, root, comp, csize); pd::count_launch();
    std::vector<int32_t> hs((size_t)(root + 1));
    PD_TRY_CUDA(c, cudaMemcpyAsync(hs.data(), csize, sizeof(int32_t) * (root + 1), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    const int32_t anchor = (int32_t)(std::max_element(hs.begin(), hs.end()) - hs.begin());
    k_component_sum<<<grid_for(n, 256), 256, 0, st>>>(r.pi, comp, n, anchor, sum); pd::count_launch();
    unsigned long long hsum = 0;
    PD_TRY_CUDA(c, cudaMemcpyAsync(&hsum, sum, sizeof(hsum), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    const double mean = (double)(int64_t)hsum / (double)std::max(hs[(size_t)anchor], 1);
    // base potentials: the network learns the correction to them
    double* db = nullptr;
    double bmean = 0.0;
    if (base && (int64_t)base->size() >= n) {
        std::vector<int32_t> hc((size_t)n);
        PD_TRY_CUDA(c, cudaMemcpyAsync(hc.data(), comp, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        int64_t cnt = 0;
        for (int64_t v = 0; v < n; v++)
            if (hc[(size_t)v] == anchor) {
                bmean += (*base)[(size_t)v];
                cnt++;
            }
        bmean = cnt ? bmean / (double)cnt : 0.0;
        db = bufT<double>(c, B_CO_P2, n);
        if (!db) return PD_ENOMEM;
        PD_TRY_CUDA(c, cudaMemcpyAsync(db, base->data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    }
    k_targets<<<grid_for(n, 256), 256, 0, st>>>(r.pi, comp, n, anchor, mean, db, bmean, box,
                                                db ? c->last_coarse_cell : 0, T + have, M + have); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));  // the base copy's host memory belongs to the caller
    (void)d_res;
    (void)cmax;
    c->ws_rows = have + n;
    return PD_OK;
}

}  // namespace pd

// ---------------------------------------------------------------------------
// C ABI of the network
// ---------------------------------------------------------------------------

using namespace pd;

static_assert(PD_WS_NPARAMS == WS_NPARAMS && PD_WS_NFEAT == WS_IN, "warm-start layout differs from the header");

extern "C" pd_status pd_ws_get_params(pd_ctx* cx, float* params) {
    Ctx* c = cx;
    if (!c || !params) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    return mlp_get(c, params, 0);
}

extern "C" pd_status pd_ws_set_params(pd_ctx* cx, const float* params) {
    Ctx* c = cx;
    if (!c || !params) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    return mlp_set(c, params, 0);
}

// Host feature rows -> bf16 device rows in B_WS_IN.
static pd_status upload_rows(Ctx* c, const float* feats, int64_t n, __nv_bfloat16** out, cudaStream_t st) {
    std::vector<__nv_bfloat16> hb((size_t)(n * WS_IN));
    for (int64_t t = 0; t < n * WS_IN; t++) hb[(size_t)t] = __float2bfloat16(feats[t]);
    __nv_bfloat16* F = bufT<__nv_bfloat16>(c, B_WS_IN, std::max<int64_t>(n, 1) * WS_IN);
    if (!F) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemcpyAsync(F, hb.data(), sizeof(__nv_bfloat16) * n * WS_IN, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));  // hb is freed on return
    *out = F;
    return PD_OK;
}

extern "C" pd_status pd_ws_forward(pd_ctx* cx, const float* feats, int64_t n, float* y, void* stream) {
    Ctx* c = cx;
    if (!c || n < 0 || (n > 0 && (!feats || !y))) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return PD_OK;
    __nv_bfloat16* F;
    PD_TRY(upload_rows(c, feats, n, &F, st));
    float* dy = bufT<float>(c, B_WS_Y, n);
    if (!dy) return PD_ENOMEM;
    PD_TRY(mlp_forward(c, F, n, dy, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(y, dy, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    return PD_OK;
}

extern "C" pd_status pd_ws_grad(pd_ctx* cx, const float* feats, const float* target, const float* mask, int64_t n,
                                float* grad, float* loss, void* stream) {
    Ctx* c = cx;
    if (!c || n <= 0 || !feats || !target || !grad) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    __nv_bfloat16* F;
    PD_TRY(upload_rows(c, feats, n, &F, st));
    float* dt = bufT<float>(c, B_WS_TIN, n);
    float* dm = bufT<float>(c, B_WS_MIN, n);
    float* g = bufT<float>(c, B_MLP_G, WS_PART);
    if (!dt || !dm || !g) return PD_ENOMEM;
    std::vector<float> ones;
    if (!mask) {
        ones.assign((size_t)n, 1.f);
        mask = ones.data();
    }
    PD_TRY_CUDA(c, cudaMemcpyAsync(dt, target, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(dm, mask, sizeof(float) * n, cudaMemcpyHostToDevice, st));
    PD_TRY(mlp_grad(c, F, dt, dm, n, 1.f / (float)n, g, st));
    std::vector<float> hg(WS_PART);
    PD_TRY_CUDA(c, cudaMemcpyAsync(hg.data(), g, sizeof(float) * WS_PART, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    std::memcpy(grad, hg.data(), sizeof(float) * WS_NPARAMS);
    if (loss) *loss = hg[WS_NPARAMS] / (float)n;
    return PD_OK;
}

static const char WS_MAGIC[8] = {'P', 'D', 'W', 'S', '0', '0', '0', '1'};

extern "C" pd_status pd_ws_save(pd_ctx* cx, const char* path) {
    Ctx* c = cx;
    if (!c || !path) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    std::vector<float> p(WS_NPARAMS);
    PD_TRY(mlp_get(c, p.data(), 0));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(c, PD_EINVAL, std::string("cannot open ") + path);
    const int64_t n = WS_NPARAMS;
    bool ok = fwrite(WS_MAGIC, 1, 8, f) == 8 && fwrite(&n, sizeof(n), 1, f) == 1 &&
              fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? PD_OK : fail(c, PD_EINVAL, std::string("cannot write ") + path);
}

extern "C" pd_status pd_ws_load(pd_ctx* cx, const char* path) {
    Ctx* c = cx;
    if (!c || !path) return PD_EINVAL;
    c->err.clear();
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(c, PD_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int64_t n = 0;
    std::vector<float> p(WS_NPARAMS);
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, WS_MAGIC, 8) == 0 && fread(&n, sizeof(n), 1, f) == 1 &&
              n == WS_NPARAMS && fread(p.data(), sizeof(float), p.size(), f) == p.size();
    fclose(f);
    if (!ok) return fail(c, PD_EINVAL, std::string("not a warm-start parameter file: ") + path);
    return mlp_set(c, p.data(), 0);
}
