// Nearest-neighbour search of one diagram in a database of diagrams (the
// NN-search application of the experiments section): the answer is the
// database diagram with the smallest approximate W1 (Algorithm 4's optimum
// OPT_int, ties to the lowest index).  Pairs are solved in ascending order of
// a lower bound on OPT_int, a wave of pairs at a time through the batched
// solve, and a pair whose bound exceeds the best optimum found is skipped.
//
// The bounds.  RWMD (Algorithm 1) of the 0-condensed diagrams is a lower
// bound on the real W1 of the pair, and so is half the word centroid distance
// of A + B~ against B + A~ (Appendix, WCD; ~ = diagonal projections), which
// reduces to |T_A - T_B| / (2 sqrt 2) with T the total persistence sum
// (d - b): each point minus its projection is (b - d, d - b) / 2.
// delta-condensation (Algorithm 2) moves every point by at most
// sqrt(2) (G/2 + P) <= delta / sqrt(2), which by the choice of delta totals at
// most eps_c * L_lo <= eps_c * W1 (eps_c = 8 / (s - 4)), and OPT_int, with
// costs rounded up on a network whose paths are never shorter than the direct
// routes, is at least the real W1 of the condensed diagrams.  Hence
// OPT_int >= (1 - eps_c) max(RWMD, WCD / 2).  The RWMD only has to be a valid
// lower bound, so it is computed in float32 over all database nodes at once,
// every distance shrunk by 2^-20 to cover rounding; the WCD comes from exact
// integer persistence sums (one per database diagram, summed at build time).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "prims.cuh"

namespace pd {

constexpr int LB_THREADS = 256;
constexpr int LB_R = 4;          // nodes per thread
constexpr int LB_TILE = 2048;    // nodes of the other side staged in shared memory
constexpr float LB_SHRINK = 1.0f - 1.0f / 1048576.0f;
constexpr float LB_INV_SQRT2 = 0.70710677f;  // below 1/sqrt(2)

// Coordinates below 2^23 in magnitude are exact in float32, and so are their
// differences; larger ones (up to the 2^29 input limit) can be off by at most
// 64 quanta per axis after conversion and subtraction, covered by an absolute
// margin of LB_MARGIN quanta taken off every distance.
constexpr float LB_MARGIN = 128.0f;
constexpr int32_t LB_EXACT = 1 << 23;

// Destruction / creation cost of a unit at (x, y), rounded down: kappa times
// the distance to the diagonal plus tau (tau_lo: tau rounded down to float).
PD_D float diag_lb(float2 p, float margin, int kappa, float tau_lo) {
    return (kappa ? fmaxf(fabsf(p.y - p.x) * LB_INV_SQRT2 * LB_SHRINK - margin, 0.f) : 0.f) + tau_lo;
}

PD_D float dist_lb(float m2, float margin) { return fmaxf(sqrtf(m2) * LB_SHRINK - margin, 0.f); }

// 0-condensed nodes of one diagram (int32 X, Y, int64 count) -> packed float
// coordinates, int32 counts and the diagram's id, at offset `at`.
// big: set to 1 if a coordinate is not exact in float32 arithmetic.
__global__ void k_db_pack(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                          const int64_t* __restrict__ cnt, int64_t n, int32_t id, int64_t at,
                          float2* __restrict__ xy, int32_t* __restrict__ c, int32_t* __restrict__ ids,
                          int32_t* __restrict__ big) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t x = X[i], y = Y[i];
    xy[at + i] = make_float2((float)x, (float)y);
    c[at + i] = (int32_t)cnt[i];
    if (ids) ids[at + i] = id;
    if (x >= LB_EXACT || x <= -LB_EXACT || y >= LB_EXACT || y <= -LB_EXACT) *big = 1;
}

// Total persistence sum cnt * (Y - X) of a diagram's 0-condensed nodes into
// *out (two's-complement 64-bit sums: exact and order-free).
__global__ void k_pers_sum(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                           const int64_t* __restrict__ cnt, int64_t n, unsigned long long* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long v = i < n ? (long long)cnt[i] * ((long long)Y[i] - X[i]) : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(out, (unsigned long long)v);
}

// Staging (raw offsets, id -1 in the gaps) -> compact store.
__global__ void k_db_compact(const float2* __restrict__ sxy, const int32_t* __restrict__ sc,
                             const int32_t* __restrict__ sid, int64_t n, const int64_t* __restrict__ roff,
                             const int64_t* __restrict__ off, float2* __restrict__ xy, int32_t* __restrict__ c,
                             int32_t* __restrict__ ids) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int32_t id = sid[t];
    if (id < 0) return;
    int64_t d = off[id] + (t - roff[id]);
    xy[d] = sxy[t];
    c[d] = sc[t];
    ids[d] = id;
}

// Database side: every database node v gets cnt(v) * min(d(v, query), d_diag(v)),
// its term of L_B of its diagram (summed per diagram by k_lb_segsum).
__global__ void __launch_bounds__(LB_THREADS) k_lb_db_side(const float2* __restrict__ dxy,
                                                           const int32_t* __restrict__ dcnt, int64_t T,
                                                           const float2* __restrict__ qxy, int64_t nq,
                                                           float margin, int kappa, float tau_lo,
                                                           double* __restrict__ val) {
    __shared__ float2 sq[LB_TILE];
    const int64_t base = (int64_t)blockIdx.x * (LB_THREADS * LB_R);
    float2 p[LB_R];
    float m[LB_R];
#pragma unroll
    for (int r = 0; r < LB_R; r++) {
        int64_t v = base + r * LB_THREADS + threadIdx.x;
        p[r] = v < T ? dxy[v] : make_float2(0.f, 0.f);
        m[r] = INFINITY;
    }
    for (int64_t t0 = 0; t0 < nq; t0 += LB_TILE) {
        int tn = (int)min((int64_t)LB_TILE, nq - t0);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += LB_THREADS) sq[j] = qxy[t0 + j];
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < tn; j++) {
            float2 q = sq[j];
#pragma unroll
            for (int r = 0; r < LB_R; r++) {
                float dx = q.x - p[r].x, dy = q.y - p[r].y;
                m[r] = fminf(m[r], fmaf(dx, dx, dy * dy));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < LB_R; r++) {
        int64_t v = base + r * LB_THREADS + threadIdx.x;
        if (v < T) val[v] = (double)dcnt[v] * (double)fminf(dist_lb(m[r], margin), diag_lb(p[r], margin, kappa, tau_lo));
    }
}

// Sum of the values of [off[i], off[i + 1]) for every diagram i (one block per
// diagram, a fixed order of additions: the same bits on every run).
__global__ void __launch_bounds__(LB_THREADS) k_lb_segsum(const double* __restrict__ val,
                                                          const int64_t* __restrict__ off, int64_t stride,
                                                          double* __restrict__ out) {
    __shared__ double red[LB_THREADS];
    const int64_t i = blockIdx.x;
    const int64_t b0 = stride > 0 ? i * stride : off[i];
    const int64_t b1 = stride > 0 ? b0 + stride : off[i + 1];
    double t = 0.0;
    for (int64_t v = b0 + threadIdx.x; v < b1; v += LB_THREADS) t += val[v];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = LB_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = red[0];
}

// Query side: blockIdx.y = database diagram i; every query node u adds
// cnt(u) * min(d(u, D_i), d_diag(u)) to the block's partial sum of L_A of
// diagram i, part[i * gridDim.x + blockIdx.x] (summed by k_lb_segsum).
__global__ void __launch_bounds__(LB_THREADS) k_lb_query_side(const float2* __restrict__ qxy,
                                                              const int32_t* __restrict__ qcnt, int64_t nq,
                                                              const float2* __restrict__ dxy,
                                                              const int64_t* __restrict__ doff, float margin,
                                                              int kappa, float tau_lo, double* __restrict__ part) {
    __shared__ float2 sd[LB_TILE];
    __shared__ double red[LB_THREADS / 32];
    const int32_t i = blockIdx.y;
    const int64_t d0 = doff[i], d1 = doff[i + 1];
    const int64_t base = (int64_t)blockIdx.x * (LB_THREADS * LB_R);
    float2 p[LB_R];
    float m[LB_R];
#pragma unroll
    for (int r = 0; r < LB_R; r++) {
        int64_t u = base + r * LB_THREADS + threadIdx.x;
        p[r] = u < nq ? qxy[u] : make_float2(0.f, 0.f);
        m[r] = INFINITY;
    }
    for (int64_t t0 = d0; t0 < d1; t0 += LB_TILE) {
        int tn = (int)min((int64_t)LB_TILE, d1 - t0);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += LB_THREADS) sd[j] = dxy[t0 + j];
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < tn; j++) {
            float2 q = sd[j];
#pragma unroll
            for (int r = 0; r < LB_R; r++) {
                float dx = q.x - p[r].x, dy = q.y - p[r].y;
                m[r] = fminf(m[r], fmaf(dx, dx, dy * dy));
            }
        }
    }
    double val = 0.0;
#pragma unroll
    for (int r = 0; r < LB_R; r++) {
        int64_t u = base + r * LB_THREADS + threadIdx.x;
        if (u < nq) val += (double)qcnt[u] * (double)fminf(dist_lb(m[r], margin), diag_lb(p[r], margin, kappa, tau_lo));
    }
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < LB_THREADS / 32; w++) t += red[w];
        part[(int64_t)i * gridDim.x + blockIdx.x] = t;
    }
}

}  // namespace pd

using namespace pd;

static float ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

extern "C" pd_status pd_db_build(pd_ctx* cx, const pd_diagram* dbs, int64_t n_db, const pd_opts* opts,
                                 void* stream) {
    Ctx* c = cx;
    if (!c) return PD_EINVAL;
    c->err.clear();
    if (n_db < 0 || (n_db > 0 && !dbs)) return fail(c, PD_EINVAL, "bad database arguments");
    if (n_db >= (int64_t(1) << 31)) return fail(c, PD_ECAPACITY, "more than 2^31 - 1 database diagrams");
    pd_opts o;
    pd_opts_default(&o);
    if (opts) o = *opts;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    c->db.clear();
    c->db_hats.clear();
    c->db_total = 0;
    const int dtype = n_db > 0 ? dbs[0].dtype : PD_F32;
    for (int64_t i = 0; i < n_db; i++) {
        PD_TRY(check_diag(c, dbs[i]));
        if (dbs[i].dtype != dtype) return fail(c, PD_EINVAL, "database diagrams differ in dtype");
    }
    const int k = o.coord_shift >= 0 ? o.coord_shift : default_shift(dtype);
    // staging at raw offsets (every diagram has at most as many nodes as points)
    std::vector<int64_t> roff((size_t)n_db + 1, 0), off((size_t)n_db + 1, 0), hats((size_t)n_db, 0);
    for (int64_t i = 0; i < n_db; i++) roff[(size_t)i + 1] = roff[(size_t)i] + dbs[i].n;
    const int64_t R = roff[(size_t)n_db];
    float2* sxy = bufT<float2>(c, B_DB_SXY, R);
    int32_t* sc = bufT<int32_t>(c, B_DB_SCNT, R);
    int32_t* sid = bufT<int32_t>(c, B_DB_SID, R);
    if (!sxy || !sc || !sid) return PD_ENOMEM;
    int32_t* big = bufT<int32_t>(c, B_DB_BIG, 2);
    unsigned long long* pers = bufT<unsigned long long>(c, B_DB_PERS, n_db + 1);
    if (!big || !pers) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(big, 0, sizeof(int32_t) * 2, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(pers, 0, sizeof(unsigned long long) * (n_db + 1), st));
    if (R > 0) PD_TRY_CUDA(c, cudaMemsetAsync(sid, 0xff, sizeof(int32_t) * R, st));
    const pd_diagram empty{nullptr, 0, dtype, 0};
    for (int64_t i = 0; i < n_db; i++) {
        DevDiag a, b;
        PD_TRY(stage_inputs(c, dbs[i], empty, &a, &b, st));
        Hats h;
        pd_status e = stage_condense0(c, a, b, k, &h, st);
        if (e != PD_OK) return fail(c, e, "database diagram " + std::to_string(i) + ": " + c->err);
        if (h.nA > 0) {
            k_db_pack<<<grid_for(h.nA, 256), 256, 0, st>>>(h.X, h.Y, h.cnt, h.nA, (int32_t)i, roff[(size_t)i], sxy, sc,
                                                             sid, big); pd::count_launch();
            k_pers_sum<<<grid_for(h.nA, 256), 256, 0, st>>>(h.X, h.Y, h.cnt, h.nA, pers + i); pd::count_launch();
        }
        PD_TRY_CUDA(c, cudaGetLastError());
        hats[(size_t)i] = h.nA;
    }
    for (int64_t i = 0; i < n_db; i++) off[(size_t)i + 1] = off[(size_t)i] + hats[(size_t)i];
    const int64_t T = off[(size_t)n_db];
    float2* xy = bufT<float2>(c, B_DB_XY, T);
    int32_t* cn = bufT<int32_t>(c, B_DB_CNT, T);
    int32_t* ids = bufT<int32_t>(c, B_DB_ID, T);
    int64_t* doff = bufT<int64_t>(c, B_DB_OFF, n_db + 1);
    int64_t* droff = bufT<int64_t>(c, B_DB_ROFF, n_db + 1);
    if (!xy || !cn || !ids || !doff || !droff) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (n_db + 1), cudaMemcpyHostToDevice, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(droff, roff.data(), sizeof(int64_t) * (n_db + 1), cudaMemcpyHostToDevice, st));
    if (R > 0) k_db_compact<<<grid_for(R, 256), 256, 0, st>>>(sxy, sc, sid, R, droff, doff, xy, cn, ids); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    int32_t hbig = 0;
    std::vector<int64_t> hp((size_t)n_db + 1);
    PD_TRY_CUDA(c, cudaMemcpyAsync(&hbig, big, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(hp.data(), pers, sizeof(int64_t) * (n_db + 1), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    c->db_big = hbig != 0;
    hp.resize((size_t)n_db);
    c->db_pers = hp;
    c->db.assign(dbs, dbs + n_db);
    c->db_hats = hats;
    c->db_total = T;
    c->db_k = k;
    c->db_dtype = dtype;
    return PD_OK;
}

extern "C" pd_status pd_nn_search(pd_ctx* cx, pd_diagram query, double eps, const pd_opts* opts,
                                  pd_nn_result* out, int64_t* opt_out, int64_t* lb_out, int64_t* wcd_out,
                                  void* stream) {
    Ctx* c = cx;
    if (!c || !out) return PD_EINVAL;
    c->err.clear();
    pd_opts o;
    pd_opts_default(&o);
    if (opts) o = *opts;
    if (!(eps > 0.0) && o.s_override <= 0) return fail(c, PD_EINVAL, "eps must be > 0 (or set s_override)");
    if (o.solver == 1) return fail(c, PD_EINVAL, "the search runs the network simplex only");
    if (o.nn_wave0 < 0) return fail(c, PD_EINVAL, "nn_wave0 must be >= 0");
    PD_TRY(check_diag_cost(c, o));
    PD_TRY(check_diag(c, query));
    const int64_t n_db = (int64_t)c->db.size();
    if (n_db > 0 && query.dtype != c->db_dtype) return fail(c, PD_EINVAL, "query dtype differs from the database");
    const int k = o.coord_shift >= 0 ? o.coord_shift : default_shift(query.dtype);
    if (n_db > 0 && k != c->db_k) return fail(c, PD_EINVAL, "coord_shift differs from the database build");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const auto t_all = std::chrono::steady_clock::now();
    pd_nn_result r;
    memset(&r, 0, sizeof(r));
    r.nn_index = -1;
    r.nn_opt_quanta = -1;
    r.coord_shift = k;
    if (n_db == 0) {
        *out = r;
        return PD_OK;
    }
    const int64_t s = o.s_override > 0 ? o.s_override : s_for_eps(eps);
    if (s < 1) return fail(c, PD_EINVAL, "no WSPD parameter s for this eps");
    // ---- lower bounds ----------------------------------------------------
    cudaEvent_t e0, e1;
    PD_TRY_CUDA(c, cudaEventCreate(&e0));
    PD_TRY_CUDA(c, cudaEventCreate(&e1));
    PD_TRY_CUDA(c, cudaEventRecord(e0, st));
    const pd_diagram empty{nullptr, 0, query.dtype, 0};
    DevDiag a, b;
    PD_TRY(stage_inputs(c, query, empty, &a, &b, st));
    Hats h;
    PD_TRY(stage_condense0(c, a, b, k, &h, st));
    const int64_t nq = h.nA;
    float2* qxy = bufT<float2>(c, B_Q_XY, nq);
    int32_t* qc = bufT<int32_t>(c, B_Q_CNT, nq);
    double* LA = bufT<double>(c, B_DB_LA, 2 * n_db);
    if (!qxy || !qc || !LA) return PD_ENOMEM;
    double* LB = LA + n_db;
    int32_t* big = bufT<int32_t>(c, B_DB_BIG, 2);
    unsigned long long* pers = bufT<unsigned long long>(c, B_DB_PERS, n_db + 1);
    if (!big || !pers) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(big + 1, 0, sizeof(int32_t), st));
    PD_TRY_CUDA(c, cudaMemsetAsync(pers + n_db, 0, sizeof(unsigned long long), st));
    if (nq > 0) {
        k_db_pack<<<grid_for(nq, 256), 256, 0, st>>>(h.X, h.Y, h.cnt, nq, 0, 0, qxy, qc, nullptr, big + 1); pd::count_launch();
        k_pers_sum<<<grid_for(nq, 256), 256, 0, st>>>(h.X, h.Y, h.cnt, nq, pers + n_db); pd::count_launch();
    }
    int32_t qbig = 0;
    int64_t qpers = 0;
    PD_TRY_CUDA(c, cudaMemcpyAsync(&qbig, big + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(&qpers, pers + n_db, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    const float margin = (qbig || c->db_big) ? LB_MARGIN : 0.f;
    const int64_t T = c->db_total;
    const int64_t per = (int64_t)LB_THREADS * LB_R;
    // tau in float rounded down, so every destruction cost stays a lower bound
    float tau_lo = (float)o.diag_tau;
    if ((double)tau_lo > (double)o.diag_tau) tau_lo = nextafterf(tau_lo, 0.f);
    const int64_t gq = (nq + per - 1) / per;  // query tiles: partial sums per diagram
    double* val = bufT<double>(c, B_DB_VAL, std::max<int64_t>(T, gq * n_db));
    if (!val) return PD_ENOMEM;
    // sums in a fixed order (no floating-point atomics): the bounds are the same bits on every run
    if (T > 0) {
        k_lb_db_side<<<(unsigned)((T + per - 1) / per), LB_THREADS, 0, st>>>(
            (const float2*)c->ptr[B_DB_XY], (const int32_t*)c->ptr[B_DB_CNT], T, qxy, nq, margin, o.diag_kappa,
            tau_lo, val);
        pd::count_launch();
    }
    k_lb_segsum<<<(unsigned)n_db, LB_THREADS, 0, st>>>(val, (const int64_t*)c->ptr[B_DB_OFF], 0, LB);
    pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    if (nq > 0) {
        for (int64_t y0 = 0; y0 < n_db; y0 += 65535) {
            const int64_t ny = std::min<int64_t>(65535, n_db - y0);
            k_lb_query_side<<<dim3((unsigned)gq, (unsigned)ny), LB_THREADS, 0, st>>>(
                qxy, qc, nq, (const float2*)c->ptr[B_DB_XY], (const int64_t*)c->ptr[B_DB_OFF] + y0, margin,
                o.diag_kappa, tau_lo, val + y0 * gq); pd::count_launch();
        }
        k_lb_segsum<<<(unsigned)n_db, LB_THREADS, 0, st>>>(val, nullptr, gq, LA);
        pd::count_launch();
    } else {
        PD_TRY_CUDA(c, cudaMemsetAsync(LA, 0, sizeof(double) * n_db, st));
    }
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaEventRecord(e1, st));
    std::vector<double> hl((size_t)(2 * n_db));
    PD_TRY_CUDA(c, cudaMemcpyAsync(hl.data(), LA, sizeof(double) * 2 * n_db, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    cudaEventElapsedTime(&r.lb_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // OPT_int >= (1 - eps_c) max(RWMD, WCD / 2); the last factor covers double rounding
    const double ec = o.condense ? (s >= 12 ? 8.0 / (double)(s - 4) : 1.0) : 0.0;
    std::vector<int64_t> lb((size_t)n_db), lbw((size_t)n_db);
    for (int64_t i = 0; i < n_db; i++) {
        double L = std::max(hl[(size_t)i], hl[(size_t)(n_db + i)]) * (1.0 - ec) * (1.0 - 1e-9);
        lb[(size_t)i] = L > 0.0 ? (int64_t)std::floor(L) : 0;
        // WCD / 2 = |T_q - T_i| / (2 sqrt(2)): the persistence sums are exact
        // integers; the double quotient is shrunk to cover its rounding
        // (only for persistence-diagram costs, kappa 1: W1 with tau >= 0 is at least the plain W1)
        const double dT = o.diag_kappa == 1 ? std::fabs((double)(qpers - c->db_pers[(size_t)i])) : 0.0;
        const double W = dT / (2.0 * std::sqrt(2.0)) * (1.0 - ec) * (1.0 - 1e-9);
        lbw[(size_t)i] = W > 0.0 ? (int64_t)std::floor(W) : 0;
        if (lbw[(size_t)i] > lb[(size_t)i]) {
            r.wcd_above++;
            lb[(size_t)i] = lbw[(size_t)i];
        }
    }
    // ---- waves in ascending bound ------------------------------------------
    std::vector<int64_t> order((size_t)n_db), opt((size_t)n_db, -1);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return lb[(size_t)x] < lb[(size_t)y]; });
    // waves grow from nn_wave0 pairs, doubling up to the batch size: the pairs
    // of smallest bound are solved first, so their optimum can prune the rest
    // before a wide wave is spent on pairs it would have ruled out
    const int64_t W = o.batch_slots > 0 ? o.batch_slots : 2 * std::max(c->sm_count, 1);
    int64_t wsize = std::min<int64_t>(W, o.nn_wave0 > 0 ? o.nn_wave0 : (o.nn_prune != 0 ? 16 : W));
    int64_t best = INT64_MAX, best_i = -1, pos = 0;
    std::vector<pd_diagram> qa, db;
    std::vector<pd_result> res;
    const auto t_solve = std::chrono::steady_clock::now();
    while (pos < n_db) {
        if (o.nn_prune != 0 && lb[(size_t)order[(size_t)pos]] > best) break;  // the rest are no better
        qa.clear();
        db.clear();
        std::vector<int64_t> wave;
        while (pos < n_db && (int64_t)wave.size() < wsize) {
            const int64_t i = order[(size_t)pos];
            if (o.nn_prune != 0 && lb[(size_t)i] > best) break;
            wave.push_back(i);
            qa.push_back(query);
            db.push_back(c->db[(size_t)i]);
            pos++;
        }
        res.assign(wave.size(), pd_result{});
        PD_TRY(batch_solve(c, qa.data(), db.data(), (int64_t)wave.size(), eps, o, res.data(), st));
        r.waves++;
        wsize = std::min<int64_t>(W, 2 * wsize);
        for (size_t q = 0; q < wave.size(); q++) {
            const int64_t i = wave[q], v = res[q].opt_quanta;
            opt[(size_t)i] = v;
            r.solved++;
            if (v < best || (v == best && i < best_i)) {
                best = v;
                best_i = i;
            }
        }
    }
    r.solve_ms = ms_since(t_solve);
    r.pruned = n_db - r.solved;
    r.nn_index = best_i;
    r.nn_opt_quanta = best;
    r.nn_w1 = std::ldexp((double)best, -k);
    r.total_ms = ms_since(t_all);
    if (opt_out) std::copy(opt.begin(), opt.end(), opt_out);
    if (lb_out) std::copy(lb.begin(), lb.end(), lb_out);
    if (wcd_out) std::copy(lbw.begin(), lbw.end(), wcd_out);
    *out = r;
    return PD_OK;
}
