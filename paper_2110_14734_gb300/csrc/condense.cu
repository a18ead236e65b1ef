// Quantisation, 0-condensation, RWMD (Algorithm 1) and delta-condensation
// (Algorithm 2) on the device.
#include "internal.h"
#include "prims.cuh"

#include <algorithm>
#include <cmath>

namespace pd {

// small-scalar slots in B_SMALL (int64)
enum : int {
    S_MNX = 0, S_MXX, S_MNY, S_MXY, S_FA, S_FB, S_ERR, S_NA, S_M, S_L0, S_L1,
    S_CMNX, S_CMXX, S_CMNY, S_CMXY, S_N, S_NMNX, S_NMXX, S_NMNY, S_NMXY, S_COUNT = 32
};

__global__ void k_init_small(int64_t* s) {
    int i = threadIdx.x;
    if (i < S_COUNT) {
        int64_t v = 0;
        if (i == S_MNX || i == S_MNY || i == S_CMNX || i == S_CMNY || i == S_NMNX || i == S_NMNY) v = INT64_MAX;
        if (i == S_MXX || i == S_MXY || i == S_CMXX || i == S_CMXY || i == S_NMXX || i == S_NMXY) v = INT64_MIN;
        s[i] = v;
    }
}

// a1: X = rint(b 2^k), Y = rint(d 2^k); keep unless X == Y; flag non-finite
// or |X|,|Y| >= 2^29; track min/max and the masses of A and B.
__global__ void k_quantize(const void* __restrict__ a, int64_t na, int dta, const void* __restrict__ b, int64_t nb,
                           int dtb, int k, int32_t* __restrict__ X, int32_t* __restrict__ Y,
                           uint8_t* __restrict__ keep, int64_t* __restrict__ sm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = na + nb;
    int64_t mnx = INT64_MAX, mxx = INT64_MIN, mny = INT64_MAX, mxy = INT64_MIN;
    int isB = 0, kp = 0, bad = 0;
    if (i < n) {
        isB = i >= na;
        int64_t j = isB ? i - na : i;
        const void* p = isB ? b : a;
        int dt = isB ? dtb : dta;
        int64_t qx, qy;
        if (dt == PD_F32) {
            float2 v = ((const float2*)p)[j];
            double fb = v.x, fd = v.y;
            double s = ldexp(1.0, k);
            if (!isfinite(fb) || !isfinite(fd)) {
                bad = 1;
                qx = qy = 0;
            } else {
                double rb = rint(fb * s), rd = rint(fd * s);
                if (fabs(rb) >= (double)COORD_LIMIT || fabs(rd) >= (double)COORD_LIMIT) {
                    bad = 1;
                    qx = qy = 0;
                } else {
                    qx = (int64_t)rb;
                    qy = (int64_t)rd;
                }
            }
        } else {
            uchar2 v = ((const uchar2*)p)[j];
            qx = (int64_t)v.x << k;
            qy = (int64_t)v.y << k;
            if (qx >= COORD_LIMIT || qy >= COORD_LIMIT) bad = 1;
        }
        kp = !bad && qx != qy;
        X[i] = (int32_t)qx;
        Y[i] = (int32_t)qy;
        keep[i] = (uint8_t)kp;
        if (kp) {
            mnx = mxx = qx;
            mny = mxy = qy;
        }
    }
    // warp-reduce then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mnx, o));
        mxx = max(mxx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mxx, o));
        mny = min(mny, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mny, o));
        mxy = max(mxy, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mxy, o));
    }
    unsigned ka = __ballot_sync(0xffffffffu, kp && !isB), kb = __ballot_sync(0xffffffffu, kp && isB);
    unsigned bd = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (ka | kb) {
            atomicMin((long long*)&sm[S_MNX], (long long)mnx);
            atomicMax((long long*)&sm[S_MXX], (long long)mxx);
            atomicMin((long long*)&sm[S_MNY], (long long)mny);
            atomicMax((long long*)&sm[S_MXY], (long long)mxy);
        }
        if (ka) atomicAdd((unsigned long long*)&sm[S_FA], (unsigned long long)__popc(ka));
        if (kb) atomicAdd((unsigned long long*)&sm[S_FB], (unsigned long long)__popc(kb));
        if (bd) atomicAdd((unsigned long long*)&sm[S_ERR], 1ull);
    }
}

// Sort key: diagram bit, then X, then Y (lexicographic); dropped points get
// the all-ones key so that they sort last.
__global__ void k_point_keys(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                             const uint8_t* __restrict__ keep, int64_t na, int64_t n, const int64_t* __restrict__ sm,
                             int bx, int by, uint64_t* __restrict__ key) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t sent = (bx + by + 2 >= 64) ? ~0ull : ((1ull << (bx + by + 2)) - 1);
    if (!keep[i]) {
        key[i] = sent;
        return;
    }
    uint64_t isB = i >= na;
    key[i] = (isB << (bx + by)) | ((uint64_t)(X[i] - sm[S_MNX]) << by) | (uint64_t)(Y[i] - sm[S_MNY]);
}

__global__ void k_run_flags(const uint64_t* __restrict__ key, int64_t n, uint64_t sent, int64_t* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key[i];
    flag[i] = (k != sent && (i == 0 || key[i - 1] != k)) ? 1 : 0;
}

// Node j of the 0-condensation starts at sorted position start[j].
__global__ void k_hat_compact(const uint64_t* __restrict__ key, int64_t n, uint64_t sent,
                              const int64_t* __restrict__ idx, const int64_t* __restrict__ sm, int bx, int by,
                              int32_t* __restrict__ HX, int32_t* __restrict__ HY, int64_t* __restrict__ start,
                              int64_t* __restrict__ nA) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key[i];
    if (k == sent || (i > 0 && key[i - 1] == k)) return;
    int64_t j = idx[i];
    uint64_t ymask = (by >= 64) ? ~0ull : ((1ull << by) - 1);
    uint64_t xmask = (bx >= 64) ? ~0ull : ((1ull << bx) - 1);
    HX[j] = (int32_t)((int64_t)((k >> by) & xmask) + sm[S_MNX]);
    HY[j] = (int32_t)((int64_t)(k & ymask) + sm[S_MNY]);
    start[j] = i;
    if (!((k >> (bx + by)) & 1ull)) atomicAdd((unsigned long long*)nA, 1ull);
}

__global__ void k_hat_counts(const int64_t* __restrict__ start, int64_t M, int64_t nvalid, int64_t* __restrict__ cnt) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int64_t e = (j + 1 < M) ? start[j + 1] : nvalid;
    cnt[j] = e - start[j];
}

pd_status stage_condense0(Ctx* c, const DevDiag& A, const DevDiag& B, int k, Hats* out, cudaStream_t st) {
    int64_t n = A.n + B.n;
    int64_t* sm = bufT<int64_t>(c, B_SMALL, 64);
    if (!sm) return PD_ENOMEM;
    k_init_small<<<1, 64, 0, st>>>(sm); pd::count_launch();
    out->nA = out->nB = out->FA = out->FB = 0;
    out->X = bufT<int32_t>(c, B_HAT_X, n);
    out->Y = bufT<int32_t>(c, B_HAT_Y, n);
    out->cnt = bufT<int64_t>(c, B_HAT_C, n);
    if (!out->X || !out->Y || !out->cnt) return PD_ENOMEM;
    if (n == 0) return PD_OK;
    int32_t* X = bufT<int32_t>(c, B_QX, n);
    int32_t* Y = bufT<int32_t>(c, B_QY, n);
    uint8_t* keep = bufT<uint8_t>(c, B_FLAG, n);
    uint64_t* key = bufT<uint64_t>(c, B_QKEY, n);
    uint64_t* key2 = bufT<uint64_t>(c, B_QKEY2, n);
    int64_t* flag = bufT<int64_t>(c, B_IDX, n);
    int64_t* start = bufT<int64_t>(c, B_QVAL, n);
    if (!X || !Y || !keep || !key || !key2 || !flag || !start) return PD_ENOMEM;
    k_quantize<<<grid_for(n, 256), 256, 0, st>>>(A.bd, A.n, A.dtype, B.bd, B.n, B.dtype, k, X, Y, keep, sm); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    int64_t* h = c->h_small;
    if (h[S_ERR]) return fail(c, PD_EINVAL, "diagram has a non-finite coordinate or |coordinate| * 2^k >= 2^29");
    out->FA = h[S_FA];
    out->FB = h[S_FB];
    int64_t nvalid = h[S_FA] + h[S_FB];
    if (nvalid == 0) return PD_OK;
    int bx = bits_for((uint64_t)(h[S_MXX] - h[S_MNX])), by = bits_for((uint64_t)(h[S_MXY] - h[S_MNY]));
    int kb = bx + by + 2;
    uint64_t sent = (kb >= 64) ? ~0ull : ((1ull << kb) - 1);
    k_point_keys<<<grid_for(n, 256), 256, 0, st>>>(X, Y, keep, A.n, n, sm, bx, by, key); pd::count_launch();
    PD_TRY(sort_u64(c, key, key2, nullptr, nullptr, n, kb, st));
    k_run_flags<<<grid_for(n, 256), 256, 0, st>>>(key, n, sent, flag); pd::count_launch();
    PD_TRY(scan_i64(c, flag, flag, n, sm + S_M, st));
    k_hat_compact<<<grid_for(n, 256), 256, 0, st>>>(key, n, sent, flag, sm, bx, by, out->X, out->Y, start,
                                                      sm + S_NA); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    int64_t M = h[S_M];
    out->nA = h[S_NA];
    out->nB = M - out->nA;
    k_hat_counts<<<grid_for(M, 256), 256, 0, st>>>(start, M, nvalid, out->cnt); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    return PD_OK;
}

// ---------------------------------------------------------------------------
// RWMD (Algorithm 1, with the diagonal option of the relaxed flow)
// ---------------------------------------------------------------------------

constexpr int RW_THREADS = 256;
constexpr int RW_TILE = 2048;

// Exact minimum squared distance from every node of one side to the nodes of
// the other side; blockIdx.y splits the other side, blockIdx.z = direction.
__global__ void __launch_bounds__(RW_THREADS) k_rwmd_min(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                                                         int64_t nA, int64_t nB, int64_t chunk,
                                                         unsigned long long* __restrict__ mind2) {
    __shared__ int2 q[RW_TILE];
    int dir = blockIdx.z;
    int64_t pbase = dir == 0 ? 0 : nA, np = dir == 0 ? nA : nB;
    int64_t qbase = dir == 0 ? nA : 0, nq = dir == 0 ? nB : nA;
    int64_t u = (int64_t)blockIdx.x * RW_THREADS + threadIdx.x;
    int64_t q0 = (int64_t)blockIdx.y * chunk, q1 = min(nq, q0 + chunk);
    if ((int64_t)blockIdx.x * RW_THREADS >= np || q0 >= q1) return;
    int32_t ux = 0, uy = 0;
    if (u < np) {
        ux = X[pbase + u];
        uy = Y[pbase + u];
    }
    unsigned long long best = ~0ull;
    for (int64_t t0 = q0; t0 < q1; t0 += RW_TILE) {
        int tn = (int)min((int64_t)RW_TILE, q1 - t0);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += RW_THREADS) q[j] = make_int2(X[qbase + t0 + j], Y[qbase + t0 + j]);
        __syncthreads();
        for (int j = 0; j < tn; j++) {
            int2 v = q[j];
            long long dx = (long long)(ux - v.x), dy = (long long)(uy - v.y);
            unsigned long long d2 = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy);
            best = d2 < best ? d2 : best;
        }
    }
    if (u < np) atomicMin(&mind2[pbase + u], best);
}

__global__ void k_rwmd_sum(const int32_t* __restrict__ X, const int32_t* __restrict__ Y,
                           const int64_t* __restrict__ cnt, int64_t nA, int64_t n,
                           const unsigned long long* __restrict__ mind2, DiagCost dc, int64_t* __restrict__ L) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long va = 0, vb = 0;
    if (i < n) {
        int64_t c = cost_make(X[i], Y[i], dc);
        unsigned long long m = mind2[i];
        if (m != ~0ull) {
            int64_t cn = (int64_t)ceil_sqrt_u64(m);
            c = cn < c ? cn : c;
        }
        unsigned long long v = (unsigned long long)(c * cnt[i]);
        if (i < nA)
            va = v;
        else
            vb = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        va += __shfl_xor_sync(0xffffffffu, va, o);
        vb += __shfl_xor_sync(0xffffffffu, vb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (va) atomicAdd((unsigned long long*)&L[0], va);
        if (vb) atomicAdd((unsigned long long*)&L[1], vb);
    }
}

// ---- the same minima through a uniform grid over each side ----------------
// Large sides make the all-pairs scan quadratic (about 10^12 distance
// evaluations at a million nodes a side).  Each side's nodes are bucketed
// into a grid of about two nodes a cell (a counting sort by cell), and every
// node of the other side searches square rings of cells around its own cell.
// After ring K every node not yet seen lies beyond one of the square's sides
// that are not the grid's border, so its distance is at least LB, the
// distance from the query to the nearest such side.  The search stops when
// LB^2 >= the best squared distance found (the minimum is exact), or when
// LB >= the query's diagonal cost c_make: every unseen node then costs at
// least c_make, the relaxed flow takes min(c(u, nearest), c_make) either way,
// and the stored value min(best, c_make^2) gives the same term.  A query that
// has not stopped after RW_KMAX rings (a far outlier) keeps its best as an
// upper bound and is finished by the all-pairs scan over the other side.

constexpr int RW_KMAX = 24;
constexpr int64_t RW_GRID_MIN = int64_t(1) << 28;  // nA * nB from which the grid is used

struct RwGrid {
    int64_t x0, y0, h;  // origin and cell side (quanta)
    int32_t gw, gh;     // cells per axis
    int64_t base;       // first cell of this grid in the shared cell arrays
};

__global__ void k_rw_box_init(int* box) {
    if (threadIdx.x < 8) box[threadIdx.x] = (threadIdx.x & 1) ? INT32_MIN : INT32_MAX;
}

// Bounding box of each side: box[4 s ..] = xmin, xmax, ymin, ymax of side s.
__global__ void k_rw_box(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t nA, int64_t n,
                         int* __restrict__ box) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int v[8];  // per side: -xmin, xmax, -ymin, ymax (maxima of all four)
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = INT32_MIN;
    if (i < n) {
        const int s = i < nA ? 0 : 4;
        v[s + 0] = -X[i];  // coordinates are above -2^30: negation is exact
        v[s + 1] = X[i];
        v[s + 2] = -Y[i];
        v[s + 3] = Y[i];
    }
#pragma unroll
    for (int k = 0; k < 8; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] = max(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    if ((threadIdx.x & 31) == 0)
        for (int s = 0; s < 8; s += 4)
            if (v[s + 1] != INT32_MIN) {
                atomicMin(&box[s + 0], -v[s + 0]);
                atomicMax(&box[s + 1], v[s + 1]);
                atomicMin(&box[s + 2], -v[s + 2]);
                atomicMax(&box[s + 3], v[s + 3]);
            }
}

PD_D int32_t rw_cell_axis(int64_t v, int64_t o, int64_t h, int32_t g) {
    if (v < o) return 0;
    const int64_t c = (v - o) / h;
    return c >= g ? g - 1 : (int32_t)c;
}

// Node i of side s goes into grid s (its cell's count).
__global__ void k_rw_hist(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t nA, int64_t n,
                          RwGrid g0, RwGrid g1, unsigned long long* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RwGrid& g = i < nA ? g0 : g1;
    const int64_t c = g.base + (int64_t)rw_cell_axis(Y[i], g.y0, g.h, g.gh) * g.gw + rw_cell_axis(X[i], g.x0, g.h, g.gw);
    atomicAdd(&cnt[c], 1ull);
}

// Nodes placed by cell (order inside a cell is arbitrary: only minima are read).
__global__ void k_rw_scatter(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t nA, int64_t n,
                             RwGrid g0, RwGrid g1, unsigned long long* __restrict__ cur, int2* __restrict__ pts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RwGrid& g = i < nA ? g0 : g1;
    const int64_t c = g.base + (int64_t)rw_cell_axis(Y[i], g.y0, g.h, g.gh) * g.gw + rw_cell_axis(X[i], g.x0, g.h, g.gw);
    const unsigned long long k = atomicAdd(&cur[c], 1ull);
    pts[k] = make_int2(X[i], Y[i]);
}

// Ring search of node i (side s) in the other side's grid; see above.
// Unfinished queries are listed: side A's from list[0], side B's from
// list[nA], their counts in nl[0], nl[1].
__global__ void k_rw_query(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t nA, int64_t n,
                           RwGrid g0, RwGrid g1, const unsigned long long* __restrict__ start,
                           const int2* __restrict__ pts, DiagCost dc, unsigned long long* __restrict__ mind2,
                           int32_t* __restrict__ list, int* __restrict__ nl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool sa = i < nA;
    const RwGrid& g = sa ? g1 : g0;  // the other side's grid
    const int64_t ux = X[i], uy = Y[i];
    const int64_t cm = cost_make((int32_t)ux, (int32_t)uy, dc);
    const int32_t cx = rw_cell_axis(ux, g.x0, g.h, g.gw), cy = rw_cell_axis(uy, g.y0, g.h, g.gh);
    unsigned long long best = ~0ull;
    auto visit = [&](int32_t x, int32_t y) {
        const int64_t c = g.base + (int64_t)y * g.gw + x;
        const unsigned long long k1 = start[c + 1];
        for (unsigned long long k = start[c]; k < k1; k++) {
            const int2 v = pts[k];
            const long long dx = ux - v.x, dy = uy - v.y;
            const unsigned long long d2 = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy);
            best = d2 < best ? d2 : best;
        }
    };
    int state = 0;  // 0 searching, 1 exact, 2 stopped by the diagonal cost
    for (int32_t K = 0; K <= RW_KMAX && state == 0; K++) {
        if (K == 0) {
            visit(cx, cy);
        } else {
            const int32_t xlo = max(cx - K, 0), xhi = min(cx + K, g.gw - 1);
            if (cy - K >= 0)
                for (int32_t x = xlo; x <= xhi; x++) visit(x, cy - K);
            if (cy + K < g.gh)
                for (int32_t x = xlo; x <= xhi; x++) visit(x, cy + K);
            const int32_t ylo = max(cy - K + 1, 0), yhi = min(cy + K - 1, g.gh - 1);
            if (cx - K >= 0)
                for (int32_t y = ylo; y <= yhi; y++) visit(cx - K, y);
            if (cx + K < g.gw)
                for (int32_t y = ylo; y <= yhi; y++) visit(cx + K, y);
        }
        // distance to the nearest side of the searched square beyond which nodes may remain
        int64_t lb = INT64_MAX;
        if (cx - K > 0) lb = min(lb, ux - (g.x0 + (int64_t)(cx - K) * g.h));
        if (cx + K < g.gw - 1) lb = min(lb, g.x0 + (int64_t)(cx + K + 1) * g.h - ux);
        if (cy - K > 0) lb = min(lb, uy - (g.y0 + (int64_t)(cy - K) * g.h));
        if (cy + K < g.gh - 1) lb = min(lb, g.y0 + (int64_t)(cy + K + 1) * g.h - uy);
        if (lb == INT64_MAX) {
            state = 1;  // the whole grid is searched
        } else {
            lb = lb < 0 ? 0 : lb;
            if ((unsigned long long)lb * (unsigned long long)lb >= best) state = 1;
            else if (lb >= cm) state = 2;
        }
    }
    if (state == 2) {
        const unsigned long long c2 = (unsigned long long)cm * (unsigned long long)cm;
        best = c2 < best ? c2 : best;
    }
    mind2[i] = best;
    if (state == 0) {
        const int k = atomicAdd(&nl[sa ? 0 : 1], 1);
        list[(sa ? 0 : nA) + k] = (int32_t)(sa ? i : i - nA);
    }
}

// The all-pairs scan for listed queries only (indices within their side);
// blockIdx.z = direction, blockIdx.y splits the other side.
__global__ void __launch_bounds__(RW_THREADS) k_rwmd_min_list(const int32_t* __restrict__ X,
                                                              const int32_t* __restrict__ Y, int64_t nA, int64_t nB,
                                                              const int32_t* __restrict__ list, int nlA, int nlB,
                                                              int64_t chunk, unsigned long long* __restrict__ mind2) {
    __shared__ int2 q[RW_TILE];
    const int dir = blockIdx.z;
    const int64_t pbase = dir == 0 ? 0 : nA, np = dir == 0 ? nlA : nlB;
    const int64_t qbase = dir == 0 ? nA : 0, nq = dir == 0 ? nB : nA;
    const int64_t t = (int64_t)blockIdx.x * RW_THREADS + threadIdx.x;
    const int64_t q0 = (int64_t)blockIdx.y * chunk, q1 = min(nq, q0 + chunk);
    if ((int64_t)blockIdx.x * RW_THREADS >= np || q0 >= q1) return;
    int64_t u = -1;
    int32_t ux = 0, uy = 0;
    if (t < np) {
        u = pbase + list[pbase + t];
        ux = X[u];
        uy = Y[u];
    }
    unsigned long long best = ~0ull;
    for (int64_t t0 = q0; t0 < q1; t0 += RW_TILE) {
        const int tn = (int)min((int64_t)RW_TILE, q1 - t0);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += RW_THREADS) q[j] = make_int2(X[qbase + t0 + j], Y[qbase + t0 + j]);
        __syncthreads();
        for (int j = 0; j < tn; j++) {
            const int2 v = q[j];
            const long long dx = (long long)(ux - v.x), dy = (long long)(uy - v.y);
            const unsigned long long d2 = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy);
            best = d2 < best ? d2 : best;
        }
    }
    if (u >= 0) atomicMin(&mind2[u], best);
}

__global__ void k_fill_u64(unsigned long long* p, int64_t n, unsigned long long v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Grid geometry of one side with box b (xmin, xmax, ymin, ymax) and n nodes:
// about two nodes a cell, at most 4 n + 64 cells.
static RwGrid rw_grid(const int* b, int64_t n, int64_t base) {
    RwGrid g{};
    const int64_t W = (int64_t)b[1] - b[0], H = (int64_t)b[3] - b[2];
    const double cells = (double)std::max<int64_t>(1, n / 2);
    int64_t hs = (int64_t)ceil(sqrt((double)(W + 1) * (double)(H + 1) / cells));
    hs = std::max<int64_t>(hs, 1);
    for (;;) {
        const int64_t gw = W / hs + 1, gh = H / hs + 1;
        if (gw * gh <= 4 * n + 64) {
            g.gw = (int32_t)gw;
            g.gh = (int32_t)gh;
            break;
        }
        hs *= 2;
    }
    g.x0 = b[0];
    g.y0 = b[2];
    g.h = hs;
    g.base = base;
    return g;
}

// Exact minima of both directions through the grids (see k_rw_query), the
// queries the rings did not finish completed by the all-pairs scan.
static pd_status rwmd_grid(Ctx* c, const Hats& h, DiagCost dc, unsigned long long* mind2, int64_t chunk, int64_t gy,
                           cudaStream_t st) {
    const int64_t n = h.nA + h.nB;
    int* box = bufT<int>(c, B_RW_BOX, 8);
    int* nl = bufT<int>(c, B_RW_NL, 2);
    if (!box || !nl) return PD_ENOMEM;
    k_rw_box_init<<<1, 32, 0, st>>>(box); pd::count_launch();
    k_rw_box<<<grid_for(n, 256), 256, 0, st>>>(h.X, h.Y, h.nA, n, box); pd::count_launch();
    int hb[8];
    PD_TRY_CUDA(c, cudaMemcpyAsync(hb, box, sizeof(hb), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    const RwGrid g0 = rw_grid(hb, h.nA, 0);
    const RwGrid g1 = rw_grid(hb + 4, h.nB, (int64_t)g0.gw * g0.gh);
    const int64_t cells = g1.base + (int64_t)g1.gw * g1.gh;
    unsigned long long* start = bufT<unsigned long long>(c, B_RW_START, cells + 1);
    unsigned long long* cur = bufT<unsigned long long>(c, B_RW_CUR, cells + 1);
    unsigned long long* part = bufT<unsigned long long>(c, B_SCAN_PART, scan_tiles(cells + 1) + 1);
    int2* pts = bufT<int2>(c, B_RW_PTS, n);
    int32_t* list = bufT<int32_t>(c, B_RW_LIST, n);
    if (!start || !cur || !part || !pts || !list) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(start, 0, sizeof(unsigned long long) * (cells + 1), st));
    PD_TRY_CUDA(c, cudaMemsetAsync(nl, 0, 2 * sizeof(int), st));
    k_rw_hist<<<grid_for(n, 256), 256, 0, st>>>(h.X, h.Y, h.nA, n, g0, g1, start); pd::count_launch();
    PD_TRY_CUDA(c, exclusive_scan<unsigned long long>(start, start, cells + 1, part, nullptr, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(cur, start, sizeof(unsigned long long) * (cells + 1), cudaMemcpyDeviceToDevice, st));
    k_rw_scatter<<<grid_for(n, 256), 256, 0, st>>>(h.X, h.Y, h.nA, n, g0, g1, cur, pts); pd::count_launch();
    k_rw_query<<<grid_for(n, 128), 128, 0, st>>>(h.X, h.Y, h.nA, n, g0, g1, start, pts, dc, mind2, list, nl); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    int hn[2];
    PD_TRY_CUDA(c, cudaMemcpyAsync(hn, nl, sizeof(hn), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (hn[0] + hn[1] > 0) {
        const int64_t gx = (std::max(hn[0], hn[1]) + RW_THREADS - 1) / RW_THREADS;
        k_rwmd_min_list<<<dim3((unsigned)gx, (unsigned)gy, 2), RW_THREADS, 0, st>>>(h.X, h.Y, h.nA, h.nB, list, hn[0],
                                                                                    hn[1], chunk, mind2); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
    }
    return PD_OK;
}

pd_status stage_rwmd(Ctx* c, const Hats& h, int64_t L[3], DiagCost dc, cudaStream_t st) {
    int64_t n = h.nA + h.nB;
    int64_t* sm = bufT<int64_t>(c, B_SMALL, 64);
    unsigned long long* mind2 = bufT<unsigned long long>(c, B_QKEY2, n);
    if (!sm || !mind2) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(sm + S_L0, 0, 2 * sizeof(int64_t), st));
    if (n > 0) {
        k_fill_u64<<<grid_for(n, 256), 256, 0, st>>>(mind2, n, ~0ull); pd::count_launch();
        int64_t npmax = h.nA > h.nB ? h.nA : h.nB;
        int64_t gx = (npmax + RW_THREADS - 1) / RW_THREADS;
        int64_t want = 4LL * (c->sm_count > 0 ? c->sm_count : 152);
        int64_t gy = (want + gx - 1) / gx;
        int64_t nqmax = npmax;
        int64_t chunk = (nqmax + gy - 1) / gy;
        if (chunk < 256) chunk = 256;
        gy = (nqmax + chunk - 1) / chunk;
        if (gy < 1) gy = 1;
        if (h.nA > 0 && h.nB > 0 && h.nA * h.nB >= RW_GRID_MIN) {
            PD_TRY(rwmd_grid(c, h, dc, mind2, chunk, gy, st));
        } else if (gx > 0 && h.nA > 0 && h.nB > 0) {
            k_rwmd_min<<<dim3((unsigned)gx, (unsigned)gy, 2), RW_THREADS, 0, st>>>(h.X, h.Y, h.nA, h.nB, chunk, mind2); pd::count_launch();
        }
        k_rwmd_sum<<<grid_for(n, 256), 256, 0, st>>>(h.X, h.Y, h.cnt, h.nA, n, mind2, dc, sm + S_L0); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
    }
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    L[0] = c->h_small[S_L0];
    L[1] = c->h_small[S_L1];
    L[2] = L[0] > L[1] ? L[0] : L[1];
    return PD_OK;
}

// ---------------------------------------------------------------------------
// delta-condensation (Algorithm 2) and Morton order
// ---------------------------------------------------------------------------

__global__ void k_cells(const int32_t* __restrict__ X, const int32_t* __restrict__ Y, int64_t n, int64_t G,
                        int64_t* __restrict__ CX, int64_t* __restrict__ CY, int64_t* __restrict__ sm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t cx = INT64_MAX, cy = INT64_MAX, xx = INT64_MIN, xy = INT64_MIN;
    if (i < n) {
        cx = floor_div(2 * (int64_t)X[i] + G, 2 * G);  // nearest lattice point, ties up
        cy = floor_div(2 * (int64_t)Y[i] + G, 2 * G);
        CX[i] = cx;
        CY[i] = cy;
        xx = cx;
        xy = cy;
    }
    for (int o = 16; o > 0; o >>= 1) {
        cx = min(cx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)cx, o));
        cy = min(cy, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)cy, o));
        xx = max(xx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)xx, o));
        xy = max(xy, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)xy, o));
    }
    if ((threadIdx.x & 31) == 0 && xx != INT64_MIN) {
        atomicMin((long long*)&sm[S_CMNX], (long long)cx);
        atomicMin((long long*)&sm[S_CMNY], (long long)cy);
        atomicMax((long long*)&sm[S_CMXX], (long long)xx);
        atomicMax((long long*)&sm[S_CMXY], (long long)xy);
    }
}

__global__ void k_cell_keys(const int64_t* __restrict__ CX, const int64_t* __restrict__ CY, int64_t n,
                            const int64_t* __restrict__ sm, int bcy, uint64_t* __restrict__ key,
                            uint32_t* __restrict__ val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = ((uint64_t)(CX[i] - sm[S_CMNX]) << bcy) | (uint64_t)(CY[i] - sm[S_CMNY]);
    val[i] = (uint32_t)i;
}

// One node per distinct cell: place it at G * cell + shift(seed, cell).
__global__ void k_cell_place(const uint64_t* __restrict__ key, int64_t n, const int64_t* __restrict__ idx,
                             const int64_t* __restrict__ sm, int bcy, int64_t G, int64_t P, uint64_t seed,
                             int32_t* __restrict__ NX, int32_t* __restrict__ NY, int64_t* __restrict__ smw) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t x = INT64_MAX, y = INT64_MAX, xx = INT64_MIN, xy = INT64_MIN;
    bool bad = false;
    if (i < n && (i == 0 || key[i - 1] != key[i])) {
        uint64_t k = key[i];
        uint64_t ymask = bcy >= 64 ? ~0ull : ((1ull << bcy) - 1);
        int64_t cx = (int64_t)(k >> bcy) + sm[S_CMNX];
        int64_t cy = (int64_t)(k & ymask) + sm[S_CMNY];
        int64_t dx, dy;
        cell_shift(seed, cx, cy, P, &dx, &dy);
        x = G * cx + dx;
        y = G * cy + dy;
        const int64_t lim = int64_t(1) << 30;
        bad = x <= -lim || x >= lim || y <= -lim || y >= lim;
        int64_t j = idx[i];
        NX[j] = (int32_t)x;
        NY[j] = (int32_t)y;
        xx = x;
        xy = y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        x = min(x, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)x, o));
        y = min(y, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)y, o));
        xx = max(xx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)xx, o));
        xy = max(xy, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)xy, o));
    }
    unsigned b = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (xx != INT64_MIN) {
            atomicMin((long long*)&smw[S_NMNX], (long long)x);
            atomicMin((long long*)&smw[S_NMNY], (long long)y);
            atomicMax((long long*)&smw[S_NMXX], (long long)xx);
            atomicMax((long long*)&smw[S_NMXY], (long long)xy);
        }
        if (b) atomicAdd((unsigned long long*)&smw[S_ERR], 1ull);
    }
}

// Aggregate the multiplicities of the nodes snapped into each cell.
__global__ void k_cell_accum(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, int64_t n,
                             const int64_t* __restrict__ idx, const int64_t* __restrict__ cnt, int64_t nA,
                             int64_t* __restrict__ CA, int64_t* __restrict__ CB) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = idx[i] + ((i == 0 || key[i - 1] != key[i]) ? 1 : 0) - 1;
    uint32_t v = val[i];
    atomicAdd((unsigned long long*)((int64_t)v < nA ? &CA[j] : &CB[j]), (unsigned long long)cnt[v]);
}

__global__ void k_morton_keys(const int32_t* __restrict__ NX, const int32_t* __restrict__ NY, int64_t N,
                              const int64_t* __restrict__ sm, uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    key[i] = morton2((uint32_t)(NX[i] - sm[S_NMNX]), (uint32_t)(NY[i] - sm[S_NMNY]));
    val[i] = (uint32_t)i;
}

__global__ void k_node_gather(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, int64_t N,
                              const int32_t* __restrict__ NX, const int32_t* __restrict__ NY,
                              const int64_t* __restrict__ CA, const int64_t* __restrict__ CB, int32_t* __restrict__ OX,
                              int32_t* __restrict__ OY, int64_t* __restrict__ OA, int64_t* __restrict__ OB,
                              uint64_t* __restrict__ OC) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t v = val[i];
    OX[i] = NX[v];
    OY[i] = NY[v];
    OA[i] = CA[v];
    OB[i] = CB[v];
    OC[i] = key[i];
}

pd_status stage_condense_delta(Ctx* c, const Hats& h, int64_t G, int64_t P, uint64_t seed, pd_nodes* out,
                               cudaStream_t st) {
    int64_t n = h.nA + h.nB;
    out->n_nodes = 0;
    out->X = bufT<int32_t>(c, B_NX, n);
    out->Y = bufT<int32_t>(c, B_NY, n);
    out->cntA = bufT<int64_t>(c, B_NCA, n);
    out->cntB = bufT<int64_t>(c, B_NCB, n);
    out->morton = bufT<uint64_t>(c, B_NCODE, n);
    int64_t* sm = bufT<int64_t>(c, B_SMALL, 64);
    if (!out->X || !out->Y || !out->cntA || !out->cntB || !out->morton || !sm) return PD_ENOMEM;
    if (n == 0) return PD_OK;
    int64_t* CX = bufT<int64_t>(c, B_CX, n);
    int64_t* CY = bufT<int64_t>(c, B_CY, n);
    uint64_t* key = bufT<uint64_t>(c, B_CKEY, n);
    uint64_t* key2 = bufT<uint64_t>(c, B_CKEY2, n);
    uint32_t* val = bufT<uint32_t>(c, B_CVAL, n);
    uint32_t* val2 = bufT<uint32_t>(c, B_CVAL2, n);
    int64_t* idx = bufT<int64_t>(c, B_CIDX, n);
    int32_t* NX = bufT<int32_t>(c, B_QX, n);
    int32_t* NY = bufT<int32_t>(c, B_QY, n);
    int64_t* CA = bufT<int64_t>(c, B_CA, n);
    int64_t* CB = bufT<int64_t>(c, B_CB, n);
    if (!CX || !CY || !key || !key2 || !val || !val2 || !idx || !NX || !NY || !CA || !CB) return PD_ENOMEM;
    k_init_small<<<1, 64, 0, st>>>(sm); pd::count_launch();
    k_cells<<<grid_for(n, 256), 256, 0, st>>>(h.X, h.Y, n, G, CX, CY, sm); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    int64_t* hs = c->h_small;
    int bcx = bits_for((uint64_t)(hs[S_CMXX] - hs[S_CMNX])), bcy = bits_for((uint64_t)(hs[S_CMXY] - hs[S_CMNY]));
    k_cell_keys<<<grid_for(n, 256), 256, 0, st>>>(CX, CY, n, sm, bcy, key, val); pd::count_launch();
    PD_TRY(sort_u64(c, key, key2, val, val2, n, bcx + bcy, st));
    k_run_flags<<<grid_for(n, 256), 256, 0, st>>>(key, n, ~0ull, idx); pd::count_launch();
    PD_TRY(scan_i64(c, idx, idx, n, sm + S_N, st));
    k_cell_place<<<grid_for(n, 256), 256, 0, st>>>(key, n, idx, sm, bcy, G, P, seed, NX, NY, sm); pd::count_launch();
    PD_TRY_CUDA(c, cudaMemsetAsync(CA, 0, sizeof(int64_t) * n, st));
    PD_TRY_CUDA(c, cudaMemsetAsync(CB, 0, sizeof(int64_t) * n, st));
    k_cell_accum<<<grid_for(n, 256), 256, 0, st>>>(key, val, n, idx, h.cnt, h.nA, CA, CB); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (hs[S_ERR]) return fail(c, PD_EINVAL, "condensed node coordinate outside (-2^30, 2^30)");
    int64_t N = hs[S_N];
    int bm = bits_for((uint64_t)(hs[S_NMXX] - hs[S_NMNX]));
    int bm2 = bits_for((uint64_t)(hs[S_NMXY] - hs[S_NMNY]));
    if (bm2 > bm) bm = bm2;
    k_morton_keys<<<grid_for(N, 256), 256, 0, st>>>(NX, NY, N, sm, key, val); pd::count_launch();
    PD_TRY(sort_u64(c, key, key2, val, val2, N, 2 * bm, st));
    k_node_gather<<<grid_for(N, 256), 256, 0, st>>>(key, val, N, NX, NY, CA, CB, out->X, out->Y, out->cntA,
                                                      out->cntB, out->morton); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    out->n_nodes = N;
    return PD_OK;
}

}  // namespace pd
