// Exact integer min-cost flow on an uncapacitated network by cost scaling
// (successive approximation with push / relabel), run as one persistent
// cooperative kernel with bounded grid barriers.
//
// Residual graph.  Every arc (u, v, c) becomes an edge with a net flow x
// stored on two slots, x[u->v] = -x[v->u].  An antiparallel pair of arcs with
// equal cost (the WSPD biarcs) shares one edge; any other arc gets an edge
// whose reverse slot only allows cancelling.  From slot (u -> v): if x < 0
// the residual arc cancels flow of v -> u (cost -c, capacity -x); otherwise,
// if u -> v is an arc, it is the arc itself (cost c, unbounded).
//
// Phases (scaled costs c*K, K = n + 1, so 1-optimality is optimality):
//   1. price repair: the largest prices p' <= p with p'(u) <= c K + eps + p'(v)
//      on every arc (a monotone min-plus fixed point, iterated in place);
//   2. flows whose cancelling arc now has reduced cost < -eps are cancelled,
//      which leaves an eps-optimal pseudoflow;
//   3. rounds of (push | relabel) until no node has excess.  A push moves
//      excess along admissible residual arcs (reduced cost c - p(u) + p(v)
//      < 0) with all prices fixed; a relabel, done in a separate sub-step
//      with all flows fixed, sets p(u) = min over residual arcs (c + p(v)) + eps.
//      Prices only rise within a phase, so concurrent relabels keep
//      eps-optimality.
//   eps <- max(1, eps / alpha) until a phase with eps = 1 has finished.
#include <cooperative_groups.h>

#include "internal.h"
#include "prims.cuh"

namespace pd {

constexpr uint32_t FWD = 0x80000000u;
constexpr int SV_THREADS = 256;

struct SolverCtl {
    unsigned int bar_count;
    unsigned int bar_gen;
    int status;
    int phases;
    long long active[3];
    long long changed[3];
    long long dmax[3];
    long long rounds, pushes, relabels, repairs, updates, update_passes;
    long long relabel_total;  // monotone: relabels so far (read after barriers)
};

struct SolverArgs {
    int64_t n;
    const int64_t* rp;
    const int32_t* hd;
    const uint32_t* cw;
    const int64_t* tw;
    int64_t* x;
    int64_t* e;
    int64_t* p;
    int64_t* d;
    int64_t* cur;
    int8_t* relab;
    int64_t K;
    int64_t eps0;
    int alpha;
    int64_t max_rounds;
    int64_t update_every;  // relabels between global price updates (0 = only at phase start)
    int64_t seq_threshold; // at most this many active nodes: block 0 discharges them alone
    int64_t seq_budget;    // node discharges per sequential session
    int32_t* q;            // ring of n nodes for the sequential sessions
    int64_t spin_limit;
    uint64_t time_limit_ns;
    SolverCtl* ctl;
};

PD_D uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier for a cooperative launch (all blocks resident).  The wait is
// bounded: after spin_limit polls the block records ERR_TIMEOUT and leaves.
PD_D void grid_sync(SolverCtl* ctl, int64_t spin_limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* genp = &ctl->bar_gen;
        unsigned int gen = *genp;
        __threadfence();
        unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            int64_t spins = 0;
            while (*genp == gen) {
                if (++spins > spin_limit) {
                    atomicOr(&ctl->status, (int)ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

PD_D int status_of(SolverCtl* ctl) { return *(volatile int*)&ctl->status; }

PD_D long long vload(long long* p) { return *(volatile long long*)p; }

PD_D int64_t warp_min64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// Residual arc of slot s seen from its row: returns false if none; else the
// scaled residual cost and the capacity (INT64_MAX = unbounded).
PD_D bool residual(uint32_t cw, int64_t xs, int64_t K, int64_t* rc, int64_t* cap) {
    int64_t c = (int64_t)(cw & ~FWD) * K;
    if (xs < 0) {
        *rc = -c;
        *cap = -xs;
        return true;
    }
    if (cw & FWD) {
        *rc = c;
        *cap = INT64_MAX;
        return true;
    }
    return false;
}

constexpr int64_t D_INF = int64_t(1) << 60;
constexpr int64_t D_CAP = int64_t(1) << 50;

// Block 0 checks the device wall clock before a barrier so that every block
// reads the same status after it.
PD_D void check_time(const SolverArgs& a, unsigned long long t0) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && global_ns() - t0 > a.time_limit_ns)
        atomicOr(&a.ctl->status, (int)ERR_TIMEOUT);
}

// Global price update (Goldberg): d(u) = shortest distance from u to a node
// with a deficit in the residual graph, arc length floor(rc / eps) + 1 >= 0;
// then p(u) += eps d(u) (nodes that reach no deficit take the largest finite
// d).  Keeps eps-optimality, only raises prices, and makes every node's first
// arc on a shortest path admissible.  Returns false if the solve must stop.
PD_D bool global_update(const SolverArgs& a, int64_t eps, int& slotC, int& slotD, unsigned long long t0,
                        long long& passes) {
    SolverCtl* ctl = a.ctl;
    const int lane = threadIdx.x & 31;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
    __shared__ int blk;
    for (int64_t u = gtid; u < a.n; u += gthreads) __stcg(&a.d[u], __ldcg(&a.e[u]) < 0 ? (int64_t)0 : D_INF);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->dmax[(slotD + 1) % 3] = 0;
    grid_sync(ctl, a.spin_limit);
    for (;;) {
        if (threadIdx.x == 0) blk = 0;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->changed[(slotC + 1) % 3] = 0;
        __syncthreads();
        for (int64_t u = gwarp; u < a.n; u += nwarps) {
            int64_t du = __ldcg(&a.d[u]);
            if (du == 0) continue;
            int64_t pu = __ldcg(&a.p[u]);
            int64_t m = D_INF;
            for (int64_t s = a.rp[u] + lane; s < a.rp[u + 1]; s += 32) {
                int64_t rc, cap;
                if (!residual(a.cw[s], __ldcg(&a.x[s]), a.K, &rc, &cap)) continue;
                int64_t v = a.hd[s];
                int64_t dv = __ldcg(&a.d[v]);
                if (dv >= D_INF) continue;
                rc = rc - pu + __ldcg(&a.p[v]);
                int64_t l = floor_div(rc, eps) + 1;
                if (l < 0) l = 0;
                int64_t cand = l > D_CAP ? D_INF : l + dv;
                if (cand > D_CAP) cand = D_INF;
                m = cand < m ? cand : m;
            }
            m = warp_min64(m);
            if (m < du) {
                if (lane == 0) __stcg(&a.d[u], m);
                blk = 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && blk) atomicAdd((unsigned long long*)&ctl->changed[slotC], 1ull);
        check_time(a, t0);
        grid_sync(ctl, a.spin_limit);
        long long ch = vload(&ctl->changed[slotC]);
        slotC = (slotC + 1) % 3;
        passes++;
        if (status_of(ctl)) return false;
        if (ch == 0) break;
    }
    long long mx = 0;
    for (int64_t u = gtid; u < a.n; u += gthreads) {
        int64_t du = __ldcg(&a.d[u]);
        if (du < D_INF && du > mx) mx = du;
    }
    for (int o = 16; o > 0; o >>= 1) {
        long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if (lane == 0 && mx > 0) atomicMax((unsigned long long*)&ctl->dmax[slotD], (unsigned long long)mx);
    grid_sync(ctl, a.spin_limit);
    int64_t dmax = vload(&ctl->dmax[slotD]);
    slotD = (slotD + 1) % 3;
    if (status_of(ctl)) return false;
    for (int64_t u = gtid; u < a.n; u += gthreads) {
        int64_t du = __ldcg(&a.d[u]);
        if (du >= D_INF) du = dmax;
        if (du > 0) {
            if (du > ((int64_t(1) << 61) / eps)) {
                atomicOr(&ctl->status, (int)ERR_OVERFLOW);
            } else {
                __stcg(&a.p[u], __ldcg(&a.p[u]) + eps * du);
            }
        }
        __stcg(&a.cur[u], a.rp[u]);
    }
    grid_sync(ctl, a.spin_limit);
    return status_of(ctl) == 0;
}


// Sequential discharge by block 0 alone (the other blocks wait at a grid
// barrier): FIFO push/relabel on the few active nodes, the standard
// sequential algorithm, with the block scanning 256 slots of a row at a time.
// relab[] marks queued nodes during the session and is clear on exit.
constexpr int SEQ_T = SV_THREADS;

PD_D void seq_session(const SolverArgs& a, int64_t eps, unsigned long long t0, long long& n_push,
                      long long& n_relabel) {
    __shared__ int64_t sh_cap[SEQ_T], sh_need[SEQ_T];
    __shared__ int32_t sh_v[SEQ_T];
    __shared__ unsigned char sh_adm[SEQ_T];
    __shared__ int64_t qhead, qtail, sh_e, sh_min;
    __shared__ int32_t sh_u;
    __shared__ int sh_stop;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t n = a.n;
    if (t == 0) {
        qhead = 0;
        qtail = 0;
    }
    __syncthreads();
    for (int64_t u = t; u < n; u += SEQ_T) {
        if (__ldcg(&a.e[u]) > 0) {
            unsigned long long pos = atomicAdd((unsigned long long*)&qtail, 1ull);
            a.q[pos] = (int32_t)u;
            a.relab[u] = 1;
        }
    }
    __syncthreads();
    int64_t ops = 0;
    for (;;) {
        if (t == 0) {
            sh_stop = (qhead == qtail) || ops >= a.seq_budget || (global_ns() - t0 > a.time_limit_ns);
            if (!sh_stop) {
                sh_u = a.q[qhead % n];
                qhead++;
                a.relab[sh_u] = 0;
                sh_e = __ldcg(&a.e[sh_u]);
            }
        }
        __syncthreads();
        if (sh_stop) break;
        const int32_t u = sh_u;
        const int64_t e0 = a.rp[u], end = a.rp[u + 1];
        ops++;
        if (t == 0) sh_stop = 0;
        __syncthreads();
        while (sh_e > 0) {
            int64_t pu = __ldcg(&a.p[u]);
            int64_t s = __ldcg(&a.cur[u]);
            bool done = false;
            while (s < end && !done) {
                int64_t idx = s + t;
                bool adm = false;
                int64_t cap = 0, need = 0;
                int32_t v = 0;
                if (idx < end) {
                    int64_t rc;
                    v = a.hd[idx];
                    if (residual(a.cw[idx], __ldcg(&a.x[idx]), a.K, &rc, &cap)) adm = rc - pu + __ldcg(&a.p[v]) < 0;
                    if (adm) {
                        int64_t ev = __ldcg(&a.e[v]);
                        need = ev < 0 ? -ev : 0;
                    }
                }
                sh_adm[t] = adm;
                sh_cap[t] = cap;
                sh_need[t] = need;
                sh_v[t] = v;
                int nadm = __syncthreads_count(adm);
                if (nadm == 0) {
                    s += SEQ_T;
                    continue;
                }
                if (w == 0) {
                    int64_t rem = sh_e;
                    for (int pass = 0; pass < 2 && rem > 0; pass++) {
                        for (int g = 0; g < SEQ_T / 32 && rem > 0; g++) {
                            int tt = g * 32 + lane;
                            bool ok = sh_adm[tt] && sh_cap[tt] > 0 && (pass == 1 || sh_need[tt] > 0);
                            unsigned m = __ballot_sync(0xffffffffu, ok);
                            while (m && rem > 0) {
                                int l = __ffs(m) - 1;
                                m &= m - 1;
                                int ts = g * 32 + l;
                                int64_t want = pass == 0 ? (sh_need[ts] < sh_cap[ts] ? sh_need[ts] : sh_cap[ts])
                                                         : sh_cap[ts];
                                int64_t dd = rem < want ? rem : want;
                                if (lane == l) {
                                    int64_t si = s + ts;
                                    int32_t v2 = sh_v[ts];
                                    __stcg(&a.x[si], __ldcg(&a.x[si]) + dd);
                                    int64_t tw = a.tw[si];
                                    __stcg(&a.x[tw], __ldcg(&a.x[tw]) - dd);
                                    int64_t ev = __ldcg(&a.e[v2]);
                                    __stcg(&a.e[v2], ev + dd);
                                    if (ev <= 0 && ev + dd > 0 && !a.relab[v2]) {
                                        a.relab[v2] = 1;
                                        a.q[qtail % n] = v2;
                                        qtail++;
                                    }
                                    if (sh_cap[ts] != INT64_MAX) sh_cap[ts] -= dd;
                                    if (sh_need[ts] > 0) sh_need[ts] -= dd < sh_need[ts] ? dd : sh_need[ts];
                                }
                                rem -= dd;
                                n_push++;
                                __syncwarp();
                                if (pass == 1 && rem > 0) {
                                    // this slot is exhausted, continue with the next
                                }
                            }
                        }
                    }
                    if (lane == 0) sh_e = rem;
                }
                __syncthreads();
                if (sh_e == 0) {
                    if (t == 0) __stcg(&a.cur[u], s);
                    done = true;
                } else {
                    s += SEQ_T;
                }
                __syncthreads();
            }
            if (sh_e <= 0) break;
            // relabel: no admissible arc left in the row
            int64_t best = INT64_MAX;
            for (int64_t sl = e0 + t; sl < end; sl += SEQ_T) {
                int64_t rc, cap;
                if (residual(a.cw[sl], __ldcg(&a.x[sl]), a.K, &rc, &cap)) {
                    int64_t val = rc + __ldcg(&a.p[a.hd[sl]]);
                    best = val < best ? val : best;
                }
            }
            best = warp_min64(best);
            if (t == 0) sh_min = INT64_MAX;
            __syncthreads();
            if (lane == 0) atomicMin((long long*)&sh_min, (long long)best);
            __syncthreads();
            if (t == 0) {
                if (sh_min == INT64_MAX) {
                    atomicOr(&a.ctl->status, (int)ERR_INFEASIBLE);
                    sh_e = 0;
                } else {
                    int64_t np = sh_min + eps;
                    if (np > (int64_t(1) << 62)) atomicOr(&a.ctl->status, (int)ERR_OVERFLOW);
                    if (np > pu) __stcg(&a.p[u], np);
                }
                __stcg(&a.cur[u], e0);
                n_relabel++;
                sh_stop = *(volatile int*)&a.ctl->status;
            }
            ops++;
            __syncthreads();
            if (sh_stop) break;
        }
        // nothing pushes into u while u is discharged: its excess is sh_e
        if (t == 0) {
            __stcg(&a.e[u], sh_e);
            sh_stop = *(volatile int*)&a.ctl->status;
        }
        __syncthreads();
        if (sh_stop) break;
    }
    // leave relab[] clear for the parallel rounds
    __syncthreads();
    for (int64_t i = qhead + t; i < qtail; i += SEQ_T) a.relab[a.q[i % n]] = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(SV_THREADS) k_solve(SolverArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    SolverCtl* ctl = a.ctl;
    int64_t eps = a.eps0;
    long long n_push = 0, n_relabel = 0, n_updates = 0, upd_passes = 0;
    int64_t rounds = 0;
    int slotC = 0, slotA = 0, slotD = 0;
    int64_t repairs = 0;
    long long last_update = 0;
    bool stop = false;
    __shared__ int blk_flag;
    __shared__ unsigned long long t_start;
    if (threadIdx.x == 0) t_start = global_ns();
    __syncthreads();
    const unsigned long long t0 = t_start;

    for (int phase = 0; !stop; phase++) {
        // ---- 1. price repair -------------------------------------------
        for (;;) {
            if (threadIdx.x == 0) blk_flag = 0;
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->changed[(slotC + 1) % 3] = 0;
            __syncthreads();
            for (int64_t u = gwarp; u < a.n; u += nwarps) {
                int64_t m = INT64_MAX;
                int64_t e0 = a.rp[u], e1 = a.rp[u + 1];
                for (int64_t s = e0 + lane; s < e1; s += 32) {
                    uint32_t cw = a.cw[s];
                    if (cw & FWD) {
                        int64_t v = a.hd[s];
                        int64_t cand = (int64_t)(cw & ~FWD) * a.K + eps + __ldcg(&a.p[v]);
                        m = cand < m ? cand : m;
                    }
                }
                m = warp_min64(m);
                int64_t pu = __ldcg(&a.p[u]);
                if (m < pu) {
                    if (lane == 0) __stcg(&a.p[u], m);
                    blk_flag = 1;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && blk_flag) atomicAdd((unsigned long long*)&ctl->changed[slotC], 1ull);
            check_time(a, t0);
            grid_sync(ctl, a.spin_limit);
            long long ch = vload(&ctl->changed[slotC]);
            slotC = (slotC + 1) % 3;
            repairs++;
            if (status_of(ctl)) {
                stop = true;
                break;
            }
            if (ch == 0) break;
        }
        if (stop) break;
        // ---- 2. cancel flow whose cancelling arc violates eps-optimality --
        for (int64_t u = gwarp; u < a.n; u += nwarps) {
            int64_t e0 = a.rp[u], e1 = a.rp[u + 1];
            int64_t pu = __ldcg(&a.p[u]);
            for (int64_t s = e0 + lane; s < e1; s += 32) {
                int64_t xs = __ldcg(&a.x[s]);
                if (xs < 0) {
                    int64_t v = a.hd[s];
                    int64_t rc = -(int64_t)(a.cw[s] & ~FWD) * a.K - pu + __ldcg(&a.p[v]);
                    if (rc < -eps) {
                        __stcg(&a.x[s], (int64_t)0);
                        __stcg(&a.x[a.tw[s]], (int64_t)0);
                        atomicAdd((unsigned long long*)&a.e[u], (unsigned long long)xs);       // e(u) -= f
                        atomicAdd((unsigned long long*)&a.e[v], (unsigned long long)(-xs));    // e(v) += f
                    }
                }
            }
            if (lane == 0) {
                __stcg(&a.cur[u], e0);
                __stcg(&a.relab[u], (int8_t)0);
            }
        }
        grid_sync(ctl, a.spin_limit);
        if (status_of(ctl)) break;
        // ---- 3. global price update, then push / relabel rounds -----------
        if (!global_update(a, eps, slotC, slotD, t0, upd_passes)) break;
        n_updates++;
        last_update = vload(&ctl->relabel_total);
        for (;;) {
            // push sub-step: prices fixed.  Excess goes first to admissible
            // neighbours with a deficit, the rest along the first admissible arc.
            for (int64_t u = gwarp; u < a.n; u += nwarps) {
                int64_t eu = __ldcg(&a.e[u]);
                if (eu <= 0) continue;
                int64_t pu = __ldcg(&a.p[u]);
                int64_t s = __ldcg(&a.cur[u]);
                int64_t end = a.rp[u + 1];
                int64_t rem = eu;
                int64_t stop_at = s;
                while (s < end && rem > 0) {
                    int64_t idx = s + lane;
                    bool adm = false;
                    int64_t cap = 0, v = 0, need = 0;
                    if (idx < end) {
                        uint32_t cw = a.cw[idx];
                        int64_t xs = __ldcg(&a.x[idx]);
                        int64_t rc;
                        v = a.hd[idx];
                        if (residual(cw, xs, a.K, &rc, &cap)) adm = rc - pu + __ldcg(&a.p[v]) < 0;
                        if (adm) {
                            int64_t ev = __ldcg(&a.e[v]);
                            need = ev < 0 ? -ev : 0;
                        }
                    }
                    unsigned mask = __ballot_sync(0xffffffffu, adm);
                    if (mask == 0) {
                        s += 32;
                        continue;
                    }
                    unsigned dmask = __ballot_sync(0xffffffffu, adm && need > 0);
                    while (dmask && rem > 0) {
                        int l = __ffs(dmask) - 1;
                        dmask &= dmask - 1;
                        int64_t want = __shfl_sync(0xffffffffu, need < cap ? need : cap, l);
                        int64_t dd = rem < want ? rem : want;
                        if (lane == l) {
                            __stcg(&a.x[idx], __ldcg(&a.x[idx]) + dd);
                            int64_t t = a.tw[idx];
                            __stcg(&a.x[t], __ldcg(&a.x[t]) - dd);
                            atomicAdd((unsigned long long*)&a.e[v], (unsigned long long)dd);
                            if (cap != INT64_MAX) cap -= dd;
                        }
                        rem -= dd;
                        n_push++;
                    }
                    mask = __ballot_sync(0xffffffffu, adm && cap > 0);
                    while (mask && rem > 0) {
                        int l = __ffs(mask) - 1;
                        int64_t capl = __shfl_sync(0xffffffffu, cap, l);
                        int64_t dd = rem < capl ? rem : capl;
                        if (lane == l) {
                            __stcg(&a.x[idx], __ldcg(&a.x[idx]) + dd);
                            int64_t t = a.tw[idx];
                            __stcg(&a.x[t], __ldcg(&a.x[t]) - dd);
                            atomicAdd((unsigned long long*)&a.e[v], (unsigned long long)dd);
                        }
                        rem -= dd;
                        n_push++;
                        if (dd == capl)
                            mask &= mask - 1;
                        else
                            break;
                    }
                    if (rem == 0) {
                        stop_at = s;  // admissible arcs of this chunk may remain
                        break;
                    }
                    s += 32;
                }
                if (lane == 0) {
                    if (rem > 0) {
                        __stcg(&a.relab[u], (int8_t)1);
                    } else {
                        __stcg(&a.cur[u], stop_at);
                    }
                    if (eu - rem > 0) atomicAdd((unsigned long long*)&a.e[u], (unsigned long long)(rem - eu));
                }
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->active[(slotA + 1) % 3] = 0;
            grid_sync(ctl, a.spin_limit);
            if (status_of(ctl)) {
                stop = true;
                break;
            }
            // relabel sub-step: flows fixed.  p(u) = min(c + p(v)) + eps over
            // residual arcs, never lowered.
            long long act = 0, rl = 0;
            for (int64_t u = gwarp; u < a.n; u += nwarps) {
                if (__ldcg(&a.relab[u])) {
                    int64_t e0 = a.rp[u], e1 = a.rp[u + 1];
                    int64_t best = INT64_MAX;
                    for (int64_t s = e0 + lane; s < e1; s += 32) {
                        int64_t rc, cap;
                        if (residual(a.cw[s], __ldcg(&a.x[s]), a.K, &rc, &cap)) {
                            int64_t val = rc + __ldcg(&a.p[a.hd[s]]);
                            best = val < best ? val : best;
                        }
                    }
                    best = warp_min64(best);
                    if (lane == 0) {
                        if (best == INT64_MAX) {
                            atomicOr(&ctl->status, (int)ERR_INFEASIBLE);
                        } else {
                            int64_t np = best + eps;
                            if (np > (int64_t(1) << 62) || np < -(int64_t(1) << 62))
                                atomicOr(&ctl->status, (int)ERR_OVERFLOW);
                            int64_t pu = __ldcg(&a.p[u]);
                            if (np > pu) __stcg(&a.p[u], np);
                        }
                        __stcg(&a.cur[u], e0);
                        __stcg(&a.relab[u], (int8_t)0);
                        rl++;
                    }
                }
                if (lane == 0 && __ldcg(&a.e[u]) > 0) act++;
            }
            if (lane == 0 && act) atomicAdd((unsigned long long*)&ctl->active[slotA], (unsigned long long)act);
            if (lane == 0 && rl) atomicAdd((unsigned long long*)&ctl->relabel_total, (unsigned long long)rl);
            n_relabel += rl;
            check_time(a, t0);
            if (rounds + 1 >= a.max_rounds && blockIdx.x == 0 && threadIdx.x == 0)
                atomicOr(&ctl->status, (int)ERR_TIMEOUT);
            grid_sync(ctl, a.spin_limit);
            long long active = vload(&ctl->active[slotA]);
            long long rtot = vload(&ctl->relabel_total);
            slotA = (slotA + 1) % 3;
            rounds++;
            if (status_of(ctl)) {
                stop = true;
                break;
            }
            if (active == 0) break;
            if (active <= a.seq_threshold) {
                long long sr = 0;
                if (blockIdx.x == 0) {
                    seq_session(a, eps, t0, n_push, sr);
                    if (threadIdx.x == 0 && sr) atomicAdd((unsigned long long*)&ctl->relabel_total, (unsigned long long)sr);
                }
                check_time(a, t0);
                grid_sync(ctl, a.spin_limit);
                rtot = vload(&ctl->relabel_total);
                if (status_of(ctl)) {
                    stop = true;
                    break;
                }
            }
            if (a.update_every > 0 && rtot - last_update >= a.update_every) {
                if (!global_update(a, eps, slotC, slotD, t0, upd_passes)) {
                    stop = true;
                    break;
                }
                n_updates++;
                last_update = rtot;
            }
        }
        if (stop) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->phases = phase + 1;
        if (eps == 1) break;
        eps = eps / a.alpha;
        if (eps < 1) eps = 1;
    }
    if (lane == 0) {
        if (n_push) atomicAdd((unsigned long long*)&ctl->pushes, (unsigned long long)n_push);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->rounds = rounds;
        ctl->repairs = repairs;
        ctl->relabels = vload(&ctl->relabel_total);
        ctl->updates = n_updates;
        ctl->update_passes = upd_passes;
    }
}

// ---------------------------------------------------------------------------
// residual graph construction
// ---------------------------------------------------------------------------

__global__ void k_arc_tails(const int64_t* __restrict__ rp, int64_t n, int64_t m, int32_t* __restrict__ tail) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    int64_t lo = 0, hi = n;  // largest r with rp[r] <= a
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (rp[mid] <= a)
            lo = mid;
        else
            hi = mid;
    }
    tail[a] = (int32_t)lo;
}

// Pair every arc with its antiparallel arc of equal cost, if any; arcs
// without one get a cancel-only reverse slot (keyed for sorting by its row).
__global__ void k_pairing(const int64_t* __restrict__ rp, const int32_t* __restrict__ hd,
                          const int64_t* __restrict__ cost, const int32_t* __restrict__ tail, int64_t m, int hb,
                          uint64_t sent, int64_t* __restrict__ pair, uint64_t* __restrict__ xkey,
                          uint32_t* __restrict__ xval, int* __restrict__ err,
                          unsigned long long* __restrict__ n_extra) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    int64_t u = tail[a], v = hd[a];
    int64_t c = cost[a];
    if (c < 0 || c >= (int64_t(1) << 31)) atomicOr(err, (int)ERR_OVERFLOW);
    int64_t lo = rp[v], hi = rp[v + 1] - 1, j = -1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        int64_t h = hd[mid];
        if (h == u) {
            j = mid;
            break;
        }
        if (h < u)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    if (j >= 0 && cost[j] != c) j = -1;
    pair[a] = j;
    xkey[a] = j >= 0 ? sent : (((uint64_t)v << hb) | (uint64_t)u);
    xval[a] = (uint32_t)a;
    if (j < 0) atomicAdd(n_extra, 1ull);
}

__global__ void k_sym_rowptr(const int64_t* __restrict__ rp, const int64_t* __restrict__ xp, int64_t n,
                             int64_t* __restrict__ srp) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r <= n) srp[r] = rp[r] + xp[r];
}

__global__ void k_fill_extra(const uint64_t* __restrict__ xkey, const uint32_t* __restrict__ xval, int64_t E, int hb,
                             const int64_t* __restrict__ rp, const int64_t* __restrict__ xp,
                             const int64_t* __restrict__ srp, const int64_t* __restrict__ cost,
                             int32_t* __restrict__ shd, uint32_t* __restrict__ scw, int64_t* __restrict__ stw,
                             int64_t* __restrict__ xpos) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    uint64_t k = xkey[e];
    int64_t v = (int64_t)(k >> hb), u = (int64_t)(k & ((1ull << hb) - 1));
    int64_t a = xval[e];
    int64_t pos = srp[v] + (rp[v + 1] - rp[v]) + (e - xp[v]);
    shd[pos] = (int32_t)u;
    scw[pos] = (uint32_t)cost[a];
    stw[pos] = srp[u] + (a - rp[u]);
    xpos[a] = pos;
}

__global__ void k_fill_dir(const int64_t* __restrict__ rp, const int32_t* __restrict__ hd,
                           const int64_t* __restrict__ cost, const int32_t* __restrict__ tail,
                           const int64_t* __restrict__ pair, const int64_t* __restrict__ xpos, int64_t m,
                           const int64_t* __restrict__ srp, int32_t* __restrict__ shd, uint32_t* __restrict__ scw,
                           int64_t* __restrict__ stw) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    int64_t u = tail[a], v = hd[a];
    int64_t pos = srp[u] + (a - rp[u]);
    shd[pos] = (int32_t)v;
    scw[pos] = (uint32_t)cost[a] | FWD;
    int64_t j = pair[a];
    stw[pos] = j >= 0 ? srp[v] + (j - rp[v]) : xpos[a];
}

__global__ void k_max_cost(const int64_t* __restrict__ cost, int64_t m, unsigned long long* __restrict__ out) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = a < m ? (unsigned long long)cost[a] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, c, o);
        c = u > c ? u : c;
    }
    if ((threadIdx.x & 31) == 0 && c) atomicMax(out, c);
}

__global__ void k_max_cost32(const int32_t* __restrict__ cost, int64_t m, unsigned long long* __restrict__ out) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = a < m ? (unsigned long long)(uint32_t)cost[a] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, c, o);
        c = u > c ? u : c;
    }
    if ((threadIdx.x & 31) == 0 && c) atomicMax(out, c);
}

// OPT = sum of c * x over slots carrying flow in their arc's direction;
// slack = total flow (each rounded-up unit cost exceeds the real one by < 1).
__global__ void k_objective(const uint32_t* __restrict__ cw, const int64_t* __restrict__ x, int64_t ms,
                            unsigned long long* __restrict__ out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long o = 0, f = 0, bad = 0;
    if (s < ms) {
        int64_t xs = x[s];
        if (xs > 0) {
            if (!(cw[s] & FWD)) bad = 1;
            o = (unsigned long long)((int64_t)(cw[s] & ~FWD) * xs);
            f = (unsigned long long)xs;
        }
    }
    for (int q = 16; q > 0; q >>= 1) {
        o += __shfl_xor_sync(0xffffffffu, o, q);
        f += __shfl_xor_sync(0xffffffffu, f, q);
        bad += __shfl_xor_sync(0xffffffffu, bad, q);
    }
    if ((threadIdx.x & 31) == 0) {
        if (o) atomicAdd(&out[0], o);
        if (f) atomicAdd(&out[1], f);
        if (bad) atomicAdd(&out[2], bad);
    }
}

// Certificate: every node balanced and every residual arc with reduced cost
// >= -1 in scaled units (1-optimal with K = n + 1 means optimal).
__global__ void k_certify(const int64_t* __restrict__ rp, const int32_t* __restrict__ hd,
                          const uint32_t* __restrict__ cw, const int64_t* __restrict__ x,
                          const int64_t* __restrict__ e, const int64_t* __restrict__ p, int64_t n, int64_t K,
                          unsigned long long* __restrict__ viol) {
    int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (u >= n) return;
    unsigned long long bad = 0;
    if (lane == 0 && e[u] != 0) bad++;
    int64_t pu = p[u];
    for (int64_t s = rp[u] + lane; s < rp[u + 1]; s += 32) {
        int64_t rc, cap;
        if (residual(cw[s], x[s], K, &rc, &cap) && rc - pu + p[hd[s]] < -1) bad++;
    }
    for (int q = 16; q > 0; q >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, q);
    if (lane == 0 && bad) atomicAdd(viol, bad);
}

__global__ void k_copy_i64(const int64_t* __restrict__ src, int64_t* __restrict__ dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

__global__ void k_check_network(const int64_t* __restrict__ rp, const int32_t* __restrict__ hd, int64_t n, int64_t m,
                                unsigned long long* __restrict__ bad) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int64_t a0 = rp[u], a1 = rp[u + 1];
    bool b = (u == 0 && a0 != 0) || (u == n - 1 && a1 != m) || a1 < a0 || a0 < 0 || a1 > m;
    if (!b) {
        int64_t prev = -1;
        for (int64_t a = a0; a < a1; a++) {
            int64_t h = hd[a];
            if (h < 0 || h >= n || h == u || h <= prev) {
                b = true;
                break;
            }
            prev = h;
        }
    }
    if (b) atomicAdd(bad, 1ull);
}

pd_status validate_network(Ctx* c, const pd_network& net, cudaStream_t st) {
    int64_t n = net.n_nodes, m = net.n_arcs;
    if (n == 0) return m == 0 ? PD_OK : fail(c, PD_EINVAL, "arcs without nodes");
    if (!net.row_ptr || !net.supply || (m > 0 && (!net.head || !net.cost))) return fail(c, PD_EINVAL, "NULL network array");
    unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
    if (!sm) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, sizeof(unsigned long long), st));
    k_check_network<<<grid_for(n, 256), 256, 0, st>>>(net.row_ptr, net.head, n, m, sm); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (c->h_small[0])
        return fail(c, PD_EINVAL, "network needs row_ptr[0] = 0, row_ptr[n] = m, and in every row strictly "
                                  "increasing heads in [0, n) without self-loops");
    return PD_OK;
}

pd_status stage_solve(Ctx* c, const pd_network& net, const pd_opts& o, SolveStats* out, cudaStream_t st) {
    *out = SolveStats{};
    int64_t n = net.n_nodes, m = net.n_arcs;
    if (n <= 0) return PD_OK;
    if (m >= (int64_t(1) << 32) - 1) return fail(c, PD_ECAPACITY, "more than 2^32 - 2 arcs");
    int hb = bits_for((uint64_t)n + 1);
    if (2 * hb > 64) return fail(c, PD_ECAPACITY, "too many nodes");
    uint64_t sent = (2 * hb >= 64) ? ~0ull : ((1ull << (2 * hb)) - 1);
    unsigned long long* sm = bufT<unsigned long long>(c, B_SMALL, 64);
    int32_t* tail = bufT<int32_t>(c, B_S_TAIL, m);
    int64_t* pair = bufT<int64_t>(c, B_S_PAIR, m);
    uint64_t* xkey = bufT<uint64_t>(c, B_S_XKEY, m);
    uint64_t* xkey2 = bufT<uint64_t>(c, B_S_XKEY2, m);
    uint32_t* xval = bufT<uint32_t>(c, B_S_XVAL, m);
    uint32_t* xval2 = bufT<uint32_t>(c, B_S_XVAL2, m);
    int64_t* xptr = bufT<int64_t>(c, B_S_XPTR, n + 1);
    int64_t* xpos = bufT<int64_t>(c, B_S_XPOS, m);
    if (!sm || !tail || !pair || !xkey || !xkey2 || !xval || !xval2 || !xptr || !xpos) return PD_ENOMEM;
    PD_TRY_CUDA(c, cudaMemsetAsync(sm, 0, 64 * sizeof(unsigned long long), st));
    k_arc_tails<<<grid_for(m, 256), 256, 0, st>>>(net.row_ptr, n, m, tail); pd::count_launch();
    k_pairing<<<grid_for(m, 256), 256, 0, st>>>(net.row_ptr, net.head, net.cost, tail, m, hb, sent, pair, xkey, xval,
                                                 (int*)&sm[0], &sm[2]); pd::count_launch();
    k_max_cost<<<grid_for(m, 256), 256, 0, st>>>(net.cost, m, &sm[1]); pd::count_launch();
    PD_TRY_CUDA(c, cudaGetLastError());
    PD_TRY(sort_u64(c, xkey, xkey2, xval, xval2, m, 2 * hb, st));
    PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PD_TRY_CUDA(c, cudaStreamSynchronize(st));
    if (c->h_small[0] & 0xffffffff) return fail(c, PD_EOVERFLOW, "arc cost outside [0, 2^31)");
    int64_t cmax = c->h_small[1];
    {
        int64_t E = c->h_small[2];
        int64_t ms = m + E;
        // rows of the extras
        if (E > 0) {
            k_row_ptr<<<grid_for(E, 256), 256, 0, st>>>(xkey, E, hb, n, xptr); pd::count_launch();
        } else {
            PD_TRY_CUDA(c, cudaMemsetAsync(xptr, 0, sizeof(int64_t) * (n + 1), st));
        }
        int64_t* srp = bufT<int64_t>(c, B_S_ROWPTR, n + 1);
        int32_t* shd = bufT<int32_t>(c, B_S_HEAD, ms);
        uint32_t* scw = bufT<uint32_t>(c, B_S_CW, ms);
        int64_t* stw = bufT<int64_t>(c, B_S_TWIN, ms);
        int64_t* sx = bufT<int64_t>(c, B_S_X, ms);
        int64_t* se = bufT<int64_t>(c, B_S_E, n);
        int64_t* sp = bufT<int64_t>(c, B_S_P, n);
        int64_t* scur = bufT<int64_t>(c, B_S_CUR, n);
        int64_t* sd = bufT<int64_t>(c, B_S_D, n);
        int8_t* srl = bufT<int8_t>(c, B_S_RELAB, n);
        SolverCtl* ctl = bufT<SolverCtl>(c, B_S_CTL, 1);
        if (!srp || !shd || !scw || !stw || !sx || !se || !sp || !scur || !srl || !ctl || !sd) return PD_ENOMEM;
        k_sym_rowptr<<<grid_for(n + 1, 256), 256, 0, st>>>(net.row_ptr, xptr, n, srp); pd::count_launch();
        if (E > 0)
            k_fill_extra<<<grid_for(E, 256), 256, 0, st>>>(xkey, xval, E, hb, net.row_ptr, xptr, srp, net.cost, shd,
                                                           scw, stw, xpos); pd::count_launch();
        k_fill_dir<<<grid_for(m, 256), 256, 0, st>>>(net.row_ptr, net.head, net.cost, tail, pair, xpos, m, srp, shd,
                                                      scw, stw); pd::count_launch();
        PD_TRY_CUDA(c, cudaMemsetAsync(sx, 0, sizeof(int64_t) * ms, st));
        PD_TRY_CUDA(c, cudaMemsetAsync(sp, 0, sizeof(int64_t) * n, st));
        k_copy_i64<<<grid_for(n, 256), 256, 0, st>>>(net.supply, se, n); pd::count_launch();
        PD_TRY_CUDA(c, cudaMemsetAsync(ctl, 0, sizeof(SolverCtl), st));
        PD_TRY_CUDA(c, cudaGetLastError());

        int64_t K = n + 1;
        if (cmax > 0 && cmax > (INT64_MAX >> 2) / K) return fail(c, PD_EOVERFLOW, "scaled costs exceed 2^61");
        int alpha = o.alpha >= 2 ? o.alpha : 8;
        SolverArgs args;
        args.n = n;
        args.rp = srp;
        args.hd = shd;
        args.cw = scw;
        args.tw = stw;
        args.x = sx;
        args.e = se;
        args.p = sp;
        args.cur = scur;
        args.d = sd;
        args.update_every = o.update_every > 0 ? o.update_every : (o.update_every < 0 ? 0 : (n > 64 ? n : 64));
        args.seq_threshold = o.seq_threshold >= 0 ? o.seq_threshold : 64;
        args.seq_budget = 4 * n + 1024;
        args.q = bufT<int32_t>(c, B_S_Q, n);
        if (!args.q) return PD_ENOMEM;
        args.relab = srl;
        args.K = K;
        int64_t cm = cmax * K;
        args.eps0 = cm / alpha > 1 ? cm / alpha : 1;
        args.alpha = alpha;
        args.max_rounds = o.max_rounds > 0 ? o.max_rounds : (int64_t(1) << 40);
        args.spin_limit = int64_t(1) << 25;
        args.time_limit_ns = (o.time_limit_ms > 0 ? (uint64_t)o.time_limit_ms : 60000ull) * 1000000ull;
        args.ctl = ctl;
        int occ = 0;
        PD_TRY_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve, SV_THREADS, 0));
        if (occ < 1) return fail(c, PD_ECUDA, "solver kernel cannot be resident");
        // enough warps for the nodes, but no more blocks than needed: every
        // block takes part in every grid barrier
        int64_t per_sm = (n + (int64_t)c->sm_count * 64 - 1) / ((int64_t)c->sm_count * 64);
        if (per_sm < 1) per_sm = 1;
        if (per_sm > occ) per_sm = occ;
        if (per_sm > 4) per_sm = 4;
        int blocks = c->sm_count * (int)per_sm;
        void* kargs[] = {&args};
        PD_TRY_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_solve, dim3(blocks), dim3(SV_THREADS), kargs, 0, st));
        pd::count_launch();
        PD_TRY_CUDA(c, cudaMemsetAsync(sm + 4, 0, 8 * sizeof(unsigned long long), st));
        k_objective<<<grid_for(ms, 256), 256, 0, st>>>(scw, sx, ms, sm + 4); pd::count_launch();
        if (o.verify) k_certify<<<grid_for(n * 32, 256), 256, 0, st>>>(srp, shd, scw, sx, se, sp, n, K, sm + 8); pd::count_launch();
        PD_TRY_CUDA(c, cudaGetLastError());
        SolverCtl hc;
        PD_TRY_CUDA(c, cudaMemcpyAsync(&hc, ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaMemcpyAsync(c->h_small, sm, 16 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PD_TRY_CUDA(c, cudaStreamSynchronize(st));
        out->rounds = hc.rounds;
        out->pushes = hc.pushes;
        out->relabels = hc.relabels;
        out->repairs = hc.repairs;
        out->updates = hc.updates;
        out->update_passes = hc.update_passes;
        out->phases = hc.phases;
        if (hc.status & ERR_TIMEOUT) return fail(c, PD_ETIMEOUT, "solver round cap or a grid barrier wait ran out");
        if (hc.status & ERR_INFEASIBLE) return fail(c, PD_EINFEASIBLE, "a node with excess has no residual arc");
        if (hc.status & ERR_OVERFLOW) return fail(c, PD_EOVERFLOW, "a price left (-2^62, 2^62)");
        if (c->h_small[6]) return fail(c, PD_EINFEASIBLE, "flow against an arc direction");
        out->opt = c->h_small[4];
        out->slack = c->h_small[5];
        out->verified = o.verify ? (c->h_small[8] == 0 ? 1 : 0) : 0;
        if (o.verify && c->h_small[8] != 0) return fail(c, PD_EINFEASIBLE, "optimality certificate failed");
    }
    return PD_OK;
}

}  // namespace pd
