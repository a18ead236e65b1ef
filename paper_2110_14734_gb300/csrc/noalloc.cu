// pd_mcf_solve_noalloc: the min-cost flow solve of pd_mcf_solve without any
// device allocation.  All scratch lives in one file-scope __device__ array of
// fixed size; the network simplex kernel is the same one pd_mcf_solve runs.
//
// Every GPU that loads this library holds the array until the process exits.
// All calls share it and it keeps the previous call's contents; everything a
// solve reads is written by that solve first (the small status words are
// cleared with a memset), so nothing has to start at zero.  Two calls whose
// work overlaps on the GPU (different streams, or different host threads on
// the same device) race on the array and must not be issued.
#include <mutex>

#include "internal.h"
#include "netsimplex.cuh"
#include "prims.cuh"

namespace pd {
namespace {

constexpr int64_t NA_NODES = PD_NOALLOC_MAX_NODES;  // n_nodes + 1 (the simplex root) must not exceed this
constexpr int64_t NA_ARCS = PD_NOALLOC_MAX_ARCS;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_TAIL = 0;
constexpr size_t OFF_COST = OFF_TAIL + al(4 * NA_ARCS);
constexpr size_t OFF_PI = OFF_COST + al(4 * NA_ARCS);
constexpr size_t OFF_PRED = OFF_PI + al(8 * NA_NODES);
constexpr size_t OFF_PARENT = OFF_PRED + al(4 * NA_NODES);
constexpr size_t OFF_FLOW = OFF_PARENT + al(4 * NA_NODES);
constexpr size_t OFF_UP = OFF_FLOW + al(4 * NA_NODES);
constexpr size_t OFF_ORD = OFF_UP + al(NA_NODES);
constexpr size_t OFF_POS = OFF_ORD + al(4 * NA_NODES);
constexpr size_t OFF_SIZE = OFF_POS + al(4 * NA_NODES);
constexpr size_t OFF_TMP = OFF_SIZE + al(4 * NA_NODES);
constexpr size_t OFF_PATH = OFF_TMP + al(4 * NA_NODES);
constexpr size_t OFF_SEG = OFF_PATH + al(8 * NA_NODES);
constexpr size_t OFF_INST = OFF_SEG + al(12 * (2 * NA_NODES + 3));
constexpr size_t OFF_FLAGS = OFF_INST + al(sizeof(NSInst));
constexpr size_t SCRATCH_BYTES = OFF_FLAGS + al(64);
static_assert(SCRATCH_BYTES <= (size_t)12 << 20, "scratch of the allocation-free solve exceeds 12 MiB");

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

std::mutex g_setup_mu;
void* g_setup_addr[64] = {};

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_setup_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_setup_addr[dev] = p;
    }
    *out = g_setup_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" pd_status pd_mcf_solve_noalloc(const pd_network* net, int64_t* opt_out, void* stream) {
    if (!net || !opt_out) return PD_EINVAL;
    const int64_t n = net->n_nodes, m = net->n_arcs;
    if (n < 0 || m < 0) return PD_EINVAL;
    if (n == 0) {
        if (m != 0) return PD_EINVAL;
        *opt_out = 0;
        return PD_OK;
    }
    if (!net->row_ptr || !net->supply || (m > 0 && (!net->head || !net->cost))) return PD_EINVAL;
    if (n + 1 > NA_NODES || m > NA_ARCS) return PD_ECAPACITY;
    cudaStream_t st = (cudaStream_t)stream;
    void* basev = nullptr;
    if (scratch_address(&basev) != cudaSuccess) {
        cudaGetLastError();
        return PD_ECUDA;
    }
    unsigned char* base = (unsigned char*)basev;
    int32_t* tail = (int32_t*)(base + OFF_TAIL);
    int32_t* c32 = (int32_t*)(base + OFF_COST);
    unsigned long long* flags = (unsigned long long*)(base + OFF_FLAGS);
    NSInst* dinst = (NSInst*)(base + OFF_INST);

#define NA_TRY(expr)                              \
    do {                                          \
        if ((expr) != cudaSuccess) {              \
            cudaGetLastError();                   \
            return PD_ECUDA;                      \
        }                                         \
    } while (0)

    // validation, int32 costs, largest cost, total supply -- results in flags[0..3]
    NA_TRY(cudaMemsetAsync(flags, 0, 64, st));
    k_check_network<<<grid_for(n, 256), 256, 0, st>>>(net->row_ptr, net->head, n, m, flags); pd::count_launch();
    if (m > 0) {
        k_arc_tails<<<grid_for(m, 256), 256, 0, st>>>(net->row_ptr, n, m, tail); pd::count_launch();
        k_i64_to_i32_cost<<<grid_for(m, 256), 256, 0, st>>>(net->cost, m, c32, flags + 1); pd::count_launch();
        k_max_cost<<<grid_for(m, 256), 256, 0, st>>>(net->cost, m, flags + 2); pd::count_launch();
    }
    k_abs_sum<<<grid_for(n, 256), 256, 0, st>>>(net->supply, n, flags + 3); pd::count_launch();
    NA_TRY(cudaGetLastError());
    unsigned long long hf[4];
    NA_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (hf[0]) return PD_EINVAL;
    if (hf[1]) return PD_EOVERFLOW;
    if (hf[3] >= (1ull << 31)) return PD_ECAPACITY;
    const int64_t N1 = n + 1;
    const int64_t cmax = (int64_t)hf[2];
    if (cmax > (INT64_MAX / 8) / N1) return PD_EOVERFLOW;

    NSInst h{};
    h.n = (int32_t)n;
    h.m = m;
    h.mst = 0;
    h.nS = 0;
    h.nT = 1;
    h.cmat = nullptr;
    h.tail = tail;
    h.head = net->head;
    h.cost = c32;
    h.supply = net->supply;
    h.big = N1 * (cmax + 1) + 1;
    h.pi = (int64_t*)(base + OFF_PI);
    h.pred = (int32_t*)(base + OFF_PRED);
    h.parent = (int32_t*)(base + OFF_PARENT);
    h.flow = (int32_t*)(base + OFF_FLOW);
    h.up = (uint8_t*)(base + OFF_UP);
    h.ord = (int32_t*)(base + OFF_ORD);
    h.pos = (int32_t*)(base + OFF_POS);
    h.size = (int32_t*)(base + OFF_SIZE);
    h.tmp = (int32_t*)(base + OFF_TMP);
    h.path = (int32_t*)(base + OFF_PATH);
    h.seg = (int32_t*)(base + OFF_SEG);
    int64_t M = m + n;
    int64_t blk = (int64_t)sqrt((double)M);
    if (blk < 8 * NS_THREADS) blk = 8 * NS_THREADS;
    h.block = (blk + 7) & ~(int64_t)7;
    h.max_pivots = int64_t(1) << 40;
    h.time_limit_ns = 60000ull * 1000000ull;
    int dev = 0, max_optin = 0;
    NA_TRY(cudaGetDevice(&dev));
    NA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    h.smem_nodes = ns_smem_layout(N1, max_optin);
    const size_t smem = h.smem_nodes ? ns_smem_bytes(N1, h.smem_nodes) : 0;
    NA_TRY(ns_kernel_setup());
    NA_TRY(cudaMemcpyAsync(dinst, &h, sizeof(NSInst), cudaMemcpyHostToDevice, st));
    int32_t* order = (int32_t*)(flags + 4);  // zeroed with the flags: order = {0}, next = 0
    k_netsimplex<<<1, NS_THREADS, smem, st>>>(dinst, order, 1, order + 1); pd::count_launch();
    NA_TRY(cudaGetLastError());
    NSInst r;
    NA_TRY(cudaMemcpyAsync(&r, dinst, sizeof(NSInst), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
#undef NA_TRY
    if (r.status == 2) return PD_ETIMEOUT;
    if (r.status == 1 || r.status == 3) return PD_EINFEASIBLE;
    if (r.status != 0) return PD_ECUDA;
    *opt_out = r.opt;
    return PD_OK;
}
