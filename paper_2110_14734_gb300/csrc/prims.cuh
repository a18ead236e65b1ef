// Device-wide primitives written for this library: exclusive scan (reduce,
// scan of tile sums, scan of tiles) and a stable LSD radix sort (8-bit
// digits; per-tile digit histograms, a scan over the digit-major histogram,
// and a stable in-tile scatter that ranks equal digits with warp match).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pd {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
PD_D T warp_incl_scan(T v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <typename T>
PD_D T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive scan of one value per thread over the block; returns the block
// total through *total (all threads).  blockDim.x must be a multiple of 32.
template <typename T>
PD_D T block_excl_scan(T v, T* total) {
    __shared__ T wsum[33];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = lane < nw ? wsum[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wsum[32] = si;
    }
    __syncthreads();
    T res = inc - v + wsum[w];
    *total = wsum[32];
    __syncthreads();
    return res;
}

template <typename T>
__global__ void k_tile_sum(const T* __restrict__ in, int64_t n, T* __restrict__ part) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    s = warp_sum(s);
    __shared__ T ws[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += ws[w];
        part[blockIdx.x] = t;
    }
}

// One block of 1024 threads scans all tile sums in place (exclusive).
template <typename T>
__global__ void k_scan_partials(T* part, int64_t nb, T* total) {
    T carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        T v = i < nb ? part[i] : T(0);
        T tot;
        T ex = block_excl_scan(v, &tot);
        if (i < nb) part[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_tile_scan(const T* in, T* out, int64_t n, const T* __restrict__ part) {
    __shared__ T tile[SCAN_TILE];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        tile[j * SCAN_THREADS + threadIdx.x] = i < n ? in[i] : T(0);
    }
    __syncthreads();
    T loc[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        loc[j] = tile[threadIdx.x * SCAN_ITEMS + j];
        s += loc[j];
    }
    T tot;
    T ex = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        tile[threadIdx.x * SCAN_ITEMS + j] = ex;
        ex += loc[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] = tile[j * SCAN_THREADS + threadIdx.x];
    }
}

inline int64_t scan_tiles(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// One block of 1024 threads scans in[0..n) into out (exclusive; in == out
// allowed: every element is read before the barrier that precedes its
// write), 4 consecutive elements a thread per step.  For short arrays, where
// the three-launch scan is all launch overhead.
constexpr int64_t SCAN_SMALL_MAX = int64_t(1) << 14;
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_small(const T* in, T* out, int64_t n, T* total) {
    T carry = 0;
    for (int64_t base = 0; base < n; base += 4 * (int64_t)blockDim.x) {
        const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
        T v[4];
        T s = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            v[j] = i0 + j < n ? in[i0 + j] : T(0);
            s += v[j];
        }
        T tot;
        T ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (i0 + j < n) out[i0 + j] = ex;
            ex += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// out[i] = sum of in[0..i-1]; in == out allowed.  part: scan_tiles(n) + 1
// elements of scratch; *total_dev (device, may be NULL) gets the sum.
template <typename T>
cudaError_t exclusive_scan(const T* in, T* out, int64_t n, T* part, T* total_dev, cudaStream_t st) {
    if (n <= 0) {
        if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(T), st);
        return cudaSuccess;
    }
    if (n <= SCAN_SMALL_MAX) {
        k_scan_small<T><<<1, 1024, 0, st>>>(in, out, n, total_dev); pd::count_launch();
        return cudaGetLastError();
    }
    int64_t nb = scan_tiles(n);
    k_tile_sum<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, part); pd::count_launch();
    k_scan_partials<T><<<1, 1024, 0, st>>>(part, nb, total_dev); pd::count_launch();
    k_tile_scan<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, part); pd::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LSD radix sort
// ---------------------------------------------------------------------------

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

inline int64_t radix_tiles(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }

template <typename K>
__global__ void k_radix_hist(const K* __restrict__ keys, int64_t n, int shift, int64_t nb,
                             int64_t* __restrict__ counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_ITEMS; j++) {
        int64_t i = base + (int64_t)j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void k_radix_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
                                uint32_t* __restrict__ vout, int64_t n, int shift, int64_t nb,
                                const int64_t* __restrict__ offs) {
    __shared__ uint32_t digit_base[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    digit_base[tid] = 0;
    const int64_t my_off = offs[(int64_t)tid * nb + blockIdx.x];
    __shared__ int64_t doff[256];
    doff[tid] = my_off;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const uint32_t lt = (1u << lane) - 1u;
    for (int c = 0; c < RS_ITEMS; c++) {
        int64_t i = base + (int64_t)c * RS_THREADS + tid;
        bool valid = i < n;
        K k = valid ? kin[i] : K(0);
        uint32_t v = (valid && vin) ? vin[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(k >> shift) & 0xFFu) : 256u;
#pragma unroll
        for (int q = 0; q < RS_THREADS / 32; q++) wcnt[q][tid] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = digit_base[d];
            for (int q = 0; q < w; q++) pre += wcnt[q][d];
            int64_t pos = doff[d] + pre + rank;
            kout[pos] = k;
            if (vin) vout[pos] = v;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int q = 0; q < RS_THREADS / 32; q++) add += wcnt[q][tid];
        digit_base[tid] += add;
        __syncthreads();
    }
}

template <typename K>
struct RadixScratch {
    K* k_alt;          // n keys
    uint32_t* v_alt;   // n values (if values are sorted)
    int64_t* counts;   // 256 * radix_tiles(n)
    int64_t* part;     // scan_tiles(256 * radix_tiles(n)) + 1
};

template <typename K>
inline size_t radix_counts_elems(int64_t n) {
    return (size_t)256 * (size_t)radix_tiles(n);
}

// Stable sort of (keys, vals) by the low `bits` bits of the keys.  vals may be
// NULL.  The result is left in keys / vals.
template <typename K>
cudaError_t radix_sort(K* keys, uint32_t* vals, int64_t n, int bits, RadixScratch<K> s, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    int64_t nb = radix_tiles(n);
    K* ka = keys;
    K* kb = s.k_alt;
    uint32_t* va = vals;
    uint32_t* vb = vals ? s.v_alt : nullptr;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_radix_hist<K><<<(unsigned)nb, RS_THREADS, 0, st>>>(ka, n, shift, nb, s.counts); pd::count_launch();
        cudaError_t e = exclusive_scan<int64_t>(s.counts, s.counts, 256 * nb, s.part, nullptr, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<K><<<(unsigned)nb, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, nb, s.counts); pd::count_launch();
        K* t = ka;
        ka = kb;
        kb = t;
        uint32_t* tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        if (vals) e = cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__global__ void k_fill_i64(int64_t* p, int64_t n, int64_t v);
__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v);

inline unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 2147483647LL) g = 2147483647LL;
    return (unsigned)g;
}

}  // namespace pd
