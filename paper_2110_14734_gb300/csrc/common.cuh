// Device helpers shared by the kernels of libpdw1 (not shared with the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PD_HD __host__ __device__ __forceinline__
#define PD_D __device__ __forceinline__

namespace pd {

// Kernel launches issued by this library: per host thread (for the per-call
// counts in pd_result) and in total over the process (pd_kernel_launches).
long long& launch_count_ref();
void count_launch_total();
inline void count_launch() {
    launch_count_ref()++;
    count_launch_total();
}

// Error bits raised by kernels into a device status word (host reads it back).
enum : uint32_t {
    ERR_INPUT = 1u,       // non-finite or out-of-range coordinate
    ERR_OVERFLOW = 2u,    // price or cost left its range
    ERR_TIMEOUT = 4u,     // bounded device wait or round cap ran out
    ERR_INFEASIBLE = 8u,  // a node with excess has no residual arc
    ERR_CAPACITY = 16u,   // a device-side capacity was exceeded
};

constexpr int64_t COORD_LIMIT = int64_t(1) << 29;  // |quantised coordinate| < 2^29

// floor(sqrt(v)) for v < 2^63: a first guess from a floating-point square
// root, then the two loops make it exact.  Below 2^44 the float root is within
// 0.4 of sqrt(v) (relative error < 1.5 * 2^-24 on a value < 2^22), so the loops
// run at most once or twice and the double-precision unit is not needed;
// above, a correctly rounded double root is at most one unit away.
PD_D uint64_t isqrt_u64(uint64_t v) {
    uint64_t r = v < (1ull << 44) ? (uint64_t)sqrtf((float)v) : (uint64_t)sqrt((double)v);
    while (r * r > v) r--;
    while ((r + 1) * (r + 1) <= v) r++;
    return r;
}

PD_D uint64_t ceil_sqrt_u64(uint64_t v) {
    uint64_t r = isqrt_u64(v);
    return (r * r < v) ? r + 1 : r;
}

// Rounded-up l2 cost between two quantised points (|coordinate| < 2^30).
PD_D int64_t cost_l2(int32_t x1, int32_t y1, int32_t x2, int32_t y2) {
    int64_t dx = (int64_t)x1 - x2, dy = (int64_t)y1 - y2;
    return (int64_t)ceil_sqrt_u64((uint64_t)(dx * dx) + (uint64_t)(dy * dy));
}

// Rounded-up distance to the diagonal: smallest c with 2 c^2 >= (y - x)^2.
PD_D int64_t cost_diag(int32_t x, int32_t y) {
    int64_t t = (int64_t)y - x;
    uint64_t t2 = (uint64_t)(t * t);
    return (int64_t)ceil_sqrt_u64((t2 + 1) >> 1);
}

// Cost of destroying a unit at (x, y) (arc to ā) or creating one there (from
// b̄): kappa * (distance to the diagonal) + tau quanta; kappa 1, tau 0 for
// persistence diagrams, anything else the unbalanced transport of the
// Conclusion (ā and b̄ as destructor and creator).
struct DiagCost {
    int32_t kappa;  // 0 or 1
    int32_t pad;
    int64_t tau;    // >= 0
};

PD_D int64_t cost_make(int32_t x, int32_t y, DiagCost dc) { return (dc.kappa ? cost_diag(x, y) : 0) + dc.tau; }

PD_HD int64_t floor_div(int64_t a, int64_t b) {  // b > 0
    int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

// Morton interleave with the usual magic masks: bit i of v -> bit 2i.
PD_HD uint64_t spread2(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

PD_HD uint64_t morton2(uint32_t x, uint32_t y) { return spread2(x) | (spread2(y) << 1); }

// SplitMix64 output finaliser (Steele, Lea & Flood, OOPSLA 2014).
PD_HD uint64_t splitmix_final(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Shift of the condensed node of lattice cell (cx, cy): two rounds of the
// finaliser on the seed and the cell give offsets uniform in [-P, P].
PD_HD void cell_shift(uint64_t seed, int64_t cx, int64_t cy, int64_t P, int64_t* dx, int64_t* dy) {
    if (P <= 0) {
        *dx = 0;
        *dy = 0;
        return;
    }
    const uint64_t g = 0x9E3779B97F4A7C15ull;
    uint64_t h1 = splitmix_final(seed ^ ((uint64_t)cx * g) ^ ((uint64_t)cy * 0xC2B2AE3D27D4EB4Full));
    uint64_t h2 = splitmix_final(h1 + g);
    uint64_t span = (uint64_t)(2 * P + 1);
    *dx = (int64_t)(h1 % span) - P;
    *dy = (int64_t)(h2 % span) - P;
}

PD_HD int bits_for(uint64_t v) {  // number of bits to hold values 0..v
    int b = 0;
    while (b < 64 && (v >> b) != 0) b++;
    return b;
}

// Loads that bypass L1: data written by other SMs earlier in the same kernel.
template <typename T>
PD_D T ld_cg(const T* p) {
    return __ldcg(p);
}

}  // namespace pd
