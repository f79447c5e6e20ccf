// Device helpers shared by the kernels of libqadic.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "qadic_internal.h"

namespace qadic {

// Division by an invariant integer d (1 <= d < 2^63) with one multiply-high,
// after Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), Fig. 4.1: with l = ceil(log2 d) and
// m = floor(2^64 (2^l - d) / d) + 1, floor(n/d) = (t + ((n - t) >> 1)) >> (l-1)
// where t = mulhi(m, n), for every 64-bit n.
struct Div64 {
    uint64_t m;
    uint32_t sh1, sh2;
};

inline Div64 make_div64(uint64_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned __int128 num = two64 * (((unsigned __int128)1 << l) - d);
    Div64 r;
    r.m = (uint64_t)(num / d + 1);
    r.sh1 = l < 1 ? l : 1;
    r.sh2 = l >= 1 ? l - 1 : 0;
    return r;
}

__device__ __forceinline__ uint64_t div64(uint64_t n, const Div64 &d) {
    const uint64_t t = __umul64hi(d.m, n);
    return (t + ((n - t) >> d.sh1)) >> d.sh2;
}

// The same for 32-bit n and 1 <= d < 2^32 (l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1).
struct Div32 {
    uint32_t m;
    uint32_t sh1, sh2;
};

inline Div32 make_div32(uint32_t d) {
    uint32_t l = 0;
    while (((uint64_t)1 << l) < d) ++l;
    const uint64_t num = ((uint64_t)1 << 32) * ((((uint64_t)1) << l) - d);
    Div32 r;
    r.m = (uint32_t)(num / d + 1);
    r.sh1 = l < 1 ? l : 1;
    r.sh2 = l >= 1 ? l - 1 : 0;
    return r;
}

__device__ __forceinline__ Div32 make_div32_device(uint32_t d) {
    const uint32_t l = d > 1 ? 32 - __clz(d - 1) : 0;   // ceil(log2 d)
    const uint64_t num = ((uint64_t)1 << 32) * ((((uint64_t)1) << l) - d);
    Div32 r;
    r.m = (uint32_t)(num / d + 1);
    r.sh1 = l < 1 ? l : 1;
    r.sh2 = l >= 1 ? l - 1 : 0;
    return r;
}

__device__ __forceinline__ uint32_t div32(uint32_t n, const Div32 &d) {
    const uint32_t t = __umulhi(d.m, n);
    return (t + ((n - t) >> d.sh1)) >> d.sh2;
}

// x mod d for 0 <= x < 2^16 and d < 256: floor(x/d) = mulhi(x, ceil(2^32/d))
// (the round-up error (m d - 2^32) x / 2^32 < d x / 2^32 stays below 1/d).
__device__ __forceinline__ uint32_t mod_small(uint32_t x, uint32_t d, uint32_t m32) {
    return x - d * __umulhi(x, m32);
}

inline uint32_t make_mod_small(uint32_t d) {
    return (uint32_t)((((uint64_t)1 << 32) + d - 1) / d);
}

// Exact integer value of a non-negative double holding an integer < 2^53,
// read from its bit pattern (no floating-point unit involved).
// For a non-negative x < 2^53 this is floor(x) (a truncation of the fraction
// bits); other bit patterns give some value without faulting.
__device__ __forceinline__ uint64_t f64_to_u64_exact(double x) {
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const uint32_t e = (uint32_t)(bits >> 52);
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const uint32_t sh = min(1075u - e, 63u);   // e < 1023 (x < 1): shift >= 53 -> 0
    return mant >> sh;
}

// Double holding the integer v < 2^53, built from its bit pattern.
__device__ __forceinline__ double u64_to_f64_exact(uint64_t v) {
    if (v == 0) return 0.0;
    const int top = 63 - __clzll((long long)v);
    const uint64_t mant = (v << (52 - top)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)((((uint64_t)(1023 + top)) << 52) | mant));
}

// Blocks of `kern` resident on the whole device (SMs x blocks per SM at
// this block size and shared memory), cached per device and configuration:
// for the short launches (65,536 polynomial pairs take about 2 us) the
// occupancy query would otherwise cost more than the kernel.
template <typename Kern>
inline int64_t resident_blocks(Kern kern, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int64_t> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, (const void *)kern, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t r = (int64_t)std::max(sms, 1) * per_sm;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = r;
    return r;
}

__device__ __forceinline__ void record_timeout(int *status, int site) {
    if (status) atomicCAS(status, 0, site);
}

}  // namespace qadic
