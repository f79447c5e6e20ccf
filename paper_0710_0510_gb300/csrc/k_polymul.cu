// Batched polynomial products in Z_p[X] by the DQT (Alg. 1) followed by
// REDQ (Alg. 2): one thread per pair.
//
//   pack:    a~ = sum_i a_i q^i, q = 2^s, by shifts (Sec. 2, power-of-two q)
//   product: r = a~ b~ in FP64; exact as hi + lo with lo = fma(a~, b~, -hi)
//            (or the single-rounded product when Eq. 2 holds for m = 53)
//   REDQ:    rop = floor(r/p) (one multiply-high), u_i = (r >> s i) -
//            p (rop >> s i), mu_{2k-2} = u_{2k-2}, mu_i = (u_i - q u_{i+1})
//            mod p through a p^2 table (Table 1, "p^2 extra memory, d
//            accesses").
// With QADIC_POLYMUL_INT_WORDS the product is taken in 64-bit integer
// words instead (Sec. 2 allows m = 64): one integer multiply, exact.
#include <algorithm>

#include "common.cuh"

namespace qadic {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxPairs = 4;   // pairs per thread per chunk: 1 for small batches, 4 for large

// Signed integer value of a double holding an exact integer of magnitude
// < 2^53, from its bit pattern (integer instructions only).
__device__ __forceinline__ int64_t f64_to_i64_exact(double x) {
    const int64_t bits = __double_as_longlong(x);
    const int64_t mag = (int64_t)f64_to_u64_exact(__longlong_as_double(bits & INT64_MAX));
    return bits < 0 ? -mag : mag;   // the sign bit, not an FP64 compare
}

// The K coefficient bytes of pair idx, byte j at bits 8j: one vector load
// for K = 1, 2, 4, 8 (when the base is aligned), byte loads otherwise.
template <int K>
__device__ __forceinline__ uint64_t load_pair(const uint8_t *__restrict__ base, int64_t idx,
                                              bool aligned) {
    if (K == 1) return __ldg(base + idx);
    if (K == 2 && aligned) return __ldg(reinterpret_cast<const uint16_t *>(base) + idx);
    if (K == 4 && aligned) return __ldg(reinterpret_cast<const uint32_t *>(base) + idx);
    if (K == 8 && aligned)
        return (uint64_t)__ldg(reinterpret_cast<const unsigned long long *>(base) + idx);
    uint64_t v = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) v |= (uint64_t)__ldg(base + idx * K + j) << (8 * j);
    return v;
}

// DQT of one operand (Alg. 1, packing with a power-of-two q): each
// coefficient byte taken mod p, then placed at bit s j.  The shifts are
// multiplies by 2^(s j) (pw[j]) so that each coefficient costs one
// multiply-add into the word.
template <int K>
__device__ __forceinline__ uint64_t pack_word(uint64_t bytes, uint32_t p, uint32_t m32,
                                              const uint64_t (&pw)[K]) {
    uint64_t w = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t c = mod_small((uint32_t)(bytes >> (8 * j)) & 0xffu, p, m32);
        w += (uint64_t)c * pw[j];
    }
    return w;
}

// Same, when the packed word fits 32 bits (K s <= 32).
template <int K>
__device__ __forceinline__ uint32_t pack_word32(uint64_t bytes, uint32_t p, uint32_t m32,
                                                const uint64_t (&pw)[K]) {
    uint32_t w = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t c = mod_small((uint32_t)(bytes >> (8 * j)) & 0xffu, p, m32);
        w += c * (uint32_t)pw[j];
    }
    return w;
}

// Nonzero iff some byte of x is >= p, in plain 32-bit arithmetic: for
// p <= 128, bit 7 of (b & 0x7f) + 128 - p (no carry out of the byte) is set
// iff the low seven bits reach p, and a byte with bit 7 set is >= p anyway;
// for p > 128, a byte is >= p iff bit 7 is set and (b & 0x7f) + 256 - p
// reaches 128.  add = (128 - p) or (256 - p) in every byte.
__device__ __forceinline__ uint32_t any_byte_ge(uint32_t x, uint32_t add, bool p_low) {
    const uint32_t t = (x & 0x7f7f7f7fu) + add;
    return (p_low ? (t | x) : (t & x)) & 0x80808080u;
}

struct ByteGe {
    uint32_t add;
    bool p_low;
};

// Packed word of one operand: the bytes taken mod p and spaced by s bits.
// When every byte is already below p (checked four at a time) the reduction
// is skipped, and with s = 8 the loaded bytes are the packed word as they
// stand.  Same value either way.
template <int K>
__device__ __forceinline__ uint64_t operand_word(uint64_t bytes, uint32_t p, uint32_t m32,
                                                 ByteGe ge, uint32_t s, const uint64_t (&pw)[K]) {
    const bool canon = (any_byte_ge((uint32_t)bytes, ge.add, ge.p_low) |
                        (K > 4 ? any_byte_ge((uint32_t)(bytes >> 32), ge.add, ge.p_low) : 0u)) == 0;
    if (canon) {
        if (s == 8) return bytes;
        uint64_t w = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) w += ((bytes >> (8 * j)) & 0xffu) * pw[j];
        return w;
    }
    return pack_word<K>(bytes, p, m32, pw);
}

template <int K>
__device__ __forceinline__ uint32_t operand_word32(uint64_t bytes, uint32_t p, uint32_t m32,
                                                   ByteGe ge, uint32_t s, const uint64_t (&pw)[K]) {
    const uint32_t lo = (uint32_t)bytes;   // with s = 8 and K s <= 32 all K <= 4 bytes are here
    const bool canon = (any_byte_ge(lo, ge.add, ge.p_low) |
                        (K > 4 ? any_byte_ge((uint32_t)(bytes >> 32), ge.add, ge.p_low) : 0u)) == 0;
    if (canon) {
        if (s == 8) return lo;
        uint32_t w = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) w += ((uint32_t)(bytes >> (8 * j)) & 0xffu) * (uint32_t)pw[j];
        return w;
    }
    return pack_word32<K>(bytes, p, m32, pw);
}

// r = a~ b~ from two packed operand words (each below 2^53): MODE 2 one
// 64-bit integer multiply; MODE 1 the single-rounded FP64 product (Eq. 2
// with m = 53 must hold); MODE 0 the FP64 product made exact as hi + lo
// with lo = fma(a, b, -hi).  Conversions to and from double work on the bit
// patterns, so the FP64 pipe sees only the multiply and the FMA.
// A nonzero v < 2^32 as a double, from its bit pattern.
__device__ __forceinline__ double u32_to_f64_exact(uint32_t v) {
    const int top = 31 - __clz(v | 1u);
    const uint64_t mant = ((uint64_t)v << (52 - top)) & ((1ull << 52) - 1);
    const uint64_t bits = v ? (((uint64_t)(1023 + top) << 52) | mant) : 0ull;
    return __longlong_as_double((long long)bits);
}

// NARROW: both words below 2^32.
template <int MODE, bool NARROW = false>
__device__ __forceinline__ uint64_t pair_product(uint64_t aw, uint64_t bw) {
    if (MODE == 2) return aw * bw;   // < 2^((2k-1) s) <= 2^63: exact in 64 bits
    const double ad = NARROW ? u32_to_f64_exact((uint32_t)aw) : u64_to_f64_exact(aw);
    const double bd = NARROW ? u32_to_f64_exact((uint32_t)bw) : u64_to_f64_exact(bw);
    const double hi = ad * bd;
    if (MODE == 1) return f64_to_u64_exact(hi);
    // hi may reach 2^63: read it as mantissa << exponent
    const uint64_t bits = (uint64_t)__double_as_longlong(hi);
    const uint32_t e = (uint32_t)(bits >> 52);
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const uint64_t hi_u = e >= 1075 ? mant << (e - 1075) : f64_to_u64_exact(hi);
    const double lo = fma(ad, bd, -hi);   // exact error term
    return hi_u + (uint64_t)f64_to_i64_exact(lo);
}

// MODE 0: FP64 product made exact as hi + lo (lo = fma(a, b, -hi));
// MODE 1: single-rounded FP64 product (Eq. 2 with m = 53 must hold);
// MODE 2: 64-bit integer words, r = a~ b~ exactly (Sec. 2 allows m = 64).
// The conversions between the packed integers and doubles are done on the
// bit patterns, so the FP64 pipe only sees the multiply (and the FMA).
// K (the number of coefficients of an operand) is a template argument so
// that every loop over coefficients unrolls and every shift amount is a
// register computed once per thread.
template <int MODE, int K, int kPairs>
__global__ void __launch_bounds__(kThreads)
polymul_kernel(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b,
               uint8_t *__restrict__ out, int64_t count, uint32_t p, uint32_t s,
               uint32_t qneg_mod_p, Div64 divp, Div32 divp32) {
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr int kChunk = kThreads * kPairs;
    constexpr int D = 2 * K - 1;
    uint8_t *corr = smem;                           // p*p entries
    uint8_t *stage = smem + ((p * p + 15) & ~15u);  // kChunk * D bytes (16-byte aligned)

    const uint32_t m32 = (uint32_t)((((uint64_t)1 << 32) + p - 1) / p);
    const ByteGe ge{(p <= 128 ? 128u - p : 256u - p) * 0x01010101u, p <= 128};   // p <= 251
    for (uint32_t i = threadIdx.x; i < p * p; i += blockDim.x) {
        const uint32_t x = i / p, y = i % p;      // table index x*p + y -> (x + (-q) y) mod p
        corr[i] = (uint8_t)mod_small(x + qneg_mod_p * y, p, m32);
    }
    __syncthreads();

    uint64_t pw[K];
#pragma unroll
    for (int j = 0; j < K; ++j) pw[j] = 1ull << (s * j);
    const bool narrow = s * K <= 32;   // packed operands fit 32 bits
    const bool aligned = ((((uintptr_t)a | (uintptr_t)b) & (K == 8 ? 7 : K == 4 ? 3 : 1)) == 0);

    // Grid-stride over chunks of kPairs * kThreads pairs (the table is built
    // once).  Each thread issues the operand loads of its kPairs pairs first,
    // so several loads are in flight, then reduces them; the chunk's output
    // bytes leave through shared memory as 16-byte stores.
    for (int64_t base = (int64_t)blockIdx.x * kChunk; base < count;
         base += (int64_t)gridDim.x * kChunk) {
        uint64_t va[kPairs], vb[kPairs];
#pragma unroll
        for (int j = 0; j < kPairs; ++j) {
            const int64_t idx = base + j * kThreads + threadIdx.x;
            va[j] = idx < count ? load_pair<K>(a, idx, aligned) : 0;
            vb[j] = idx < count ? load_pair<K>(b, idx, aligned) : 0;
        }
#pragma unroll
        for (int j = 0; j < kPairs; ++j) {
            const int64_t idx = base + j * kThreads + threadIdx.x;
            if (idx >= count) break;
            uint64_t r;
            if (MODE == 2 && narrow)
                r = (uint64_t)operand_word32<K>(va[j], p, m32, ge, s, pw) *
                    operand_word32<K>(vb[j], p, m32, ge, s, pw);
            else
                r = pair_product<MODE>(operand_word<K>(va[j], p, m32, ge, s, pw),
                                       operand_word<K>(vb[j], p, m32, ge, s, pw));
            uint8_t *dst = stage + (j * kThreads + threadIdx.x) * D;
            {
                // REDQ (Alg. 2): rop = floor(r/p); u_i = floor(r/q^i) - p
                // floor(rop/q^i) needs only the low 32 bits of each shifted
                // word (u_i < p).
                const uint64_t rop = div64(r, divp);
                uint32_t u_next = 0;
#pragma unroll
                for (int i = D - 1; i >= 0; --i) {
                    const uint32_t sh = s * i;
                    const uint32_t ui = (uint32_t)(r >> sh) - p * (uint32_t)(rop >> sh);
                    dst[i] = (i == D - 1) ? (uint8_t)ui : corr[ui * p + u_next];
                    u_next = ui;
                }
            }
        }
        __syncthreads();
        // write-out of the chunk's contiguous output range
        const int64_t nvalid = (count - base) < kChunk ? (count - base) : kChunk;
        const int64_t nbytes = nvalid * D;
        uint8_t *gout = out + base * D;
        if (nbytes % 16 == 0 && ((uintptr_t)gout & 15) == 0) {
            const uint4 *src = reinterpret_cast<const uint4 *>(stage);
            uint4 *g4 = reinterpret_cast<uint4 *>(gout);
            for (int64_t i = threadIdx.x; i < nbytes / 16; i += blockDim.x) g4[i] = src[i];
        } else {
            for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) gout[i] = stage[i];
        }
        __syncthreads();
    }
}

// q = 2^8 and K <= 4 (the packed operands are their K coefficient bytes
// and r < 2^56 has its base-q digits as its bytes): four consecutive pairs
// per thread.  Their operand bytes (4K per operand, contiguous) come in with
// one vector load when aligned, one SWAR test says whether every byte is
// already below p, and the 4(2K-1) output bytes leave as 32-bit words into
// shared memory.  REDQ (Alg. 2) runs on the two 32-bit halves of r
// separately -- each half is a q-adic word of its own, since no digit
// carries into the next -- with one 32-bit floor by p per half, constant
// byte shifts and the p^2 correction table.
template <int MODE, int K>
__global__ void __launch_bounds__(kThreads)
polymul_q8_kernel(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b,
                  uint8_t *__restrict__ out, int64_t count, uint32_t p, uint32_t s,
                  uint32_t qneg_mod_p, Div64 divp, Div32 divp32) {
    static_assert(K >= 1 && K <= 4, "two 32-bit halves hold the 2K-1 digits");
    constexpr int G = 4;                 // pairs per thread
    constexpr int D = 2 * K - 1;         // output bytes per pair; G D bytes = D words per thread
    constexpr int kChunk = kThreads * G;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *corr = smem;                                      // p*p entries
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + ((p * p + 15) & ~15u));

    const uint32_t m32 = (uint32_t)((((uint64_t)1 << 32) + p - 1) / p);
    const ByteGe ge{(p <= 128 ? 128u - p : 256u - p) * 0x01010101u, p <= 128};
    for (uint32_t i = threadIdx.x; i < p * p; i += blockDim.x) {
        const uint32_t x = i / p, y = i % p;      // table index x*p + y -> (x + (-q) y) mod p
        corr[i] = (uint8_t)mod_small(x + qneg_mod_p * y, p, m32);
    }
    __syncthreads();
    // a group's 4K bytes start on a 4K-byte boundary of each operand
    const bool vec = ((((uintptr_t)a | (uintptr_t)b) & (K == 3 ? 3 : 4 * K - 1)) == 0);

    // the group's operand bytes (little-endian) of the chunk at `base`
    auto load_group = [&](int64_t base, uint32_t (&wa)[K], uint32_t (&wb)[K]) {
        const int64_t pair0 = base + (int64_t)threadIdx.x * G;
        if (vec && pair0 + G <= count) {
            const uint8_t *pa = a + pair0 * K, *pb = b + pair0 * K;
            if constexpr (K == 4) {
                const uint4 x = __ldcs(reinterpret_cast<const uint4 *>(pa));
                const uint4 y = __ldcs(reinterpret_cast<const uint4 *>(pb));
                wa[0] = x.x; wa[1] = x.y; wa[2] = x.z; wa[3] = x.w;
                wb[0] = y.x; wb[1] = y.y; wb[2] = y.z; wb[3] = y.w;
            } else if constexpr (K == 2) {
                const uint2 x = __ldcs(reinterpret_cast<const uint2 *>(pa));
                const uint2 y = __ldcs(reinterpret_cast<const uint2 *>(pb));
                wa[0] = x.x; wa[1] = x.y;
                wb[0] = y.x; wb[1] = y.y;
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    wa[j] = __ldcs(reinterpret_cast<const uint32_t *>(pa) + j);
                    wb[j] = __ldcs(reinterpret_cast<const uint32_t *>(pb) + j);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j) wa[j] = wb[j] = 0;
#pragma unroll
            for (int x = 0; x < 4 * K; ++x)
                if (pair0 + x / K < count) {
                    wa[x / 4] |= (uint32_t)__ldg(a + pair0 * K + x) << (8 * (x % 4));
                    wb[x / 4] |= (uint32_t)__ldg(b + pair0 * K + x) << (8 * (x % 4));
                }
        }
    };
    const int64_t step = (int64_t)gridDim.x * kChunk;
    uint32_t na[K], nb[K];   // the next chunk's bytes, loaded while this one is worked on
    if ((int64_t)blockIdx.x * kChunk < count) load_group((int64_t)blockIdx.x * kChunk, na, nb);
    for (int64_t base = (int64_t)blockIdx.x * kChunk; base < count; base += step) {
        uint32_t wa[K], wb[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            wa[j] = na[j];
            wb[j] = nb[j];
        }
        if (base + step < count) load_group(base + step, na, nb);
        uint32_t any = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) any |= any_byte_ge(wa[j], ge.add, ge.p_low) | any_byte_ge(wb[j], ge.add, ge.p_low);
        uint32_t ow[D];                 // the group's G D output bytes
#pragma unroll
        for (int j = 0; j < D; ++j) ow[j] = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            // pair g's K bytes: bits 8 K g .. of the group
            uint32_t av, bv;
            {
                constexpr int kMask = K == 4 ? -1 : (1 << (8 * K)) - 1;
                const int bit = 8 * K * g, w = bit / 32, sh = bit % 32;
                const uint64_t a2 = (uint64_t)wa[w] | (w + 1 < K ? (uint64_t)wa[w + 1] << 32 : 0ull);
                const uint64_t b2 = (uint64_t)wb[w] | (w + 1 < K ? (uint64_t)wb[w + 1] << 32 : 0ull);
                av = (uint32_t)(a2 >> sh) & (uint32_t)kMask;
                bv = (uint32_t)(b2 >> sh) & (uint32_t)kMask;
            }
            if (any) {   // some byte of the group not below p: DQT with each byte taken mod p
                uint32_t ra = 0, rb = 0;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    ra |= mod_small((av >> (8 * j)) & 0xffu, p, m32) << (8 * j);
                    rb |= mod_small((bv >> (8 * j)) & 0xffu, p, m32) << (8 * j);
                }
                av = ra;
                bv = rb;
            }
            const uint64_t r = pair_product<MODE, true>(av, bv);
            // REDQ per 32-bit half x: o = floor(x/p), u_i = floor(x/q^i) -
            // p floor(o/q^i), mu_i = (u_i - q u_{i+1}) mod p through the p^2
            // table, the half's top digit mu = u
            const uint32_t x[2] = {(uint32_t)r, (uint32_t)(r >> 32)};
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                constexpr int kLo[2] = {0, 4};
                const int nd = D - kLo[hf] < 4 ? D - kLo[hf] : 4;
                if (nd <= 0) break;
                const uint32_t o = div32(x[hf], divp32);
                uint32_t u_next = 0;
#pragma unroll
                for (int i = 3; i >= 0; --i) {
                    if (i >= nd) continue;
                    const uint32_t ui = (x[hf] >> (8 * i)) - p * (o >> (8 * i));
                    const uint32_t mu = (i == nd - 1) ? ui : corr[ui * p + u_next];
                    const int ob = g * D + kLo[hf] + i;   // output byte of the group
                    ow[ob / 4] |= mu << (8 * (ob % 4));
                    u_next = ui;
                }
            }
        }
        // D words per thread, lanes D words apart (D odd: no bank conflicts)
#pragma unroll
        for (int j = 0; j < D; ++j) stage[threadIdx.x * D + j] = ow[j];
        __syncthreads();
        // write-out of the chunk's contiguous output range
        const int64_t nvalid = (count - base) < kChunk ? (count - base) : kChunk;
        const int64_t nbytes = nvalid * D;
        uint8_t *gout = out + base * D;
        const uint8_t *sb = reinterpret_cast<const uint8_t *>(stage);
        if (nbytes % 16 == 0 && ((uintptr_t)gout & 15) == 0) {
            const uint4 *src = reinterpret_cast<const uint4 *>(stage);
            uint4 *g4 = reinterpret_cast<uint4 *>(gout);
            for (int64_t i = threadIdx.x; i < nbytes / 16; i += blockDim.x) __stcs(g4 + i, src[i]);
        } else {
            for (int64_t i = threadIdx.x; i < nbytes; i += blockDim.x) gout[i] = sb[i];
        }
        __syncthreads();
    }
}

using PolymulKernel = void (*)(const uint8_t *, const uint8_t *, uint8_t *, int64_t, uint32_t,
                               uint32_t, uint32_t, Div64, Div32);

template <int MODE, int K>
PolymulKernel pick_kernel(int pairs, bool q8) {
    if constexpr (K <= 4) {
        if (q8) return polymul_q8_kernel<MODE, K>;
    }
    return pairs == kMaxPairs ? polymul_kernel<MODE, K, kMaxPairs> : polymul_kernel<MODE, K, 1>;
}

template <int K>
PolymulKernel pick_kernel(int mode, int pairs, bool q8) {
    return mode == 2 ? pick_kernel<2, K>(pairs, q8)
                     : mode == 1 ? pick_kernel<1, K>(pairs, q8) : pick_kernel<0, K>(pairs, q8);
}

PolymulKernel select_kernel(uint32_t k, int mode, int pairs, bool q8) {
    switch (k) {
        case 1: return pick_kernel<1>(mode, pairs, q8);
        case 2: return pick_kernel<2>(mode, pairs, q8);
        case 3: return pick_kernel<3>(mode, pairs, q8);
        case 4: return pick_kernel<4>(mode, pairs, q8);
        case 5: return pick_kernel<5>(mode, pairs, q8);
        case 6: return pick_kernel<6>(mode, pairs, q8);
        case 7: return pick_kernel<7>(mode, pairs, q8);
        default: return pick_kernel<8>(mode, pairs, q8);
    }
}

}  // namespace

int launch_polymul(uint32_t p, uint32_t k, uint32_t log2_q, int mode, const uint8_t *a,
                   const uint8_t *b, uint8_t *out, int64_t count, cudaStream_t stream) {
    const uint64_t q = 1ull << log2_q;
    const uint32_t qneg = (uint32_t)((p - q % p) % p);
    int dev = 0;
    cudaGetDevice(&dev);
    static int sms_of[64] = {0};   // SM count per device, queried once
    int sms = dev >= 0 && dev < 64 ? sms_of[dev] : 0;
    if (sms == 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (dev >= 0 && dev < 64) sms_of[dev] = sms;
    }
    // four pairs per thread once the batch fills every SM twice over with
    // them; with q = 2^8 and k <= 4 always four consecutive pairs per thread
    const bool q8 = log2_q == 8 && k <= 4;
    const int pairs = q8 || count >= (int64_t)sms * kThreads * kMaxPairs * 2 ? kMaxPairs : 1;
    const int64_t chunk = (int64_t)kThreads * pairs;
    const size_t smem = ((p * p + 15) & ~15u) + (size_t)chunk * (2 * k - 1);
    const PolymulKernel kern = select_kernel(k, mode, pairs, q8);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return set_error(QADIC_E_CUDA, "smem attribute: %s",
                             cudaGetErrorString(cudaGetLastError()));
    }
    int64_t blocks = (count + chunk - 1) / chunk;
    blocks = std::min<int64_t>(blocks, resident_blocks(kern, kThreads, smem));
    kern<<<(unsigned)blocks, kThreads, smem, stream>>>(a, b, out, count, p, log2_q, qneg,
                                                       make_div64(p), make_div32(p));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "polymul launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace qadic
