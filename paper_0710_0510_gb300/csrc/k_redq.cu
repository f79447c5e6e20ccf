// Standalone REDQ (Alg. 2) over packed FP64 words: for each word
// r = sum_{j<=d} mu~_j q^j (q = 2^s) produce rho = sum_j (mu~_j mod p) q^j.
//
//   rop  = floor(r/p): Lemma 1 (multiply by 1/p rounded up, rounding up,
//          then floor) -- or an integer multiply-high (QADIC_REDQ_INT_FLOOR)
//   u_j  = (r >> s j) - p (rop >> s j)                       (Alg. 2, Thm. 2)
//   mu_d = u_d, mu_j = (u_j - q u_{j+1}) mod p               (Sec. 5.1: Q_d u)
// with the corrections evaluated per Table 1's time-memory trade-off:
//   mode 0: arithmetic (d mul/add/mod)
//   mode 1: p^2 table, d lookups   -- held in registers across the warp and
//           read with __shfl_sync when p^2 <= 64, else in shared memory
//   mode 2: p^k' table, ceil(d/(k'-1)) overlapping lookups (Alg. 3)
//   mode 3: full p^(d+1) table, one lookup returning rho itself
// Table indices are p-adic, sum u_i p^i (Sec. 5.3).
//
// A second kernel handles q a multiple of p (no corrections, divisions by
// q^j instead of shifts), the alternative choice of q left open in the
// paper's conclusion.
//
// HBM-bound: 8 bytes in and 8 bytes out per word; each thread streams pairs
// of words with 16-byte loads/stores over a grid sized to the SM count.
#include "common.cuh"

namespace qadic {

namespace {

constexpr int kThreads = 1024;
constexpr int kUnroll = 4;

struct RedqParams {
    uint32_t p, s, d;          // prime, log2 q, top digit index (ndigits - 1)
    uint32_t qneg;             // (-q) mod p
    uint32_t m32;              // ceil(2^32 / p) for mod_small
    uint32_t kk;               // table width k' (mode 2), d+1 (mode 3)
    uint32_t table_entries;
    double inv_p_up;           // 1/p rounded toward +infinity
    Div64 divp;
};

template <int MODE, bool INT_FLOOR>
__device__ __forceinline__ double redq_word(double x, const RedqParams &P, const uint8_t *t1,
                                            const uint64_t *tk, const double *tfull,
                                            uint32_t lane_t0, uint32_t lane_t1) {
    uint64_t r, rop;
    if (INT_FLOOR) {
        r = f64_to_u64_exact(x);
        rop = div64(r, P.divp);
    } else {
        r = f64_to_u64_exact(x);
        // Lemma 1: floor(RU(r * RU(1/p))); the floor of the positive product
        // is read off its bit pattern (truncation of the fraction bits).
        rop = f64_to_u64_exact(__dmul_ru(x, P.inv_p_up));
    }
    const uint32_t p = P.p, s = P.s, d = P.d;
    // u_j = floor(r/q^j) - p floor(rop/q^j) lies in [0, p) (Thm. 2), so it is
    // computed exactly from the low 32 bits of both shifted words.
    auto digit = [&](uint32_t j) -> uint32_t {
        const uint32_t sh = s * j;
        return (uint32_t)(r >> sh) - p * (uint32_t)(rop >> sh);
    };
    if (MODE == 3) {
        uint32_t idx = digit(d);   // sum_j u_j p^j by Horner from the top digit
        for (int j = (int)d - 1; j >= 0; --j) idx = idx * p + digit((uint32_t)j);
        return tfull[min(idx, P.table_entries - 1)];
    }
    if (MODE == 2) {
        // lookups at starts 0, kk-1, 2(kk-1), ..., the last clipped to d+1-kk
        const uint32_t kk = P.kk;
        uint64_t rho = 0;
        uint32_t start = 0;
        while (true) {
            const bool last = start + kk >= d + 1;
            const uint32_t st = last ? d + 1 - kk : start;
            uint32_t idx = digit(st + kk - 1);
            for (int j = (int)kk - 2; j >= 0; --j) idx = idx * p + digit(st + (uint32_t)j);
            const uint64_t e = tk[min(idx, P.table_entries - 1)];   // mu packed at s-bit spacing
            if (last) {
                // keep the positions not written by earlier lookups
                const uint32_t skip = start - st;
                const uint64_t keep = e >> (s * skip);
                rho |= keep << (s * start);
                break;
            }
            rho |= (e & ((1ull << (s * (kk - 1))) - 1)) << (s * st);
            start += kk - 1;
        }
        return u64_to_f64_exact(rho);
    }
    // MODE 0 / 1: walk j = d down to 0
    uint64_t rho = 0;
    uint32_t u_next = 0;
    for (int j = (int)d; j >= 0; --j) {
        const uint32_t sh = s * (uint32_t)j;
        const uint32_t u = digit((uint32_t)j);
        uint32_t mu;
        if (j == (int)d) {
            mu = u;
        } else if (MODE == 0) {
            mu = mod_small(u + P.qneg * u_next, p, P.m32);
        } else if (t1 == nullptr) {
            // p^2 <= 64: the table lives in two registers per lane
            const uint32_t idx = u * p + u_next;
            const uint32_t lo = __shfl_sync(0xffffffffu, lane_t0, idx & 31);
            const uint32_t hi = __shfl_sync(0xffffffffu, lane_t1, idx & 31);
            mu = idx < 32 ? lo : hi;
        } else {
            mu = t1[min(u * p + u_next, p * p - 1)];
        }
        rho |= (uint64_t)mu << sh;
        u_next = u;
    }
    return u64_to_f64_exact(rho);
}

template <int MODE, bool INT_FLOOR>
__global__ void __launch_bounds__(kThreads)
redq_kernel(const double *__restrict__ in, double *__restrict__ out, int64_t count, RedqParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint8_t *t1 = nullptr;
    const uint64_t *tk = nullptr;
    const double *tfull = nullptr;
    uint32_t lane_t0 = 0, lane_t1 = 0;
    const uint32_t p = P.p;

    if (MODE == 1) {
        if (p * p <= 64) {
            const uint32_t lane = threadIdx.x & 31;
            const uint32_t x0 = lane / p, y0 = lane % p, x1 = (lane + 32) / p, y1 = (lane + 32) % p;
            lane_t0 = lane < p * p ? mod_small(x0 + P.qneg * y0, p, P.m32) : 0;
            lane_t1 = lane + 32 < p * p ? mod_small(x1 + P.qneg * y1, p, P.m32) : 0;
        } else {
            uint8_t *t = smem;
            for (uint32_t i = threadIdx.x; i < p * p; i += blockDim.x)
                t[i] = (uint8_t)mod_small(i / p + P.qneg * (i % p), p, P.m32);
            t1 = t;
        }
    } else if (MODE == 2) {
        // entry for (u_0..u_{kk-1}) = packed (Q_{kk-1} u) at s-bit spacing
        uint64_t *t = (uint64_t *)smem;
        for (uint32_t i = threadIdx.x; i < P.table_entries; i += blockDim.x) {
            uint32_t u[16];
            uint32_t v = i;
            for (uint32_t j = 0; j < P.kk; ++j) {
                u[j] = v % p;
                v /= p;
            }
            uint64_t e = 0;
            for (uint32_t j = 0; j < P.kk; ++j) {
                const uint32_t mu = (j + 1 < P.kk) ? mod_small(u[j] + P.qneg * u[j + 1], p, P.m32)
                                                   : u[j];
                e |= (uint64_t)mu << (P.s * j);
            }
            t[i] = e;
        }
        tk = t;
    } else if (MODE == 3) {
        double *t = (double *)smem;
        for (uint32_t i = threadIdx.x; i < P.table_entries; i += blockDim.x) {
            uint32_t v = i, u_prev = 0;
            uint64_t rho = 0;
            uint32_t u[52];
            for (uint32_t j = 0; j <= P.d; ++j) {
                u[j] = v % p;
                v /= p;
            }
            for (int j = (int)P.d; j >= 0; --j) {
                const uint32_t mu =
                    (j == (int)P.d) ? u[j] : mod_small(u[j] + P.qneg * u_prev, p, P.m32);
                rho |= (uint64_t)mu << (P.s * j);
                u_prev = u[j];
            }
            t[i] = u64_to_f64_exact(rho);
        }
        tfull = t;
    }
    __syncthreads();

    // Warp-uniform grid-stride loop (every lane of a warp runs every
    // iteration, so the shuffle table of mode 1 always sees a full warp);
    // kUnroll 16-byte loads in flight per thread.
    const int64_t npairs = count >> 1;
    const double2 *in2 = reinterpret_cast<const double2 *>(in);
    double2 *out2 = reinterpret_cast<double2 *>(out);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t wb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); wb < npairs;
         wb += kUnroll * stride) {
        double2 w[kUnroll];
#pragma unroll
        for (int s = 0; s < kUnroll; ++s) {
            const int64_t i = wb + s * stride + lane;
            w[s] = i < npairs ? __ldcs(in2 + i) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int s = 0; s < kUnroll; ++s) {
            const int64_t i = wb + s * stride + lane;
            double2 o;
            o.x = redq_word<MODE, INT_FLOOR>(w[s].x, P, t1, tk, tfull, lane_t0, lane_t1);
            o.y = redq_word<MODE, INT_FLOOR>(w[s].y, P, t1, tk, tfull, lane_t0, lane_t1);
            if (i < npairs) __stcs(out2 + i, o);
        }
    }
    // odd tail word (all lanes take part in the shuffles above; here only
    // the shuffle-free modes can be used by a single thread)
    if ((count & 1) && blockIdx.x == 0) {
        const int64_t j = count - 1;
        if (MODE == 1 && t1 == nullptr) {
            const double v = redq_word<MODE, INT_FLOOR>(threadIdx.x < 32 ? in[j] : 0.0, P, t1, tk,
                                                        tfull, lane_t0, lane_t1);
            if (threadIdx.x == 0) out[j] = v;
        } else if (threadIdx.x == 0) {
            out[j] = redq_word<MODE, INT_FLOOR>(in[j], P, t1, tk, tfull, lane_t0, lane_t1);
        }
    }
}


// ---------------------------------------------------------------------------
// REDQ with q a multiple of p.  Then -q = 0 mod p, so Alg. 2's corrections
// vanish (mu_j = u_j, Thm. 2) and no table is needed; the price is that the
// divisions by q^j are no longer shifts.  They are taken as a chain:
// t_{j+1} = floor(t_j / q) with t_0 = r gives t_j = floor(r/q^j) (nested
// floors, Lemma 2), each step a Lemma 1 floor by 1/q rounded up (or an
// integer multiply-high).  Lemma 2 also gives floor(rop/q^j) =
// floor(t_j / p), so u_j = t_j - p floor(t_j/p) = t_j mod p, and as p | q,
// t_j mod p = (t_j - q t_{j+1}) mod p: the mod p of r's base-q digit, a
// number below q, by one small multiply-high.  d floors by q per word in all
// (instead of 2d+1 floors by q^j and p q^j).
constexpr int kMaxPqDigits = 51;

struct RedqPqParams {
    uint32_t p, d;
    uint32_t m32;                      // ceil(2^32 / p)
    uint32_t small_q;                  // q <= 2^32 / p: a digit's mod p is one 32-bit multiply-high
    uint32_t j32;                      // t_j < q^(d+1-j) <= 2^32 from this j on
    uint64_t q, small_lim;             // small_lim = floor(2^32 / p)
    double inv_q_up;                   // 1/q rounded toward +infinity
    Div64 div_q, div_p;
    Div32 div_q32;                     // floor(t / q) for t < 2^32 (q < 2^32)
    uint32_t split;                    // 1 <= j32 < d + 1 and q^j32 < 2^32 (see redq_pq_word_split)
    uint32_t qs;                       // q^j32 when split
    Div64 div_qs;                      // floor(r / q^j32)
    uint64_t qs_m;                     // floor(r / q^j32) = mulhi(r, qs_m) >> qs_s for r < 2^52
    uint32_t qs_s;
    double inv_qs_up;                  // 1/q^j32 rounded toward +infinity
    // digits in FP32 (QADIC_REDQ_F32_DIGITS, q^2 < 2^21)
    uint32_t Q;                        // q^2
    uint32_t k64;                      // leading floors by q^2 whose dividend may reach 2^32
    Div64 div_Q;
    Div32 div_Q32;
    float fq, inv_q, c_q;              // q, RN(1/q), RN(1/(2q) - 1/2)
    float fp, inv_p, c_p;              // the same for p
    uint64_t qpow[kMaxPqDigits];       // q^j
};

// x mod p for any 64-bit x: one 32-bit multiply-high below 2^32 / p (where
// the rounded-up reciprocal is exact), a 64-bit one above.
__device__ __forceinline__ uint32_t mod_p_any(uint64_t x, const RedqPqParams &P) {
    if (x < P.small_lim) return mod_small((uint32_t)x, P.p, P.m32);
    return (uint32_t)(x - P.p * div64(x, P.div_p));
}

// mod p of a base-q digit (< q for words below q^(d+1)).
__device__ __forceinline__ uint32_t mod_p_digit(uint64_t x, const RedqPqParams &P) {
    return P.small_q ? mod_small((uint32_t)x, P.p, P.m32) : mod_p_any(x, P);
}

// Any number of digits (loop over j, q^j from the parameter block).
template <bool INT_FLOOR>
__device__ __forceinline__ double redq_pq_word(double x, const RedqPqParams &P) {
    uint64_t t = f64_to_u64_exact(x);
    double tx = x;
    uint64_t rho = 0;
    for (uint32_t j = 0; j < P.d; ++j) {
        uint64_t tn;   // floor(r / q^(j+1))
        if (INT_FLOOR) {
            tn = div64(t, P.div_q);
        } else {
            tn = f64_to_u64_exact(__dmul_ru(tx, P.inv_q_up));
            tx = u64_to_f64_exact(tn);
        }
        rho += (uint64_t)mod_p_any(t - P.q * tn, P) * P.qpow[j];
        t = tn;
    }
    rho += (uint64_t)mod_p_any(t, P) * P.qpow[P.d];   // t_d < q for words below q^(d+1)
    return u64_to_f64_exact(rho);
}

// v < 2^52 as a double: the bits of 2^52 + v, less 2^52 (one FP64 add on
// a pipe the integer forms leave idle, instead of normalising the integer).
__device__ __forceinline__ double u52_to_f64(uint64_t v) {
    return __longlong_as_double((long long)(0x4330000000000000ull | v)) - 4503599627370496.0;
}

// When q^S < 2^32 for S = j32: one floor by q^S (64-bit integer, or
// Lemma 1 on the binary64 word) splits the word into t_S = floor(r / q^S)
// < 2^32 and r mod q^S < 2^32 (Lemma 2: the floors of t_S by q continue the
// chain), so every other floor is an exact 32-bit integer one and the two
// chains are independent, and rho = (Horner of the high digits) q^S +
// (Horner of the low digits), both sums below 2^32.
template <bool INT_FLOOR, int ND, int S>
__device__ __forceinline__ double redq_pq_word_split(double x, const RedqPqParams &P) {
    static_assert(S >= 1 && S < ND, "split point");
    const uint64_t t = f64_to_u64_exact(x);
    const uint64_t ts = INT_FLOOR ? __umul64hi(t, P.qs_m) >> P.qs_s
                                  : f64_to_u64_exact(__dmul_ru(x, P.inv_qs_up));
    uint32_t lo = (uint32_t)(t - (uint64_t)P.qs * ts), hi = (uint32_t)ts;
    const uint32_t q = (uint32_t)P.q;
    uint32_t u[ND];
#pragma unroll
    for (int j = 0; j < S - 1; ++j) {
        const uint32_t tn = div32(lo, P.div_q32);
        u[j] = mod_p_digit(lo - q * tn, P);
        lo = tn;
    }
    u[S - 1] = mod_p_digit(lo, P);   // lo < q now
#pragma unroll
    for (int j = S; j < ND - 1; ++j) {
        const uint32_t tn = div32(hi, P.div_q32);
        u[j] = mod_p_digit(hi - q * tn, P);
        hi = tn;
    }
    u[ND - 1] = mod_p_digit(hi, P);  // t_d < q
    uint32_t rh = u[ND - 1], rl = u[S - 1];
#pragma unroll
    for (int j = ND - 2; j >= S; --j) rh = rh * q + u[j];
#pragma unroll
    for (int j = S - 2; j >= 0; --j) rl = rl * q + u[j];
    return u52_to_f64((uint64_t)rh * P.qs + rl);
}

// ND = d + 1 digits known at compile time: the chain unrolls, the integer
// floors drop to 32 bits once t_j < 2^32 (j >= j32), and rho is assembled
// by Horner's rule from the top digit.
template <bool INT_FLOOR, int ND>
__device__ __forceinline__ double redq_pq_word_nd(double x, const RedqPqParams &P) {
    uint64_t t = f64_to_u64_exact(x);
    double tx = x;
    uint32_t u[ND];
#pragma unroll
    for (int j = 0; j < ND - 1; ++j) {
        if (INT_FLOOR && j >= (int)P.j32) {
            const uint32_t t32 = (uint32_t)t;
            const uint32_t tn = div32(t32, P.div_q32);
            u[j] = mod_p_digit(t32 - (uint32_t)P.q * tn, P);
            t = tn;
        } else {
            uint64_t tn;
            if (INT_FLOOR) {
                tn = div64(t, P.div_q);
            } else {
                tn = f64_to_u64_exact(__dmul_ru(tx, P.inv_q_up));
                tx = u64_to_f64_exact(tn);
            }
            u[j] = mod_p_digit(t - P.q * tn, P);
            t = tn;
        }
    }
    u[ND - 1] = ND == 1 ? mod_p_any(t, P) : mod_p_digit(t, P);
    uint64_t rho = u[ND - 1];
#pragma unroll
    for (int j = ND - 2; j >= 0; --j) rho = rho * (uint32_t)P.q + u[j];   // q < 2^26 when ND >= 2
    return u64_to_f64_exact(rho);
}

// floor(X / m) for an integer-valued float 0 <= X < 2^21 and an integer m
// >= 2: Y = (X + 1/2) / m - 1/2 lies within 1/2 - 1/(2m) of floor(X / m), so
// its nearest integer is the floor; computed as fma(X, RN(1/m), RN(1/(2m) -
// 1/2)), whose error is below (2X/m + 3/4) 2^-24 < 1/(2m) for X < 2^21, and
// rounded to an integer by adding and subtracting 1.5 * 2^23.
__device__ __forceinline__ float floor_div_f32(float X, float inv_m, float c_m) {
    constexpr float kRound = 12582912.0f;
    return __fadd_rn(__fadd_rn(__fmaf_rn(X, inv_m, c_m), kRound), -kRound);
}

// v < 2^23 as a float (placed under the exponent of 2^23), and back.
__device__ __forceinline__ float u32_to_f32_small(uint32_t v) {
    return __fadd_rn(__uint_as_float(0x4B000000u | v), -8388608.0f);
}
__device__ __forceinline__ uint32_t f32_small_to_u32(float f) {
    return __float_as_uint(__fadd_rn(f, 8388608.0f)) & 0x7FFFFFu;
}

// ND digits, q^2 < 2^21: the word is cut into chunks of two base-q digits
// by integer floors by q^2 (64-bit while the dividend may reach 2^32, then
// 32-bit); within a chunk X = hi q + lo (< 2^21, exact in FP32) the floors
// by q and by p are FP32 ones (floor_div_f32), all on the full-rate FP32
// pipe: u = digit mod p, and rho's chunk u_hi q + u_lo < q^2.  The chunks
// of rho are joined by Horner's rule in q^2.
template <int ND>
__device__ __forceinline__ double redq_pq_word_f32(double x, const RedqPqParams &P) {
    constexpr int NC = (ND + 1) / 2;   // the top chunk holds one digit when ND is odd
    uint64_t t = f64_to_u64_exact(x);
    uint32_t c[NC];
#pragma unroll
    for (int i = 0; i < NC - 1; ++i) {
        if (i < (int)P.k64) {
            const uint64_t tn = div64(t, P.div_Q);
            c[i] = (uint32_t)t - P.Q * (uint32_t)tn;
            t = tn;
        } else {
            const uint32_t t32 = (uint32_t)t;
            const uint32_t tn = div32(t32, P.div_Q32);
            c[i] = t32 - P.Q * tn;
            t = tn;
        }
    }
    c[NC - 1] = (uint32_t)t;   // below q^(ND - 2 (NC - 1)) for words below q^ND
    uint64_t rho = 0;
#pragma unroll
    for (int i = NC - 1; i >= 0; --i) {
        const float X = u32_to_f32_small(c[i]);
        float r;
        if (2 * i + 1 < ND) {
            const float hi = floor_div_f32(X, P.inv_q, P.c_q);
            const float lo = __fmaf_rn(-P.fq, hi, X);
            const float uhi = __fmaf_rn(-P.fp, floor_div_f32(hi, P.inv_p, P.c_p), hi);
            const float ulo = __fmaf_rn(-P.fp, floor_div_f32(lo, P.inv_p, P.c_p), lo);
            r = __fmaf_rn(P.fq, uhi, ulo);
        } else {
            r = __fmaf_rn(-P.fp, floor_div_f32(X, P.inv_p, P.c_p), X);
        }
        rho = rho * P.Q + f32_small_to_u32(r);
    }
    return u64_to_f64_exact(rho);
}

// S > 0: each word splits at q^S (redq_pq_word_split); S < 0: digits in
// FP32 (redq_pq_word_f32).
template <bool INT_FLOOR, int ND, int S = 0>
__global__ void __launch_bounds__(kThreads)
redq_pq_kernel(const double *__restrict__ in, double *__restrict__ out, int64_t count,
               const __grid_constant__ RedqPqParams P) {
    const int64_t npairs = count >> 1;
    const double2 *in2 = reinterpret_cast<const double2 *>(in);
    double2 *out2 = reinterpret_cast<double2 *>(out);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto word = [&](double v) {
        if constexpr (S < 0) return redq_pq_word_f32<ND>(v, P);
        else if constexpr (S > 0) return redq_pq_word_split<INT_FLOOR, ND, S>(v, P);
        else if constexpr (ND > 0) return redq_pq_word_nd<INT_FLOOR, ND>(v, P);
        else return redq_pq_word<INT_FLOOR>(v, P);
    };
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < npairs;
         b += kUnroll * stride) {
        double2 w[kUnroll];
#pragma unroll
        for (int s = 0; s < kUnroll; ++s) {
            const int64_t i = b + s * stride;
            w[s] = i < npairs ? __ldcs(in2 + i) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int s = 0; s < kUnroll; ++s) {
            const int64_t i = b + s * stride;
            if (i < npairs) {
                double2 o;
                o.x = word(w[s].x);
                o.y = word(w[s].y);
                __stcs(out2 + i, o);
            }
        }
    }
    if ((count & 1) && blockIdx.x == 0 && threadIdx.x == 0) out[count - 1] = word(in[count - 1]);
}

template <typename Kern, typename Params>
int launch_stream(Kern kern, const double *in, double *out, int64_t count, const Params &P,
                  size_t smem, cudaStream_t stream, const char *what) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return set_error(QADIC_E_CUDA, "%s smem attribute: %s", what,
                         cudaGetErrorString(cudaGetLastError()));
    const int64_t npairs = count >> 1;
    int64_t blocks = resident_blocks(kern, kThreads, smem);
    const int64_t need = (npairs + kThreads - 1) / kThreads;
    if (need < blocks) blocks = need > 0 ? need : 1;
    kern<<<(unsigned)blocks, kThreads, smem, stream>>>(in, out, count, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return QADIC_OK;
}

template <int MODE, bool INT_FLOOR>
int launch_mode(const double *in, double *out, int64_t count, const RedqParams &P, size_t smem,
                cudaStream_t stream) {
    return launch_stream(redq_kernel<MODE, INT_FLOOR>, in, out, count, P, smem, stream, "redq");
}

}  // namespace

// 1/d rounded toward +infinity (d < 2^52): the nearest double, bumped up one
// ulp if it falls below the true 1/d (checked exactly in 128-bit integers).
double inv_up(uint64_t d) {
    double inv = 1.0 / (double)d;
    int e;
    const double mfrac = frexp(inv, &e);            // inv = mfrac * 2^e, mfrac in [0.5, 1)
    const uint64_t M = (uint64_t)ldexp(mfrac, 53);  // inv = M * 2^(e-53)
    // inv >= 1/d  <=>  M * d >= 2^(53-e)
    const unsigned __int128 lhs = (unsigned __int128)M * d;
    const unsigned __int128 rhs = (unsigned __int128)1 << (53 - e);
    if (lhs < rhs) inv = nextafter(inv, 2.0);
    return inv;
}

int launch_redq(uint32_t p, uint32_t log2_q, uint32_t ndigits, const double *in, double *out,
                int64_t count, uint32_t table_mode, bool int_floor, cudaStream_t stream) {
    RedqParams P;
    P.p = p;
    P.s = log2_q;
    P.d = ndigits - 1;
    const uint64_t q = 1ull << log2_q;
    P.qneg = (uint32_t)((p - q % p) % p);
    P.m32 = make_mod_small(p);
    P.divp = make_div64(p);
    P.inv_p_up = inv_up(p);
    size_t smem = 0;
    uint32_t mode = table_mode;
    if (mode == 3) {
        uint64_t entries = 1;
        for (uint32_t j = 0; j < ndigits && entries <= 28000; ++j) entries *= p;
        if (entries * 8 > 220 * 1024) {
            mode = 2;   // full table does not fit: fall back to the largest p^k' table
        } else {
            P.kk = ndigits;
            P.table_entries = (uint32_t)entries;
            smem = entries * 8;
        }
    }
    if (mode == 2) {
        uint32_t kk = 2;
        uint64_t entries = (uint64_t)p * p;
        while (kk < ndigits && entries * p * 8 <= 96 * 1024) {
            entries *= p;
            ++kk;
        }
        if (ndigits < 2) {
            mode = 0;
        } else if (entries * 8 > 96 * 1024) {
            mode = 1;   // not even a p^2 table of packed words fits: byte table
        } else {
            P.kk = kk;
            P.table_entries = (uint32_t)entries;
            smem = entries * 8;
        }
    }
    if (mode == 1 && (uint64_t)p * p > 64) smem = ((uint64_t)p * p + 15) & ~15ull;
    if (int_floor) {
        switch (mode) {
            case 0: return launch_mode<0, true>(in, out, count, P, smem, stream);
            case 1: return launch_mode<1, true>(in, out, count, P, smem, stream);
            case 2: return launch_mode<2, true>(in, out, count, P, smem, stream);
            default: return launch_mode<3, true>(in, out, count, P, smem, stream);
        }
    }
    switch (mode) {
        case 0: return launch_mode<0, false>(in, out, count, P, smem, stream);
        case 1: return launch_mode<1, false>(in, out, count, P, smem, stream);
        case 2: return launch_mode<2, false>(in, out, count, P, smem, stream);
        default: return launch_mode<3, false>(in, out, count, P, smem, stream);
    }
}

int launch_redq_pq(uint32_t p, uint64_t q, uint32_t ndigits, const double *in, double *out,
                   int64_t count, bool int_floor, bool f32_digits, cudaStream_t stream) {
    if (ndigits < 1 || ndigits > (uint32_t)kMaxPqDigits)
        return set_error(QADIC_E_INVALID, "ndigits outside [1, %d]", kMaxPqDigits);
    if (f32_digits && (q > 1448 || ndigits > 8))   // q^2 < 2^21
        return set_error(QADIC_E_UNSUPPORTED,
                         "FP32 digits need q^2 < 2^21 and at most 8 digits (q = %llu, %u digits)",
                         (unsigned long long)q, ndigits);
    RedqPqParams P{};
    P.p = p;
    P.d = ndigits - 1;
    P.m32 = make_mod_small(p);
    P.small_lim = ((uint64_t)1 << 32) / p;
    P.q = q;
    P.inv_q_up = inv_up(q);
    P.div_q = make_div64(q);
    P.div_p = make_div64(p);
    uint64_t qj = 1;
    for (uint32_t j = 0; j < ndigits; ++j) {
        P.qpow[j] = qj;
        qj *= q;
    }
    P.small_q = q <= P.small_lim;
    P.div_q32 = make_div32(q < ((uint64_t)1 << 32) ? (uint32_t)q : 1u);
    // first j with q^(ndigits - j) <= 2^32 (then t_j < 2^32); ndigits if none
    P.j32 = ndigits;
    for (uint32_t j = 0; j < ndigits; ++j) {
        unsigned __int128 bound = 1;
        for (uint32_t i = j; i < ndigits; ++i) bound *= q;
        if (bound <= ((unsigned __int128)1 << 32)) {
            P.j32 = j;
            break;
        }
    }
    if (P.j32 >= 1 && P.j32 < ndigits && P.qpow[P.j32] < ((uint64_t)1 << 32)) {
        P.split = 1;
        P.qs = (uint32_t)P.qpow[P.j32];
        P.div_qs = make_div64(P.qpow[P.j32]);
        // round-up reciprocal with 2^s < q^S <= 2^(s+1): its error e < q^S
        // times r < 2^52 stays below 2^(64+s), so the floor is exact
        {
            const uint64_t d = P.qpow[P.j32];
            uint32_t sh = 0;
            while (((uint64_t)2 << sh) < d) ++sh;   // 2^sh < d <= 2^(sh+1)
            const unsigned __int128 two = (unsigned __int128)1 << (64 + sh);
            P.qs_m = (uint64_t)((two + d - 1) / d);
            P.qs_s = sh;
        }
        P.inv_qs_up = inv_up(P.qpow[P.j32]);
    }
    if (f32_digits) {
        P.Q = (uint32_t)(q * q);
        P.div_Q = make_div64(P.Q);
        P.div_Q32 = make_div32(P.Q);
        // the dividend of floor i is below q^(ndigits - 2i)
        P.k64 = 0;
        for (uint32_t i = 0; 2 * i + 2 <= ndigits; ++i) {
            unsigned __int128 bound = 1;
            for (uint32_t j = 2 * i; j < ndigits; ++j) bound *= q;
            if (bound > ((unsigned __int128)1 << 32)) P.k64 = i + 1;
        }
        P.fq = (float)q;
        P.inv_q = 1.0f / (float)q;
        P.c_q = (float)(0.5 / (double)q - 0.5);
        P.fp = (float)p;
        P.inv_p = 1.0f / (float)p;
        P.c_p = (float)(0.5 / (double)p - 0.5);
        switch (ndigits) {
#define QADIC_PQ_F32(N) \
    case N: return launch_stream(redq_pq_kernel<true, N, -1>, in, out, count, P, 0, stream, "redq_pq");
            QADIC_PQ_F32(1) QADIC_PQ_F32(2) QADIC_PQ_F32(3) QADIC_PQ_F32(4)
            QADIC_PQ_F32(5) QADIC_PQ_F32(6) QADIC_PQ_F32(7) QADIC_PQ_F32(8)
#undef QADIC_PQ_F32
            default: break;
        }
    }
    if (P.split) {
        switch ((int_floor ? 256 : 0) + ndigits * 16 + P.j32) {
#define QADIC_PQ_SPLIT(N, S)                                                                    \
    case 256 + N * 16 + S:                                                                      \
        return launch_stream(redq_pq_kernel<true, N, S>, in, out, count, P, 0, stream, "redq_pq"); \
    case N * 16 + S:                                                                            \
        return launch_stream(redq_pq_kernel<false, N, S>, in, out, count, P, 0, stream, "redq_pq");
            QADIC_PQ_SPLIT(2, 1)
            QADIC_PQ_SPLIT(3, 1) QADIC_PQ_SPLIT(3, 2)
            QADIC_PQ_SPLIT(4, 1) QADIC_PQ_SPLIT(4, 2) QADIC_PQ_SPLIT(4, 3)
            QADIC_PQ_SPLIT(5, 1) QADIC_PQ_SPLIT(5, 2) QADIC_PQ_SPLIT(5, 3) QADIC_PQ_SPLIT(5, 4)
            QADIC_PQ_SPLIT(6, 1) QADIC_PQ_SPLIT(6, 2) QADIC_PQ_SPLIT(6, 3) QADIC_PQ_SPLIT(6, 4)
            QADIC_PQ_SPLIT(6, 5)
            QADIC_PQ_SPLIT(7, 1) QADIC_PQ_SPLIT(7, 2) QADIC_PQ_SPLIT(7, 3) QADIC_PQ_SPLIT(7, 4)
            QADIC_PQ_SPLIT(7, 5) QADIC_PQ_SPLIT(7, 6)
            QADIC_PQ_SPLIT(8, 1) QADIC_PQ_SPLIT(8, 2) QADIC_PQ_SPLIT(8, 3) QADIC_PQ_SPLIT(8, 4)
            QADIC_PQ_SPLIT(8, 5) QADIC_PQ_SPLIT(8, 6) QADIC_PQ_SPLIT(8, 7)
#undef QADIC_PQ_SPLIT
            default: break;   // more digits: the chain below
        }
    }
    switch (int_floor ? ndigits : ndigits + 100) {
#define QADIC_PQ_CASE(N)                                                                            \
    case N: return launch_stream(redq_pq_kernel<true, N>, in, out, count, P, 0, stream, "redq_pq"); \
    case N + 100: return launch_stream(redq_pq_kernel<false, N>, in, out, count, P, 0, stream, "redq_pq");
        QADIC_PQ_CASE(1) QADIC_PQ_CASE(2) QADIC_PQ_CASE(3) QADIC_PQ_CASE(4)
        QADIC_PQ_CASE(5) QADIC_PQ_CASE(6) QADIC_PQ_CASE(7) QADIC_PQ_CASE(8)
#undef QADIC_PQ_CASE
        default: break;
    }
    if (int_floor) return launch_stream(redq_pq_kernel<true, 0>, in, out, count, P, 0, stream, "redq_pq");
    return launch_stream(redq_pq_kernel<false, 0>, in, out, count, P, 0, stream, "redq_pq");
}

}  // namespace qadic
