// DQT pack (Sec. 2 and Sec. 7, improvement 1: "replace the Horner
// evaluation by a single table lookup"; Alg. 4's pack step).
//
// Inputs: discrete-log codes (uint8/uint16), uint8 coefficient planes in
// [0, p-1], or int8 coefficient planes (any representative).  Outputs:
//   QADIC_F64    sum_i c_i q^i as a double (table lookup for logs, shifts for
//                planes since q = 2^s, Sec. 2)
//   OPERAND_A    k planes of bf16 centred coefficients, same layout
//   OPERAND_B    k planes of bf16 centred coefficients, transposed (K-major B)
//   COEFF_U8     k planes of uint8 coefficients (log input only)
//   OPERAND_B_FOLD  B's multiplication matrices for the fold-before form:
//                plane i, block j = coefficient j of B X^i mod P, transposed
//   OPERAND_A_KARA / OPERAND_B_KARA  (k = 2) three bf16 planes c_0, c_1 and
//                (c_0 + c_1) mod p, centred; B transposed (Karatsuba form)
// The log -> value tables live in shared memory when they fit (96 KB).
// HBM-bound elementwise work; the transposing variant stages 32 x 32 tiles
// in shared memory so both the reads and the writes are coalesced.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qadic {

namespace {

enum InKind { IN_LOG8 = 0, IN_LOG16 = 1, IN_U8 = 2, IN_I8 = 3 };
enum OutKind { OUT_F64 = 0, OUT_OPA = 1, OUT_OPB = 2, OUT_COEFF = 3, OUT_OPA8 = 4 };

// e4m3 code of a centred coefficient (|c| <= 15 for p <= 31: exact).
__device__ __forceinline__ uint8_t e4m3_of(int c) {
    return (uint8_t)__nv_cvt_float_to_fp8((float)c, __NV_SATFINITE, __NV_E4M3);
}

// Two bf16 small integers (low element first) -> their two e4m3 codes.
__device__ __forceinline__ uint32_t e4m3x2_of_bf16x2(uint32_t w) {
    const float2 f = make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    return (uint32_t)__nv_cvt_float2_to_fp8x2(f, __NV_SATFINITE, __NV_E4M3);
}

constexpr int kTile = 32;
constexpr int kSmemTableBytes = 96 * 1024;

struct PackParams {
    int64_t rows, cols, ld_in, ld_out;
    uint32_t p, k, s, order, h;
    uint32_t m32;                 // ceil(2^32/p)
    float inv_p;                  // 1/p rounded to FP32
    const double *log_f64;        // global tables
    const int8_t *log_centred;
    const uint8_t *antilog;
    int tables_in_smem;
    int64_t n_pad;                       // OPERAND_B_FOLD: rows per block
    uint8_t xpow[2 * kMaxK - 1][kMaxK];  // X^t mod P, t < 2k - 1
};

// Coefficient i of the input element (row r, col c), reduced to [0, p-1].
template <int IN>
__device__ __forceinline__ uint32_t coeff_canon(const void *in, const PackParams &P, int64_t r,
                                                int64_t c, uint32_t i) {
    if (IN == IN_U8) {
        return mod_small(__ldg((const uint8_t *)in + ((int64_t)i * P.rows + r) * P.ld_in + c), P.p,
                         P.m32);
    } else {
        const int32_t v = __ldg((const int8_t *)in + ((int64_t)i * P.rows + r) * P.ld_in + c);
        const uint32_t shifted = (uint32_t)(v + 128 * (int32_t)P.p);   // >= 0, < 2^16
        return mod_small(shifted, P.p, P.m32);
    }
}

__device__ __forceinline__ int32_t centre(uint32_t c, const PackParams &P) {
    return (P.p > 2 && c > P.h) ? (int32_t)c - (int32_t)P.p : (int32_t)c;
}

template <int IN>
__device__ __forceinline__ uint32_t load_code(const void *in, const PackParams &P, int64_t r,
                                              int64_t c) {
    if (IN == IN_LOG8) return __ldg((const uint8_t *)in + r * P.ld_in + c);
    return __ldg((const uint16_t *)in + r * P.ld_in + c);
}

// Elementwise outputs (F64, OPA, COEFF): one thread per element, 2-D grid.
template <int IN, int OUT>
__global__ void __launch_bounds__(256) pack_elementwise(const void *__restrict__ in,
                                                        void *__restrict__ out, PackParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    const double *tf64 = P.log_f64;
    const int8_t *tcen = P.log_centred;
    if ((IN == IN_LOG8 || IN == IN_LOG16) && P.tables_in_smem) {
        if (OUT == OUT_F64) {
            double *t = (double *)smem;
            for (uint32_t i = threadIdx.x; i < P.order; i += blockDim.x) t[i] = P.log_f64[i];
            tf64 = t;
        } else if (OUT == OUT_OPA) {
            int8_t *t = (int8_t *)smem;
            for (uint32_t i = threadIdx.x; i < P.order * P.k; i += blockDim.x)
                t[i] = P.log_centred[i];
            tcen = t;
        }
        __syncthreads();
    }
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
    if (c >= P.cols || r >= P.rows) return;
    if (IN == IN_LOG8 || IN == IN_LOG16) {
        uint32_t code = load_code<IN>(in, P, r, c);
        if (code >= P.order) code = P.order - 1;   // out-of-range codes read as zero
        if (OUT == OUT_F64) {
            ((double *)out)[r * P.ld_out + c] = tf64[code];
        } else if (OUT == OUT_OPA) {
            for (uint32_t i = 0; i < P.k; ++i)
                ((__nv_bfloat16 *)out)[((int64_t)i * P.rows + r) * P.ld_out + c] =
                    __int2bfloat16_rn(tcen[code * P.k + i]);
        } else if (OUT == OUT_OPA8) {
            for (uint32_t i = 0; i < P.k; ++i)
                ((uint8_t *)out)[((int64_t)i * P.rows + r) * P.ld_out + c] = e4m3_of(tcen[code * P.k + i]);
        } else {
            for (uint32_t i = 0; i < P.k; ++i)
                ((uint8_t *)out)[((int64_t)i * P.rows + r) * P.ld_out + c] =
                    __ldg(P.antilog + code * P.k + i);
        }
    } else {
        if (OUT == OUT_F64) {
            uint64_t w = 0;
            for (uint32_t i = 0; i < P.k; ++i) w |= (uint64_t)coeff_canon<IN>(in, P, r, c, i) << (P.s * i);
            ((double *)out)[r * P.ld_out + c] = (double)w;   // exact: w < 2^53
        } else if (OUT == OUT_OPA8) {
            for (uint32_t i = 0; i < P.k; ++i)
                ((uint8_t *)out)[((int64_t)i * P.rows + r) * P.ld_out + c] =
                    e4m3_of(centre(coeff_canon<IN>(in, P, r, c, i), P));
        } else {
            for (uint32_t i = 0; i < P.k; ++i)
                ((__nv_bfloat16 *)out)[((int64_t)i * P.rows + r) * P.ld_out + c] =
                    __int2bfloat16_rn(centre(coeff_canon<IN>(in, P, r, c, i), P));
        }
    }
}

// Transposed operand (OPERAND_B, or with OUT8 OPERAND_B_E4M3): out plane i
// is cols x rows.
template <int IN, bool OUT8 = false>
__global__ void __launch_bounds__(kTile * 8) pack_transpose(const void *__restrict__ in,
                                                           void *__restrict__ out_v,
                                                           PackParams P) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int16_t tile[kMaxK][kTile][kTile + 1];
    const int8_t *tcen = P.log_centred;
    if ((IN == IN_LOG8 || IN == IN_LOG16) && P.tables_in_smem) {
        int8_t *t = (int8_t *)smem;
        for (uint32_t i = threadIdx.x; i < P.order * P.k; i += blockDim.x) t[i] = P.log_centred[i];
        tcen = t;
        __syncthreads();
    }
    const int64_t r0 = (int64_t)blockIdx.y * kTile, c0 = (int64_t)blockIdx.x * kTile;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;   // 32 x 8
    for (int yy = ty; yy < kTile; yy += 8) {
        const int64_t r = r0 + yy, c = c0 + tx;
        if (r < P.rows && c < P.cols) {
            if (IN == IN_LOG8 || IN == IN_LOG16) {
                uint32_t code = load_code<IN>(in, P, r, c);
                if (code >= P.order) code = P.order - 1;
                for (uint32_t i = 0; i < P.k; ++i) tile[i][yy][tx] = tcen[code * P.k + i];
            } else {
                for (uint32_t i = 0; i < P.k; ++i)
                    tile[i][yy][tx] = (int16_t)centre(coeff_canon<IN>(in, P, r, c, i), P);
            }
        }
    }
    __syncthreads();
    for (int yy = ty; yy < kTile; yy += 8) {
        const int64_t oc = c0 + yy, orow = r0 + tx;   // output row = input col
        if (oc < P.cols && orow < P.rows)
            for (uint32_t i = 0; i < P.k; ++i) {
                const int64_t o = ((int64_t)i * P.cols + oc) * P.ld_out + orow;
                if constexpr (OUT8) static_cast<uint8_t *>(out_v)[o] = e4m3_of(tile[i][tx][yy]);
                else static_cast<__nv_bfloat16 *>(out_v)[o] = __int2bfloat16_rn(tile[i][tx][yy]);
            }
    }
}

// Fold-before operand: for each element b of B (K x n) and each i, j < k,
// coefficient j of b X^i mod P = sum_l b_l (X^(l+i) mod P)_j, centred, at
// row (i k + j) n_pad + c, column r of the output (K contiguous).  The
// 32 x 32 input tile is staged as canonical coefficients so both the reads
// and the writes are coalesced; columns c in [n, n_pad) are written as 0.
template <int IN>
__global__ void __launch_bounds__(kTile * 8) pack_fold_b(const void *__restrict__ in,
                                                        __nv_bfloat16 *__restrict__ out,
                                                        PackParams P) {
    __shared__ uint8_t tile[kMaxK][kTile][kTile + 1];
    const int64_t r0 = (int64_t)blockIdx.y * kTile, c0 = (int64_t)blockIdx.x * kTile;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;   // 32 x 8
    for (int yy = ty; yy < kTile; yy += 8) {
        const int64_t r = r0 + yy, c = c0 + tx;
        const bool valid = r < P.rows && c < P.cols;
        if (IN == IN_LOG8 || IN == IN_LOG16) {
            uint32_t code = valid ? load_code<IN>(in, P, r, c) : 0;
            if (code >= P.order) code = P.order - 1;
            for (uint32_t i = 0; i < P.k; ++i)
                tile[i][yy][tx] = valid ? __ldg(P.antilog + (int64_t)code * P.k + i) : 0;
        } else {
            for (uint32_t i = 0; i < P.k; ++i)
                tile[i][yy][tx] = valid ? (uint8_t)coeff_canon<IN>(in, P, r, c, i) : 0;
        }
    }
    __syncthreads();
    for (int yy = ty; yy < kTile; yy += 8) {
        const int64_t oc = c0 + yy, orow = r0 + tx;   // output row block index = input col
        if (oc >= P.n_pad || orow >= P.rows) continue;
        uint32_t b[kMaxK];
        for (uint32_t l = 0; l < P.k; ++l) b[l] = tile[l][tx][yy];
        for (uint32_t i = 0; i < P.k; ++i)
            for (uint32_t j = 0; j < P.k; ++j) {
                uint32_t v = 0;
                for (uint32_t l = 0; l < P.k; ++l)
                    v += mod_small(b[l] * P.xpow[l + i][j], P.p, P.m32);   // each term < p
                v = mod_small(v, P.p, P.m32);
                out[(((int64_t)i * P.k + j) * P.n_pad + oc) * P.ld_out + orow] =
                    __int2bfloat16_rn(centre(v, P));
            }
    }
}

// Karatsuba operands (k = 2): planes c_0, c_1, (c_0 + c_1) mod p, centred;
// TRANS writes plane v as cols x rows (B), else rows x cols (A).  32 x 32
// tiles staged in shared memory keep the transposed writes coalesced.
template <int IN, bool TRANS>
__global__ void __launch_bounds__(kTile * 8) pack_kara(const void *__restrict__ in,
                                                      __nv_bfloat16 *__restrict__ out,
                                                      PackParams P) {
    __shared__ uint8_t tile[2][kTile][kTile + 1];
    const int64_t r0 = (int64_t)blockIdx.y * kTile, c0 = (int64_t)blockIdx.x * kTile;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    for (int yy = ty; yy < kTile; yy += 8) {
        const int64_t r = r0 + yy, c = c0 + tx;
        if (r < P.rows && c < P.cols) {
            if (IN == IN_LOG8 || IN == IN_LOG16) {
                uint32_t code = load_code<IN>(in, P, r, c);
                if (code >= P.order) code = P.order - 1;
                tile[0][yy][tx] = __ldg(P.antilog + (int64_t)code * 2);
                tile[1][yy][tx] = __ldg(P.antilog + (int64_t)code * 2 + 1);
            } else {
                tile[0][yy][tx] = (uint8_t)coeff_canon<IN>(in, P, r, c, 0);
                tile[1][yy][tx] = (uint8_t)coeff_canon<IN>(in, P, r, c, 1);
            }
        }
    }
    __syncthreads();
    for (int yy = ty; yy < kTile; yy += 8) {
        // A: element (r0 + yy, c0 + tx); B: output row c0 + yy, column r0 + tx
        const int64_t r = TRANS ? r0 + tx : r0 + yy, c = TRANS ? c0 + yy : c0 + tx;
        if (r >= P.rows || c >= P.cols) continue;
        const uint32_t a0 = TRANS ? tile[0][tx][yy] : tile[0][yy][tx];
        const uint32_t a1 = TRANS ? tile[1][tx][yy] : tile[1][yy][tx];
        const uint32_t v[3] = {a0, a1, mod_small(a0 + a1, P.p, P.m32)};
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            const int64_t o = TRANS ? ((int64_t)pl * P.cols + c) * P.ld_out + r
                                    : ((int64_t)pl * P.rows + r) * P.ld_out + c;
            out[o] = __int2bfloat16_rn(centre(v[pl], P));
        }
    }
}

// Fast paths for coefficient planes (int8 / uint8) -> bf16 operands when
// every row starts on a 16-byte boundary and cols % 16 == 0: each thread
// turns 16 coefficients (one 16-byte load) into 16 bf16 (two 16-byte
// stores).
template <int IN>
__device__ __forceinline__ uint32_t centre_pair(uint32_t b0, uint32_t b1, const PackParams &P) {
    const int32_t v0 = (IN == IN_I8) ? (int32_t)(int8_t)b0 : (int32_t)b0;
    const int32_t v1 = (IN == IN_I8) ? (int32_t)(int8_t)b1 : (int32_t)b1;
    const uint32_t c0 = mod_small((uint32_t)(v0 + 128 * (int32_t)P.p), P.p, P.m32);
    const uint32_t c1 = mod_small((uint32_t)(v1 + 128 * (int32_t)P.p), P.p, P.m32);
    const __nv_bfloat16 h0 = __int2bfloat16_rn(centre(c0, P));
    const __nv_bfloat16 h1 = __int2bfloat16_rn(centre(c1, P));
    return (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
}

// Odd p, in FP32 on the full-rate pipes (no integer-to-float or bf16
// conversion instructions): a byte b placed under the exponent of 2^23 gives
// the float 2^23 + b, so one subtraction yields the coefficient v exactly
// (int8 input: b ^ 0x80 = v + 128).  r = the integer nearest v/p, by adding
// and subtracting 1.5 * 2^23 after the multiply; v/p is never within 1/(2p)
// of a half-integer for odd p, far more than the FP32 error of v * (1/p)
// for |v| <= 255, so r is exact and c = v - p r is the centred residue in
// [-(p-1)/2, (p-1)/2] (the same value, with the same +0 for zero, as
// reducing into [0, p) and centring).  |c| < 2^8 needs at most 8 significant
// bits, so its bf16 is the upper half of its FP32 bits.
template <int IN>
__device__ __forceinline__ uint32_t centre_pair_odd(uint32_t w, uint32_t sel0, uint32_t sel1,
                                                    const PackParams &P) {
    constexpr float kBias = IN == IN_I8 ? 8388608.0f + 128.0f : 8388608.0f;
    constexpr float kRound = 12582912.0f;   // 1.5 * 2^23
    const float pf = (float)P.p;
    const float v0 = __uint_as_float(__byte_perm(w, 0x4B000000u, sel0)) - kBias;
    const float v1 = __uint_as_float(__byte_perm(w, 0x4B000000u, sel1)) - kBias;
    const float r0 = __fmaf_rn(v0, P.inv_p, kRound) - kRound;
    const float r1 = __fmaf_rn(v1, P.inv_p, kRound) - kRound;
    const float c0 = __fmaf_rn(-pf, r0, v0);
    const float c1 = __fmaf_rn(-pf, r1, v1);
    return __byte_perm(__float_as_uint(c0), __float_as_uint(c1), 0x7632);
}

template <int IN>
__device__ __forceinline__ void convert16(uint4 w, const PackParams &P, uint32_t (&o)[8]) {
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    if (P.p & 1) {
        // byte j of the word to byte 0 under 0x4B (bytes 4-7 of the pair)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t x = IN == IN_I8 ? words[q] ^ 0x80808080u : words[q];
            o[2 * q] = centre_pair_odd<IN>(x, 0x7440, 0x7441, P);
            o[2 * q + 1] = centre_pair_odd<IN>(x, 0x7442, 0x7443, P);
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        o[2 * q] = centre_pair<IN>(words[q] & 0xff, (words[q] >> 8) & 0xff, P);
        o[2 * q + 1] = centre_pair<IN>((words[q] >> 16) & 0xff, words[q] >> 24, P);
    }
}

// Same layout: unit u = 16 consecutive coefficients of one row of one plane.
// Four independent 16-byte loads in flight per thread; the unit -> (row,
// chunk) split uses 32-bit division whenever the unit count allows.
template <int IN>
__device__ __forceinline__ void vec_a_body(const uint8_t *__restrict__ in,
                                           __nv_bfloat16 *__restrict__ out, const PackParams &P,
                                           int64_t block, int64_t nblocks) {
    constexpr int U = 4;
    const int64_t per_row = P.cols / 16;
    const int64_t units = (int64_t)P.k * P.rows * per_row;
    const int64_t stride = nblocks * blockDim.x;
    const bool small = units < (1ll << 31) && per_row < (1ll << 31);
    const uint32_t pr32 = (uint32_t)per_row;
    auto split = [&](int64_t u, int64_t &pr, int64_t &c16) {
        if (small) {
            const uint32_t uu = (uint32_t)u, q = uu / pr32;
            pr = q;
            c16 = uu - q * pr32;
        } else {
            pr = u / per_row;
            c16 = u - pr * per_row;
        }
    };
    for (int64_t u0 = block * blockDim.x + threadIdx.x; u0 < units; u0 += U * stride) {
        uint4 w[U];
#pragma unroll
        for (int s = 0; s < U; ++s) {
            const int64_t u = u0 + s * stride;
            if (u < units) {
                int64_t pr, c16;   // pr = plane * rows + row
                split(u, pr, c16);
                w[s] = __ldcs(reinterpret_cast<const uint4 *>(in + pr * P.ld_in + c16 * 16));
            }
        }
#pragma unroll
        for (int s = 0; s < U; ++s) {
            const int64_t u = u0 + s * stride;
            if (u >= units) break;
            int64_t pr, c16;
            split(u, pr, c16);
            uint32_t o[8];
            convert16<IN>(w[s], P, o);
            uint4 *dst = reinterpret_cast<uint4 *>(out + pr * P.ld_out + c16 * 16);
            __stcs(dst, make_uint4(o[0], o[1], o[2], o[3]));
            __stcs(dst + 1, make_uint4(o[4], o[5], o[6], o[7]));
        }
    }
}

template <int IN>
__global__ void __launch_bounds__(256) pack_vec_a(const uint8_t *__restrict__ in,
                                                  __nv_bfloat16 *__restrict__ out, PackParams P) {
    vec_a_body<IN>(in, out, P, blockIdx.x, gridDim.x);
}

// Transposed operand: RT stacked 64 x 64 input tiles per block (input rows
// RT by .. RT by + 64 RT - 1), every plane of them; the 16-byte loads of a
// thread for two planes of all RT tiles are issued together, then each tile
// and plane goes through the shared-memory transpose and leaves as 16-byte
// stores along the output rows.
template <int IN, int RT, bool OUT8 = false>
__device__ __forceinline__ void vec_b_body(const uint8_t *__restrict__ in, void *__restrict__ out_v,
                                           const PackParams &P, int64_t bx, int64_t by,
                                           uint16_t (*tile)[64 + 2]) {
    __nv_bfloat16 *out = static_cast<__nv_bfloat16 *>(out_v);
    uint8_t *out8 = static_cast<uint8_t *>(out_v);
    const int64_t c0 = bx * 64;
    const int rr = threadIdx.x / 4, cc = (threadIdx.x % 4) * 16;
    // planes in groups of two: the loads of a group are in flight together
#pragma unroll 1
    for (int g = 0; g < (int)P.k; g += 2) {
        uint4 w[RT][2];
#pragma unroll
        for (int t = 0; t < RT; ++t)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int64_t r = (by * RT + t) * 64 + rr;
                w[t][e] = make_uint4(0, 0, 0, 0);
                if (g + e < (int)P.k && r < P.rows)
                    w[t][e] = __ldcs(reinterpret_cast<const uint4 *>(
                        in + ((int64_t)(g + e) * P.rows + r) * P.ld_in + c0 + cc));
            }
#pragma unroll
        for (int t = 0; t < RT; ++t) {
            const int64_t r0 = (by * RT + t) * 64;
            if (r0 >= P.rows) break;   // block-uniform
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int plane = g + e;
                if (plane >= (int)P.k) break;   // block-uniform
                uint32_t o[8];
                convert16<IN>(w[t][e], P, o);
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    tile[rr][cc + 2 * x] = (uint16_t)o[x];
                    tile[rr][cc + 2 * x + 1] = (uint16_t)(o[x] >> 16);
                }
                __syncthreads();
                // output row (input column) oc, 8 consecutive input rows per chunk
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int idx = threadIdx.x + 256 * s;        // 64 output rows x 8 chunks
                    const int oc = idx / 8, ch = (idx % 8) * 8;
                    uint32_t v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v[q] = (uint32_t)tile[ch + 2 * q][oc] | ((uint32_t)tile[ch + 2 * q + 1][oc] << 16);
                    const int64_t orow = c0 + oc, ocol = r0 + ch;
                    if (OUT8) {
                        // e4m3 codes: 8 bytes per chunk (8-byte aligned: ld_out % 16 == 0)
                        uint8_t *dst = out8 + ((int64_t)plane * P.cols + orow) * P.ld_out + ocol;
                        const uint32_t lo = e4m3x2_of_bf16x2(v[0]) | (e4m3x2_of_bf16x2(v[1]) << 16);
                        const uint32_t hi = e4m3x2_of_bf16x2(v[2]) | (e4m3x2_of_bf16x2(v[3]) << 16);
                        if (ocol + 8 <= P.rows) {
                            *reinterpret_cast<uint2 *>(dst) = make_uint2(lo, hi);
                        } else {
                            for (int x = 0; x < 8 && ocol + x < P.rows; ++x)
                                dst[x] = (uint8_t)((x < 4 ? lo : hi) >> (8 * (x % 4)));
                        }
                    } else if (ocol + 8 <= P.rows) {
                        *reinterpret_cast<uint4 *>(out + ((int64_t)plane * P.cols + orow) * P.ld_out +
                                                   ocol) = make_uint4(v[0], v[1], v[2], v[3]);
                    } else {
                        for (int x = 0; x < 8 && ocol + x < P.rows; ++x)
                            out[((int64_t)plane * P.cols + orow) * P.ld_out + ocol + x] =
                                __ushort_as_bfloat16((uint16_t)(v[x / 2] >> (16 * (x % 2))));
                    }
                }
                __syncthreads();   // the tile is rewritten next
            }
        }
    }
}

template <int IN>
__global__ void __launch_bounds__(256) pack_vec_b(const uint8_t *__restrict__ in,
                                                  __nv_bfloat16 *__restrict__ out, PackParams P) {
    __shared__ uint16_t tile[64][64 + 2];
    vec_b_body<IN, 1>(in, out, P, blockIdx.x, blockIdx.y, tile);
}

// OPERAND_B_E4M3 from aligned planes: the same 64 x 64 transpose.
template <int IN>
__global__ void __launch_bounds__(256) pack_vec_b8(const uint8_t *__restrict__ in,
                                                   uint8_t *__restrict__ out, PackParams P) {
    __shared__ uint16_t tile[64][64 + 2];
    ptx::griddep_wait();   // launched to overlap the previous kernel's tail
    vec_b_body<IN, 1, true>(in, out, P, blockIdx.x, blockIdx.y, tile);
}

// OPERAND_A_E4M3 from aligned planes: 16 coefficients per thread, one
// 16-byte load and one 16-byte store of their codes; blocks `block` of
// `nblocks` stride over the units.
template <int IN>
__device__ __forceinline__ void vec_a8_body(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                            const PackParams &P, int64_t block, int64_t nblocks) {
    const int64_t per_row = P.cols / 16;
    const int64_t units = (int64_t)P.k * P.rows * per_row;
    for (int64_t u = block * blockDim.x + threadIdx.x; u < units; u += nblocks * blockDim.x) {
        const int64_t pr = u / per_row, c16 = u - pr * per_row;   // pr = plane * rows + row
        const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(in + pr * P.ld_in + c16 * 16));
        uint32_t o[8];
        convert16<IN>(w, P, o);
        uint4 r;
        r.x = e4m3x2_of_bf16x2(o[0]) | (e4m3x2_of_bf16x2(o[1]) << 16);
        r.y = e4m3x2_of_bf16x2(o[2]) | (e4m3x2_of_bf16x2(o[3]) << 16);
        r.z = e4m3x2_of_bf16x2(o[4]) | (e4m3x2_of_bf16x2(o[5]) << 16);
        r.w = e4m3x2_of_bf16x2(o[6]) | (e4m3x2_of_bf16x2(o[7]) << 16);
        *reinterpret_cast<uint4 *>(out + pr * P.ld_out + c16 * 16) = r;
    }
}

template <int IN>
__global__ void __launch_bounds__(256) pack_vec_a8(const uint8_t *__restrict__ in,
                                                   uint8_t *__restrict__ out, PackParams P) {
    ptx::griddep_wait();   // launched to overlap the previous kernel's tail
    vec_a8_body<IN>(in, out, P, blockIdx.x, gridDim.x);
}

// Both operands of a plane GEMM in one launch: blocks [0, na) convert A
// (same layout), the others transpose B, two 64 x 64 tiles stacked down K
// per block -- one ramp-up and one tail instead of two for these short
// HBM-bound passes.
template <int IN, bool OUT8>
__global__ void __launch_bounds__(256) pack_vec_ab(const uint8_t *__restrict__ a, void *__restrict__ oa,
                                                   PackParams PA, const uint8_t *__restrict__ b,
                                                   void *__restrict__ ob, PackParams PB, int64_t na) {
    __shared__ uint16_t tile[64][64 + 2];
    ptx::griddep_wait();   // launched to overlap the previous kernel's tail
    if ((int64_t)blockIdx.x < na) {
        if constexpr (OUT8) vec_a8_body<IN>(a, static_cast<uint8_t *>(oa), PA, blockIdx.x, na);
        else vec_a_body<IN>(a, static_cast<__nv_bfloat16 *>(oa), PA, blockIdx.x, na);
    } else {
        const int64_t t = (int64_t)blockIdx.x - na;
        const int64_t nbx = PB.cols / 64;
        vec_b_body<IN, 2, OUT8>(b, ob, PB, t % nbx, t / nbx, tile);
    }
}

// A 256-thread launch with programmatic stream serialization: it may begin
// while the previous kernel of the stream finishes (the kernel waits for it
// before touching memory).
template <class... Args>
cudaError_t launch_pdl(void (*kern)(Args...), dim3 grid, cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = grid;
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int IN>
int dispatch_out(int out_fmt, const void *in, void *out, const PackParams &P0, cudaStream_t stream) {
    PackParams P = P0;
    size_t smem = 0;
    if (IN == IN_LOG8 || IN == IN_LOG16) {
        const size_t need = (out_fmt == QADIC_FMT_QADIC_F64) ? (size_t)P.order * 8
                                                              : (size_t)P.order * P.k;
        P.tables_in_smem = (out_fmt != QADIC_FMT_COEFF_U8) && need <= (size_t)kSmemTableBytes;
        if (P.tables_in_smem) smem = (need + 15) & ~(size_t)15;
    }
    cudaError_t e = cudaSuccess;
    const bool planes_in = (IN == IN_U8 || IN == IN_I8);
    const bool aligned16 = P.cols % 16 == 0 && P.ld_in % 16 == 0 && ((uintptr_t)in & 15) == 0 &&
                           P.ld_out % 8 == 0 && ((uintptr_t)out & 15) == 0;
    if (planes_in && aligned16 && out_fmt == QADIC_FMT_OPERAND_A) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t units = (int64_t)P.k * P.rows * (P.cols / 16);
        int64_t blocks = (units + 255) / 256;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        pack_vec_a<IN><<<(unsigned)blocks, 256, 0, stream>>>((const uint8_t *)in,
                                                             (__nv_bfloat16 *)out, P);
    } else if (planes_in && aligned16 && out_fmt == QADIC_FMT_OPERAND_B && P.cols % 64 == 0 &&
               (P.rows + 63) / 64 <= 65535) {
        const dim3 grid((unsigned)(P.cols / 64), (unsigned)((P.rows + 63) / 64), 1);
        pack_vec_b<IN><<<grid, 256, 0, stream>>>((const uint8_t *)in, (__nv_bfloat16 *)out, P);
    } else if (out_fmt == QADIC_FMT_OPERAND_A_E4M3 || out_fmt == QADIC_FMT_OPERAND_B_E4M3) {
        const bool fast = planes_in && P.cols % 16 == 0 && P.ld_in % 16 == 0 &&
                          ((uintptr_t)in & 15) == 0 && P.ld_out % 16 == 0 && ((uintptr_t)out & 15) == 0;
        if (out_fmt == QADIC_FMT_OPERAND_A_E4M3 && fast) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int64_t units = (int64_t)P.k * P.rows * (P.cols / 16);
            const int64_t blocks = std::min<int64_t>((units + 255) / 256, (int64_t)sms * 8);
            e = launch_pdl(pack_vec_a8<IN>, dim3((unsigned)blocks), stream, (const uint8_t *)in,
                           (uint8_t *)out, P);
        } else if (out_fmt == QADIC_FMT_OPERAND_B_E4M3 && fast && P.cols % 64 == 0 &&
                   (P.rows + 63) / 64 <= 65535) {
            const dim3 grid((unsigned)(P.cols / 64), (unsigned)((P.rows + 63) / 64), 1);
            e = launch_pdl(pack_vec_b8<IN>, grid, stream, (const uint8_t *)in, (uint8_t *)out, P);
        } else if (out_fmt == QADIC_FMT_OPERAND_B_E4M3) {
            auto kern = pack_transpose<IN, true>;
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            const dim3 grid((unsigned)((P.cols + kTile - 1) / kTile), (unsigned)((P.rows + kTile - 1) / kTile));
            if (grid.y > 65535) return set_error(QADIC_E_INVALID, "too many rows for the transpose pack");
            kern<<<grid, kTile * 8, smem, stream>>>(in, out, P);
        } else {
            auto kern = pack_elementwise<IN, OUT_OPA8>;
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            const int64_t gy = std::min<int64_t>(P.rows, 65535);
            const int64_t gz = (P.rows + gy - 1) / gy;
            const dim3 grid((unsigned)((P.cols + 255) / 256), (unsigned)gy, (unsigned)gz);
            kern<<<grid, 256, smem, stream>>>(in, out, P);
        }
    } else if (out_fmt == QADIC_FMT_OPERAND_A_KARA || out_fmt == QADIC_FMT_OPERAND_B_KARA) {
        if (P.k != 2) return set_error(QADIC_E_UNSUPPORTED, "Karatsuba operands are for k = 2");
        const dim3 grid((unsigned)((P.cols + kTile - 1) / kTile), (unsigned)((P.rows + kTile - 1) / kTile));
        if (grid.y > 65535) return set_error(QADIC_E_INVALID, "too many rows for the Karatsuba pack");
        if (out_fmt == QADIC_FMT_OPERAND_A_KARA)
            pack_kara<IN, false><<<grid, kTile * 8, 0, stream>>>(in, (__nv_bfloat16 *)out, P);
        else
            pack_kara<IN, true><<<grid, kTile * 8, 0, stream>>>(in, (__nv_bfloat16 *)out, P);
    } else if (out_fmt == QADIC_FMT_OPERAND_B_FOLD) {
        const dim3 grid((unsigned)(P.n_pad / kTile), (unsigned)((P.rows + kTile - 1) / kTile));
        if (grid.y > 65535) return set_error(QADIC_E_INVALID, "too many rows for the fold pack");
        pack_fold_b<IN><<<grid, kTile * 8, 0, stream>>>(in, (__nv_bfloat16 *)out, P);
    } else if (out_fmt == QADIC_FMT_OPERAND_B) {
        auto kern = pack_transpose<IN>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const dim3 grid((unsigned)((P.cols + kTile - 1) / kTile), (unsigned)((P.rows + kTile - 1) / kTile));
        if (grid.y > 65535) return set_error(QADIC_E_INVALID, "too many rows for the transpose pack");
        kern<<<grid, kTile * 8, smem, stream>>>(in, (__nv_bfloat16 *)out, P);
    } else {
        void (*kern)(const void *, void *, PackParams) = nullptr;
        if (out_fmt == QADIC_FMT_QADIC_F64) kern = pack_elementwise<IN, OUT_F64>;
        else if (out_fmt == QADIC_FMT_OPERAND_A) kern = pack_elementwise<IN, OUT_OPA>;
        else if (out_fmt == QADIC_FMT_COEFF_U8 && (IN == IN_LOG8 || IN == IN_LOG16))
            kern = pack_elementwise<IN, OUT_COEFF>;
        else return set_error(QADIC_E_INVALID, "unsupported pack format pair");
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int64_t gy = std::min<int64_t>(P.rows, 65535);
        const int64_t gz = (P.rows + gy - 1) / gy;
        const dim3 grid((unsigned)((P.cols + 255) / 256), (unsigned)gy, (unsigned)gz);
        kern<<<grid, 256, smem, stream>>>(in, out, P);
    }
    const cudaError_t le = cudaGetLastError();   // clears a launch error either way
    if (e == cudaSuccess) e = le;
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "pack launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace

int launch_pack(const Field &f, int in_fmt, const void *in, int64_t rows, int64_t cols,
                int64_t ld_in, int out_fmt, void *out, int64_t ld_out, cudaStream_t stream) {
    PackParams P;
    P.rows = rows;
    P.cols = cols;
    P.ld_in = ld_in;
    P.ld_out = ld_out;
    P.p = f.p;
    P.k = f.k;
    P.s = f.log2_q;
    P.order = f.order;
    P.h = f.h;
    P.m32 = make_mod_small(f.p);
    P.inv_p = 1.0f / (float)f.p;
    P.log_f64 = f.d_log_f64;
    P.log_centred = f.d_log_centred;
    P.antilog = f.d_antilog;
    P.tables_in_smem = 0;
    P.n_pad = fold_n_pad(cols);
    for (uint32_t t = 0; t < 2 * kMaxK - 1; ++t)
        for (uint32_t j = 0; j < kMaxK; ++j) P.xpow[t][j] = 0;
    for (uint32_t t = 0; t < f.k; ++t) P.xpow[t][t] = 1;
    for (uint32_t t = 0; t + 1 < f.k; ++t)
        for (uint32_t j = 0; j < f.k; ++j) P.xpow[f.k + t][j] = f.fold[t * f.k + j];
    if (out_fmt < QADIC_FMT_COEFF_U8 || out_fmt > QADIC_FMT_OPERAND_B_E4M3 ||
        out_fmt == QADIC_FMT_INT8_PLANES)
        return set_error(QADIC_E_INVALID, "unsupported output format %d", out_fmt);
    if ((out_fmt == QADIC_FMT_OPERAND_A_E4M3 || out_fmt == QADIC_FMT_OPERAND_B_E4M3) && f.p > 31)
        return set_error(QADIC_E_UNSUPPORTED, "e4m3 operands need p <= 31 (|c| <= 15 exact)");
    switch (in_fmt) {
        case QADIC_FMT_LOG:
            return f.order <= 256 ? dispatch_out<IN_LOG8>(out_fmt, in, out, P, stream)
                                  : dispatch_out<IN_LOG16>(out_fmt, in, out, P, stream);
        case QADIC_FMT_COEFF_U8:
            if (out_fmt == QADIC_FMT_COEFF_U8) break;
            return dispatch_out<IN_U8>(out_fmt, in, out, P, stream);
        case QADIC_FMT_INT8_PLANES:
            if (out_fmt == QADIC_FMT_COEFF_U8) break;
            return dispatch_out<IN_I8>(out_fmt, in, out, P, stream);
        default:
            break;
    }
    return set_error(QADIC_E_INVALID, "unsupported pack format pair %d -> %d", in_fmt, out_fmt);
}

namespace {

PackParams pack_params(const Field &f, int64_t rows, int64_t cols, int64_t ld_in, int64_t ld_out) {
    PackParams P{};
    P.rows = rows;
    P.cols = cols;
    P.ld_in = ld_in;
    P.ld_out = ld_out;
    P.p = f.p;
    P.k = f.k;
    P.s = f.log2_q;
    P.order = f.order;
    P.h = f.h;
    P.m32 = make_mod_small(f.p);
    P.inv_p = 1.0f / (float)f.p;
    P.log_f64 = f.d_log_f64;
    P.log_centred = f.d_log_centred;
    P.antilog = f.d_antilog;
    P.tables_in_smem = 0;
    P.n_pad = fold_n_pad(cols);
    return P;
}

}  // namespace

// A (m x K) -> OPERAND_A and B (K x n) -> OPERAND_B from coefficient planes
// (with e4m3: OPERAND_A_E4M3 and OPERAND_B_E4M3), in one launch when both
// fit the vectorised paths, else two.
int launch_pack_pair(const Field &f, int in_fmt, const void *A, int64_t m, int64_t K,
                     int64_t lda_in, void *outA, int64_t lda_out, const void *B, int64_t n,
                     int64_t ldb_in, void *outB, int64_t ldb_out, cudaStream_t stream, bool e4m3) {
    const bool planes_in = in_fmt == QADIC_FMT_INT8_PLANES || in_fmt == QADIC_FMT_COEFF_U8;
    const int64_t lo = e4m3 ? 16 : 8;   // output rows in whole 16-byte units
    const bool a_ok = K % 16 == 0 && lda_in % 16 == 0 && ((uintptr_t)A & 15) == 0 &&
                      lda_out % lo == 0 && ((uintptr_t)outA & 15) == 0;
    const bool b_ok = n % 64 == 0 && ldb_in % 16 == 0 && ((uintptr_t)B & 15) == 0 &&
                      ldb_out % lo == 0 && ((uintptr_t)outB & 15) == 0 && (K + 63) / 64 <= 65535;
    if (!planes_in || !a_ok || !b_ok) {
        int st = launch_pack(f, in_fmt, A, m, K, lda_in,
                             e4m3 ? QADIC_FMT_OPERAND_A_E4M3 : QADIC_FMT_OPERAND_A, outA, lda_out, stream);
        if (st != QADIC_OK) return st;
        return launch_pack(f, in_fmt, B, K, n, ldb_in,
                           e4m3 ? QADIC_FMT_OPERAND_B_E4M3 : QADIC_FMT_OPERAND_B, outB, ldb_out, stream);
    }
    const PackParams PA = pack_params(f, m, K, lda_in, lda_out);
    const PackParams PB = pack_params(f, K, n, ldb_in, ldb_out);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t units_a = (int64_t)f.k * m * (K / 16);
    // A blocks in proportion to A's share of the bytes; B blocks one per tile
    const int64_t nb = (int64_t)(n / 64) * ((K + 127) / 128);
    const int64_t na = std::max<int64_t>(1, std::min<int64_t>((units_a + 1023) / 1024, (int64_t)sms * 8));
    if (na + nb > 0x7fffffff) return set_error(QADIC_E_INVALID, "too many pack blocks");
    // programmatic stream serialization: the launch may begin while the
    // previous kernel of the stream finishes (the kernel waits for it before
    // touching memory)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(na + nb));
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    auto kern = in_fmt == QADIC_FMT_INT8_PLANES
                    ? (e4m3 ? pack_vec_ab<IN_I8, true> : pack_vec_ab<IN_I8, false>)
                    : (e4m3 ? pack_vec_ab<IN_U8, true> : pack_vec_ab<IN_U8, false>);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, (const uint8_t *)A, outA, PA,
                                             (const uint8_t *)B, outB, PB, na);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(QADIC_E_CUDA, "pack launch: %s", cudaGetErrorString(e));
    }
    return QADIC_OK;
}

}  // namespace qadic
