// Shared pieces of the two batched GF(p^k) product kernels (k_batched.cu:
// operand bytes staged through registers; k_batched_async.cu: operands
// converted once, tiles copied with cp.async): the work-list layout, the
// tile shapes, the warp-level MMA step, the exact-chunk reduction and the
// mod p / mod P epilogue.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "common.cuh"

namespace qadic {
namespace bt {

constexpr int kThreads = 128;
constexpr int kMinBK = 32;        // K-block of every configuration 0 (the fallback): a field's
                                  // exact FP32 chunk must cover at least this much
constexpr int kMaxFields = 64;

struct BFieldParams {
    uint32_t p, k, h, m32;
    float pf, inv_pf;
    int32_t chunk_k;               // K elements per exact FP32 chunk (capped)
    int32_t chunk_k16;             // the same for f16 accumulators (GF(2^8) only)
    int32_t f16;                   // GF(2^8): f16 accumulators (see the converted-operand kernel)
    int32_t fp8;                   // p <= 31: operands converted to fp8 e4m3 (|centred| <= 15, exact)
    uint8_t fold[kMaxK * kMaxK];   // X^(k+t) mod P, row t (k coefficients)
    uint8_t fold2[kMaxK];          // p = 2: row t of `fold` as a bit mask (coefficient i at bit i)
};

struct BProd {
    const uint8_t *A;
    const uint8_t *B;
    uint8_t *C;
    const uint16_t *A16;           // converted operands, or null: 16-bit A [k][m][kp] and
    const uint16_t *B16;           // B [k][K][np]; fp8 fields: bytes, A [k][m][kp], B^T [k][n][kp]
    int32_t m, n, K, lda, ldb, ldc;
    int32_t kp, np;                // row lengths: 16-bit K up to 8 and n up to 8; fp8: K up to 16
    int32_t field, cfg;            // field index, tile configuration index
};

struct BTile {
    int32_t prod;
    int16_t tm, tn;
};

struct BHeader {
    uint32_t counter;
    int32_t ntiles;
    int32_t nprod;
    int32_t nfields;
    uint32_t fields_off, prods_off, tiles_off;
    uint32_t order_off;            // conversion items (ConvItem), largest first
    uint32_t nconv;                // number of conversion items
};

// One block of the conversion launch: 8-element chunks [begin, begin +
// kConvItemChunks) of operand `op` (product op / 2, A if op is even, else B).
struct ConvItem {
    uint32_t op, begin;
};
constexpr uint32_t kConvItemChunks = 4096;

constexpr size_t kHeaderBytes = 256;

template <int KP, int BM_, int BN_, int BK_>
struct TileCfg {
    static constexpr int BM = BM_, BN = BN_, BK = BK_;
    static constexpr int WM = BM / 2, WN = BN / 2;   // 2 x 2 warps
    static constexpr int MT = WM / 16, NT = WN / 8;
    static constexpr int NACC = 2 * KP - 1;
    static constexpr int LDA = BK + 8;               // 16-bit elements per A_s row
    static constexpr int LDB = BN + 8;               // 16-bit elements per B_s row
    static constexpr int SMEM = (KP * BM * LDA + KP * BK * LDB) * 2;
    // cp.async stages of the converted-operand kernel: more where a stage is
    // small (little MMA work per K-block to hide a copy behind)
    static constexpr int NSTAGE = SMEM <= 8192 ? 4 : SMEM <= 16384 ? 3 : 2;
    static_assert(MT >= 1 && NT >= 1 && BK % 16 == 0, "tile shape");
};

inline int async_stages(size_t stage_bytes) {
    return stage_bytes <= 8192 ? 4 : stage_bytes <= 16384 ? 3 : 2;
}

// Candidate (BM, BN, BK) per k; index 0 is the default.  Every candidate is
// at least 32 x 16 (the work-list bound); configuration 0 is kMinBK deep.
struct TileShape {
    int bm, bn, bk;
};
constexpr int kMaxCfg = 5;
constexpr TileShape kShapesK2[kMaxCfg] = {{64, 32, 32}, {64, 64, 32}, {32, 32, 32}, {64, 32, 64},
                                          {32, 32, 16}};
constexpr TileShape kShapesK4[kMaxCfg] = {{32, 32, 32}, {64, 32, 32}, {32, 16, 32}, {32, 32, 64},
                                          {32, 16, 16}};
// (k >= 5: the 16-deep K-block halves the staged operand registers, which
// the 15 accumulator sets of k = 8 otherwise push into spills)
constexpr TileShape kShapesK8[kMaxCfg] = {{32, 16, 32}, {32, 32, 32}, {32, 16, 64}, {32, 16, 16},
                                          {32, 16, 16}};

__host__ __device__ constexpr int num_cfgs(uint32_t k) { return k <= 4 ? 5 : 4; }

inline TileShape tile_shape_of(uint32_t k, int cfg) {
    if (cfg < 0 || cfg >= num_cfgs(k)) cfg = 0;
    return k <= 2 ? kShapesK2[cfg] : k <= 4 ? kShapesK4[cfg] : kShapesK8[cfg];
}

// Shared memory of one stage of operand tiles.
inline size_t tile_smem_bytes(uint32_t k, int cfg) {
    const TileShape t = tile_shape_of(k, cfg);
    return (size_t)(k * t.bm * (t.bk + 8) + k * t.bk * (t.bn + 8)) * 2;
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                        uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2_trans(uint32_t addr, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// m16n8k16 with f16 operands and f16 accumulators (two half2 registers).
__device__ __forceinline__ void mma_f16_16816(uint32_t (&d)[2], const uint32_t (&a)[4],
                                              const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f16.f16.f16.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, "
        "{%0,%1};"
        : "+r"(d[0]), "+r"(d[1])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Centred representative of a coefficient byte: c mod p in [-(p-1)/2, (p-1)/2]
// (Eq. 3's centred representation), {0, 1} for p = 2.
__device__ __forceinline__ int centred_int(uint32_t c, const BFieldParams &F) {
    const uint32_t r = mod_small(c, F.p, F.m32);
    return (F.p > 2 && r > F.h) ? (int)r - (int)F.p : (int)r;
}

__device__ __forceinline__ uint16_t bf16_bits(uint32_t c, const BFieldParams &F) {
    return __bfloat16_as_ushort(__int2bfloat16_rn(centred_int(c, F)));
}

// e4m3 holds every integer of magnitude <= 16 exactly, so the centred
// coefficients of any p <= 31 (and the 0/1 of p = 2) convert without loss.
__device__ __forceinline__ uint8_t fp8_bits(uint32_t c, const BFieldParams &F) {
    return (uint8_t)__nv_cvt_float_to_fp8((float)centred_int(c, F), __NV_SATFINITE, __NV_E4M3);
}

inline bool fp8_field(uint32_t p) { return p <= 31; }

// m16n8k32 with fp8 e4m3 operands (four per register), FP32 or f16
// accumulators.  On GB300 the legacy path runs these at about 3.6x the
// bf16 m16n8k16 rate (2177 against 600 TFLOP/s, measured).
__device__ __forceinline__ void mma_e4m3_f32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_e4m3_f16(uint32_t (&d)[2], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f16.e4m3.e4m3.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, "
        "{%0,%1};"
        : "+r"(d[0]), "+r"(d[1])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// fp8 tiles: K-blocks of at least 32 (one m16n8k32 step), rows of BK + 16
// bytes (A [KP][BM], B^T [KP][BN], both K-major) so that ldmatrix rows fall
// in distinct banks.
constexpr int fp8_bk(int bk) { return bk < 32 ? 32 : bk; }

template <int KP, int BM_, int BN_, int BK_>
struct TileCfg8 {
    using W = TileCfg<KP, BM_, BN_, 32>;   // warp layout and accumulators as the 16-bit tiles
    static constexpr int BM = BM_, BN = BN_, BK = fp8_bk(BK_);
    static constexpr int WM = W::WM, WN = W::WN, MT = W::MT, NT = W::NT, NACC = W::NACC;
    static constexpr int LDA = BK + 16, LDB = BK + 16;   // bytes
    static constexpr int SMEM = KP * BM * LDA + KP * BN * LDB;
    static constexpr int NSTAGE = SMEM <= 8192 ? 4 : SMEM <= 16384 ? 3 : 2;
};

inline size_t tile_smem_bytes8(uint32_t k, int cfg) {
    const TileShape t = tile_shape_of(k, cfg);
    const int bk = fp8_bk(t.bk);
    return (size_t)k * t.bm * (bk + 16) + (size_t)k * t.bn * (bk + 16);
}


// Accumulators of one warp: 2k-1 sets of MT x NT m16n8 fragments, FP32 (four
// registers each) or, with F16, f16 pairs (two registers each).
template <typename T, bool F16>
using AccArray = std::conditional_t<F16, uint32_t, float>[T::NACC][T::MT][T::NT][F16 ? 2 : 4];

template <typename T, bool F16>
__device__ __forceinline__ void acc_zero(AccArray<T, F16> &acc) {
#pragma unroll
    for (int t = 0; t < T::NACC; ++t)
#pragma unroll
        for (int a = 0; a < T::MT; ++a)
#pragma unroll
            for (int b = 0; b < T::NT; ++b)
#pragma unroll
                for (int e = 0; e < (F16 ? 2 : 4); ++e) acc[t][a][b][e] = 0;
}

// One 16-deep step of the k^2 plane products: plane i of A times plane j of
// B accumulates into C_{i+j}.  As is [KP][BM][LDA], Bs is [KP][BK][LDB].
template <int KP, typename T, bool F16>
__device__ __forceinline__ void tile_mma_step(AccArray<T, F16> &acc, const uint16_t *As,
                                              const uint16_t *Bs, int ks, int wm, int wn,
                                              int lane) {
    uint32_t bfr[KP][T::NT][2];
#pragma unroll
    for (int j = 0; j < KP; ++j)
#pragma unroll
        for (int nt = 0; nt < T::NT; ++nt) {
            const uint16_t *src = Bs + (j * T::BK + ks * 16 + (lane % 16)) * T::LDB + wn * T::WN + nt * 8;
            ldsm_x2_trans((uint32_t)__cvta_generic_to_shared(src), bfr[j][nt][0], bfr[j][nt][1]);
        }
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        uint32_t afr[T::MT][4];
#pragma unroll
        for (int mt = 0; mt < T::MT; ++mt) {
            const uint16_t *src =
                As + (i * T::BM + wm * T::WM + mt * 16 + (lane % 16)) * T::LDA + ks * 16 + (lane / 16) * 8;
            ldsm_x4((uint32_t)__cvta_generic_to_shared(src), afr[mt][0], afr[mt][1], afr[mt][2],
                    afr[mt][3]);
        }
#pragma unroll
        for (int j = 0; j < KP; ++j)
#pragma unroll
            for (int mt = 0; mt < T::MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < T::NT; ++nt) {
                    if constexpr (F16)
                        mma_f16_16816(acc[i + j][mt][nt], afr[mt], bfr[j][nt]);
                    else
                        mma_bf16_16816(acc[i + j][mt][nt], afr[mt], bfr[j][nt]);
                }
    }
}

// One 32-deep step of the k^2 plane products on fp8 tiles (bytes).
template <int KP, typename T8, bool F16>
__device__ __forceinline__ void tile_mma_step8(AccArray<typename T8::W, F16> &acc, const uint8_t *As,
                                               const uint8_t *Bs, int ks, int wm, int wn, int lane) {
    using T = T8;
    uint32_t bfr[KP][T::NT][2];
#pragma unroll
    for (int j = 0; j < KP; ++j)
#pragma unroll
        for (int nt = 0; nt < T::NT; ++nt) {
            // B^T rows (output columns) n, bytes k: matrix 0 = k 0-15, matrix 1 = k 16-31
            const uint8_t *src = Bs + (j * T::BN + wn * T::WN + nt * 8 + (lane % 8)) * T::LDB + ks * 32 +
                                 ((lane / 8) % 2) * 16;
            asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                         : "=r"(bfr[j][nt][0]), "=r"(bfr[j][nt][1])
                         : "r"((uint32_t)__cvta_generic_to_shared(src)));
        }
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        uint32_t afr[T::MT][4];
#pragma unroll
        for (int mt = 0; mt < T::MT; ++mt) {
            const uint8_t *src =
                As + (i * T::BM + wm * T::WM + mt * 16 + (lane % 16)) * T::LDA + ks * 32 + (lane / 16) * 16;
            ldsm_x4((uint32_t)__cvta_generic_to_shared(src), afr[mt][0], afr[mt][1], afr[mt][2], afr[mt][3]);
        }
#pragma unroll
        for (int j = 0; j < KP; ++j)
#pragma unroll
            for (int mt = 0; mt < T::MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < T::NT; ++nt) {
                    if constexpr (F16)
                        mma_e4m3_f16(acc[i + j][mt][nt], afr[mt], bfr[j][nt]);
                    else
                        mma_e4m3_f32(acc[i + j][mt][nt], afr[mt], bfr[j][nt]);
                }
    }
}

// Exact-chunk boundary: every accumulator x becomes x - p rint(x / p), an
// integer of magnitude <= p / 2 congruent to x.
template <typename T, bool F16>
__device__ __forceinline__ void tile_chunk_reduce(AccArray<T, F16> &acc, const BFieldParams &F) {
#pragma unroll
    for (int t = 0; t < T::NACC; ++t)
#pragma unroll
        for (int a = 0; a < T::MT; ++a)
#pragma unroll
            for (int b = 0; b < T::NT; ++b)
#pragma unroll
                for (int e = 0; e < (F16 ? 2 : 4); ++e) {
                    if constexpr (F16) {
                        float2 x = __half22float2(*reinterpret_cast<__half2 *>(&acc[t][a][b][e]));
                        x.x = fmaf(-F.pf, rintf(x.x * F.inv_pf), x.x);
                        x.y = fmaf(-F.pf, rintf(x.y * F.inv_pf), x.y);
                        const __half2 h = __floats2half2_rn(x.x, x.y);
                        acc[t][a][b][e] = *reinterpret_cast<const uint32_t *>(&h);
                    } else {
                        const float x = acc[t][a][b][e];
                        acc[t][a][b][e] = fmaf(-F.pf, rintf(x * F.inv_pf), x);
                    }
                }
}

// Epilogue: each C_t exactly mod p, then the fold mod P (Alg. 4, fold step,
// in coefficient form: out_i = mu_i + sum_{t >= k} mu_t (X^t mod P)_i), and
// the k output planes written as bytes.
// Value of accumulator element e of fragment (t, mt, nt).
template <typename T, bool F16>
__device__ __forceinline__ float acc_value(const AccArray<T, F16> &acc, int t, int mt, int nt, int e) {
    if constexpr (F16) {
        const __half2 h = *reinterpret_cast<const __half2 *>(&acc[t][mt][nt][e >> 1]);
        return (e & 1) ? __high2float(h) : __low2float(h);
    } else {
        return acc[t][mt][nt][e];
    }
}

template <int KP, typename T, bool F16>
__device__ __forceinline__ void tile_epilogue(const AccArray<T, F16> &acc, const BProd &P,
                                              const BFieldParams &F, int row0, int col0, int wm,
                                              int wn, int lane) {
    if (F.p == 2) {
        // GF(2^k): the 2k-1 plane sums mod 2 as the bits of one word (the low
        // bit of x + 1.5 * 2^23 is the parity of an integer-valued float of
        // magnitude < 2^22), the fold mod P as XORs of the rows X^t mod P, and
        // output plane i as bit i.
        // The two adjacent columns of a fragment row go together: their
        // parities at bits 0.. and 16.. of one word, folded by the same XORs.
        constexpr uint32_t kLow = (1u << KP) - 1u;
#pragma unroll
        for (int mt = 0; mt < T::MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < T::NT; ++nt)
#pragma unroll
                for (int eh = 0; eh < 2; ++eh) {
                    const int row = row0 + wm * T::WM + mt * 16 + (lane / 4) + 8 * eh;
                    const int col = col0 + wn * T::WN + nt * 8 + 2 * (lane % 4);   // and col + 1
                    uint32_t bits = 0;
#pragma unroll
                    for (int t = 0; t < T::NACC; ++t) {
                        const uint32_t b0 = __float_as_uint(acc_value<T, F16>(acc, t, mt, nt, 2 * eh) + 12582912.0f);
                        const uint32_t b1 = __float_as_uint(acc_value<T, F16>(acc, t, mt, nt, 2 * eh + 1) + 12582912.0f);
                        bits |= ((b0 & 1u) | ((b1 & 1u) << 16)) << t;
                    }
                    uint32_t out = bits & (kLow | (kLow << 16));
#pragma unroll
                    for (int t = 0; t < T::NACC - KP; ++t)
                        out ^= ((bits >> (KP + t)) & 0x00010001u) * F.fold2[t];   // row t at both halves
                    if (row < P.m && col < P.n) {
                        const bool pair = col + 1 < P.n;
#pragma unroll
                        for (int i = 0; i < KP; ++i) {
                            uint8_t *dst = P.C + ((int64_t)i * P.m + row) * P.ldc + col;
                            const uint32_t lo = (out >> i) & 1u, hi = (out >> (16 + i)) & 1u;
                            if (pair && (((uintptr_t)dst & 1) == 0)) {
                                *reinterpret_cast<uint16_t *>(dst) = (uint16_t)(lo | (hi << 8));
                            } else {
                                dst[0] = (uint8_t)lo;
                                if (pair) dst[1] = (uint8_t)hi;
                            }
                        }
                    }
                }
        return;
    }
#pragma unroll
    for (int mt = 0; mt < T::MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < T::NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = row0 + wm * T::WM + mt * 16 + (lane / 4) + (e >= 2 ? 8 : 0);
                const int col = col0 + wn * T::WN + nt * 8 + 2 * (lane % 4) + (e & 1);
                uint32_t mu[T::NACC];
#pragma unroll
                for (int t = 0; t < T::NACC; ++t) {
                    float x;
                    if constexpr (F16) {
                        const __half2 h = *reinterpret_cast<const __half2 *>(&acc[t][mt][nt][e >> 1]);
                        x = (e & 1) ? __high2float(h) : __low2float(h);
                    } else {
                        x = acc[t][mt][nt][e];
                    }
                    float r = fmaf(-F.pf, floorf(x * F.inv_pf), x);
                    if (r < 0.f) r += F.pf;
                    if (r >= F.pf) r -= F.pf;
                    mu[t] = (uint32_t)r;
                }
                if (row < P.m && col < P.n) {
                    // the sum stays below (p-1) + (k-1)(p-1)^2 < 2^32 / p: one
                    // mod per output coefficient, exact
#pragma unroll
                    for (int i = 0; i < KP; ++i) {
                        uint32_t o = mu[i];
#pragma unroll
                        for (int t = KP; t < T::NACC; ++t) o += mu[t] * F.fold[(t - KP) * KP + i];
                        P.C[((int64_t)i * P.m + row) * P.ldc + col] = (uint8_t)mod_small(o, F.p, F.m32);
                    }
                }
            }
}

// Launch helpers of the converted-operand kernels (k_batched_async.cu).
int prepare_async_kernel();
int64_t async_grid(size_t smem, int64_t ntiles);
size_t async_smem_bytes(uint32_t k, int cfg, bool fp8);
int launch_convert(const uint8_t *ws, int64_t nitems, cudaStream_t stream);
int launch_async(uint8_t *ws, int64_t grid, size_t smem, cudaStream_t stream);

}  // namespace bt
}  // namespace qadic
