// Shared pieces of the batched GF(p^k) product kernels: the work-list layout
// (both), and for the register-staged kernel (k_batched.cu) the tile
// shapes, the warp-level MMA step, the exact-chunk reduction and the mod p /
// mod P epilogue; the tensor-core path (k_batched_tc.cu) adds its tile
// records and launch helpers.
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
    int32_t fp8;                   // p <= 31: tensor-core operands fp8 e4m3 (|centred| <= 15, exact)
    int32_t tc_chunk_ks;           // tensor-core path: 32-byte K-blocks per exact FP32 chunk
    uint8_t fold[kMaxK * kMaxK];   // X^(k+t) mod P, row t (k coefficients)
    uint8_t fold2[kMaxK];          // p = 2: row t of `fold` as a bit mask (coefficient i at bit i)
};

struct BProd {
    const uint8_t *A;
    const uint8_t *B;
    uint8_t *C;
    const uint16_t *A16;           // tensor-core path: the converted operands in their blocked
    const uint16_t *B16;           // layout (k_batched_tc.cu); null on the register-staged path
    int32_t m, n, K, lda, ldb, ldc;
    int32_t kp, np;                // tensor-core path: 32-byte K-blocks, output columns per tile
    int32_t field, cfg;            // field index, tile configuration index
};

struct BTile {
    int32_t prod;
    int16_t tm, tn;
};

// One tile of the tensor-core path's work list, complete in itself (the
// roles of the product kernel read it with independent loads, one tile
// ahead, instead of a chain tile -> product -> field).
struct TcRec {
    const uint8_t *a;    // the tile's A blocks: K-blocks of k planes x rows8 x 32 bytes
    const uint8_t *b;    // the tile's B blocks: K-blocks of k planes x BN x 32 bytes
    uint8_t *c;          // output byte (row tm*128, column tn*BN) of plane 0
    int64_t c_plane;     // bytes between output planes (m * ldc)
    int32_t ldc;
    int16_t rows, cols;  // valid rows (<= 128) and columns (<= BN) of the tile
    int16_t ks;          // 32-byte K-blocks
    int16_t rows8;       // rows rounded up to 8
    int16_t ndrain;      // in-place reductions on the way through K
    uint8_t field, k;
};
static_assert(sizeof(TcRec) == 48, "TcRec layout");

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
    static_assert(MT >= 1 && NT >= 1 && BK % 16 == 0, "tile shape");
};

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

// Accumulators of one warp: 2k-1 sets of MT x NT m16n8 FP32 fragments.
template <typename T>
using AccArray = float[T::NACC][T::MT][T::NT][4];

template <typename T>
__device__ __forceinline__ void acc_zero(AccArray<T> &acc) {
#pragma unroll
    for (int t = 0; t < T::NACC; ++t)
#pragma unroll
        for (int a = 0; a < T::MT; ++a)
#pragma unroll
            for (int b = 0; b < T::NT; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[t][a][b][e] = 0.f;
}

// One 16-deep step of the k^2 plane products: plane i of A times plane j of
// B accumulates into C_{i+j}.  As is [KP][BM][LDA], Bs is [KP][BK][LDB].
template <int KP, typename T>
__device__ __forceinline__ void tile_mma_step(AccArray<T> &acc, const uint16_t *As,
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
                for (int nt = 0; nt < T::NT; ++nt) mma_bf16_16816(acc[i + j][mt][nt], afr[mt], bfr[j][nt]);
    }
}

// Exact-chunk boundary: every accumulator x becomes x - p rint(x / p), an
// integer of magnitude <= p / 2 congruent to x.
template <typename T>
__device__ __forceinline__ void tile_chunk_reduce(AccArray<T> &acc, const BFieldParams &F) {
#pragma unroll
    for (int t = 0; t < T::NACC; ++t)
#pragma unroll
        for (int a = 0; a < T::MT; ++a)
#pragma unroll
            for (int b = 0; b < T::NT; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float x = acc[t][a][b][e];
                    acc[t][a][b][e] = fmaf(-F.pf, rintf(x * F.inv_pf), x);
                }
}

// Epilogue: each C_t exactly mod p, then the fold mod P (Alg. 4, fold step,
// in coefficient form: out_i = mu_i + sum_{t >= k} mu_t (X^t mod P)_i), and
// the k output planes written as bytes.
template <int KP, typename T>
__device__ __forceinline__ void tile_epilogue(const AccArray<T> &acc, const BProd &P,
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
                        const uint32_t b0 = __float_as_uint(acc[t][mt][nt][2 * eh] + 12582912.0f);
                        const uint32_t b1 = __float_as_uint(acc[t][mt][nt][2 * eh + 1] + 12582912.0f);
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
                    const float x = acc[t][mt][nt][e];
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

// Output columns per tile on the tensor-core path (k_batched_tc.cu): the
// MMA N = k BN is 128 (80-112 for k = 3, 5, 6, 7) and the 2k-1 accumulators
// (four split ones for k = 2) fit in 256 tensor-memory columns, so two
// tiles' accumulators fit at once.
__host__ __device__ constexpr int tc_bn(uint32_t k) {
    return k <= 1 ? 128 : k == 2 ? 64 : k <= 4 ? 32 : 16;
}

// Launch helpers of the tensor-core path (k_batched_tc.cu).
int tc_stage_layout(uint32_t kmax, int *slot_bytes, int *stages);
int prepare_tc_kernel();
int64_t tc_grid(int64_t ntiles);
int launch_tc_convert(const uint8_t *ws, int64_t nitems, cudaStream_t stream);
int launch_tc_products(const uint8_t *ws, int64_t grid, int slot_bytes, int stages,
                       int *status, cudaStream_t stream);

}  // namespace bt
}  // namespace qadic
