// Coefficient-plane GEMM over GF(p^k) on the 5th-generation tensor cores.
//
// Eq. 1 written per coefficient: the product of two elements has the 2k-1
// coefficients C_t = sum_{i+j=t} A_i B_j.  For matrices the same holds with
// A_i, B_j the coefficient planes, so C = A*B over GF(p^k) is k^2 plane
// products accumulated into 2k-1 plane sums, each reduced mod p and then
// folded mod P with X^t mod P (the role of Alg. 4's fold step / Thm. 3).
//
// GB300 has no integer tcgen05 MMA (kind::i8 does not exist on sm_103a), so
// the planes are fed as bf16 holding small integers exactly (|c| <= 127 <
// 256) and accumulated in FP32 in tensor memory.  FP32 is exact while every
// partial sum stays within 2^24; the host derives the K-chunk for which that
// holds (a drained residue of magnitude <= 2p plus k K h^2, h = (p-1)/2,
// the delayed-reduction argument of Eq. 3 with a 24-bit mantissa), and at
// each chunk boundary the epilogue warps reduce the accumulators in place
// (tcgen05.ld, x - p*rint(x/p), tcgen05.st) before the MMAs continue.
//
// The k B-plane tiles of a stage sit next to each other in shared memory and
// form one K-major operand of N = k*BN rows; with C_t at tensor-memory
// column t*BN, one MMA of A_i against [B_0; ...; B_{k-1}] at column i*BN
// adds A_i B_j into C_{i+j} for every j (k MMAs per 16-wide K step).  For
// k = 2 the middle sum is split instead (A_0 B_1 and A_1 B_0 land in two
// accumulators, four in all), so each FP32 accumulator gathers one plane
// product only and the exact chunk grows by a factor k: at K = 4096 a tile
// needs no drain at all.
//
// Persistent: one CTA per SM walks output tiles (grouped raster) with
//   warp 0      TMA producer, streaming K-blocks of consecutive tiles into a
//               STAGES-deep ring without a break between tiles
//   warp 1      allocates tensor memory; one thread issues tcgen05.mma
//   warps 2-9   epilogue, two warps per 32-lane quarter: in-place drains; at
//               the end of a tile they read the accumulators 16 columns at
//               a time, release tensor memory to the next tile's MMAs after
//               the last read, and reduce mod p, fold mod P and store while
//               those MMAs run.
// All waits are bounded (kSpinLimit); on expiry the kernel records
// QADIC_E_DEVICE_TIMEOUT, lets its copies land and frees tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qadic {

namespace {

// K-block of 64 bf16 = 128-byte rows (128-byte swizzle), 64 KB stages for
// k = 2.  32-wide K-blocks with 64-byte swizzle fit seven stages instead of
// three but measured 30% slower on GB300.
constexpr int BM = 128, BK = 64, UMMA_K = 16;
constexpr int kRowBytes = BK * 2;
static_assert(kRowBytes == 64 || kRowBytes == 128, "supported swizzle widths");

__device__ __forceinline__ uint64_t operand_desc(const void *tile) {
    if constexpr (kRowBytes == 128) return ptx::smem_desc_sw128(tile);
    else return ptx::smem_desc_sw64(tile);
}
// Operand element type of the plane GEMMs: bf16 (64 elements per 128-byte
// K-block row, 16 per MMA) or fp8 e4m3 for p <= 31 (128 and 32: the same
// bytes per row and per MMA, so the shared-memory layout, the descriptor
// steps and the MMA count per K-block are the same; a K-block covers twice
// the K and the MMAs run at the fp8 rate).
template <bool FP8>
struct OpT {
    static constexpr int KE = FP8 ? 128 : 64;   // K elements per K-block
    __device__ static uint32_t idesc(uint32_t M, uint32_t N) {
        return FP8 ? ptx::idesc_e4m3_f32(M, N) : ptx::idesc_bf16_f32(M, N);
    }
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
        if constexpr (FP8) ptx::mma_e4m3(d, a, b, idesc, acc);
        else ptx::mma_bf16(d, a, b, idesc, acc);
    }
    __device__ static void mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
        if constexpr (FP8) ptx::mma_e4m3_pair(d, a, b, idesc, acc);
        else ptx::mma_bf16_pair(d, a, b, idesc, acc);
    }
};

constexpr int kGroupM = 16;
// Eight epilogue warps, two per 32-lane quarter of tensor memory, each taking
// half of the quarter's columns.  The epilogue is latency-bound (tensor-
// memory loads, then dependent reduce/fold chains), and tensor memory goes to
// the next tile's MMAs only when the last columns have been read, so two
// warps per sub-partition shorten that wait (register cap 204 per thread at
// 320 threads; no kernel spills).
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kSmemBudget = 227 * 1024;

// Accumulator layouts in tensor memory (C_t = sum_{i+j=t} A_i B_j):
//   shared (SPLIT = false): C_t at column t*BN, 2k-1 accumulators; the MMA of
//     A_i against [B_0; ...; B_{k-1}] starts at column i*BN, so products of
//     different A planes meet in the same accumulator;
//   split (SPLIT = true, k = 2): the MMA of A_i starts at column i*k*BN, so
//     every accumulator receives one product per K step: [C_0 | C_1a | C_1b |
//     C_2], C_1 = C_1a + C_1b in the epilogue.  One product per K step
//     doubles the exact FP32 chunk (k h^2 -> h^2 per K step).
template <int KP, int BN>
struct Cfg {
    static constexpr bool SPLIT = KP == 2;
    static constexpr int NACC = SPLIT ? KP * KP : 2 * KP - 1;   // tensor-memory accumulators
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = KP * (A_TILE + B_TILE);
    static constexpr int STAGES_RAW = (kSmemBudget - 2048) / STAGE;
    static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
    static constexpr int ACC_COLS = NACC * BN;
    // column of the MMA for A plane i
    static constexpr int a_col(int i) { return SPLIT ? i * KP * BN : i * BN; }
    // plane sum t collected by accumulator a
    static constexpr int sum_of(int a) { return SPLIT ? (a / KP) + (a % KP) : a; }
    static constexpr int TMEM_COLS = ACC_COLS <= 32 ? 32 : ACC_COLS <= 64 ? 64
                                   : ACC_COLS <= 128 ? 128 : ACC_COLS <= 256 ? 256 : 512;
    static constexpr int HALF = BN * 4 / kEpiWarps;   // columns per epilogue warp
    static constexpr int CH = HALF / 32;         // 32-column chunks per epilogue warp
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
    static_assert(ACC_COLS <= 512, "accumulators exceed tensor memory");
    static_assert(KP * BN <= 256 && (KP * BN) % 16 == 0, "combined MMA N must be <= 256");
    static_assert(HALF % 32 == 0, "epilogue works on 32-column chunks");
    static_assert(STAGES >= 2, "not enough shared memory for two stages");
};

struct TcParams {
    int64_t m, n, ldc;
    int64_t c_plane;      // elements between output planes
    // Work units are output tiles: units_m = tiles_m, nunits = units_m * tiles_n.
    int32_t tiles_m, tiles_n, units_m, nunits;
    int32_t nkb;          // K-blocks of BK
    int32_t chunk_kb;     // K-blocks per exact FP32 chunk
    uint32_t p, m32;
    float pf, inv_pf;
    uint32_t fold[kMaxK * kMaxK];   // X^(k+t) mod P, row t, k coefficients
    int *status;
};

__device__ __forceinline__ uint32_t mod_exact_f32(uint32_t bits, float pf, float inv_pf) {
    const float x = __uint_as_float(bits);
    const float nq = floorf(x * inv_pf);
    float r = fmaf(-pf, nq, x);   // exact: an integer of magnitude < 2p
    if (r < 0.f) r += pf;
    if (r >= pf) r -= pf;
    return (uint32_t)r;
}

// Grouped raster: consecutive unit indices cover kGroupM unit rows before the
// next tile column, so the A and B panels in use at one time stay in L2.
template <typename Params>
__device__ __forceinline__ void unit_coords(int unit, const Params &P, int &um, int &tn) {
    const int per_group = kGroupM * P.tiles_n;
    const int first_m = (unit / per_group) * kGroupM;
    const int gm = min(P.units_m - first_m, kGroupM);
    const int r = unit % per_group;
    um = first_m + r % gm;
    tn = r / gm;
}

// In-place reduction of a warp's share of every accumulator at an exact-
// chunk boundary: x -> x - p rint(x / p), |result| <= 1.5 p, exact in FP32.
// NB 32-column loads are in flight per wait, so the tensor-memory load
// latency is paid NACC * CH / NB times per drain, not NACC * CH.
template <class CF, int BN>
__device__ __forceinline__ void drain_accumulators(uint32_t tbase, const TcParams &P) {
    constexpr int NB = CF::CH < 4 ? CF::CH : 4;
    static_assert(CF::CH % NB == 0, "drain batches");
#pragma unroll 1
    for (int t = 0; t < CF::NACC; ++t)
#pragma unroll 1
        for (int c = 0; c < CF::HALF; c += 32 * NB) {
            uint32_t v[NB][32];
#pragma unroll
            for (int b = 0; b < NB; ++b) ptx::tmem_ld32(tbase + t * BN + c + 32 * b, v[b]);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int b = 0; b < NB; ++b) {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float x = __uint_as_float(v[b][e]);
                    const float nq = rintf(x * P.inv_pf);
                    v[b][e] = __float_as_uint(fmaf(-P.pf, nq, x));   // |.| <= 1.5 p, exact
                }
                ptx::tmem_st32(tbase + t * BN + c + 32 * b, v[b]);
            }
        }
    ptx::tmem_wait_st();
}

// Accumulators feeding plane sum t (two for C_1 with split accumulators).
template <class CF>
__host__ __device__ constexpr int feeders(int t) {
    int c = 0;
    for (int a = 0; a < CF::NACC; ++a) c += CF::sum_of(a) == t ? 1 : 0;
    return c;
}

// A plane-sum residue |s| <= 127 as one byte, s + 128: the low byte of
// s + (1.5 * 2^23 + 128), exact in FP32 (the spacing there is 1); and back.
constexpr float kByteMagic = 12583040.f;   // 1.5 * 2^23 + 128
__device__ __forceinline__ uint32_t byte_code(float s) { return __float_as_uint(s + kByteMagic); }
__device__ __forceinline__ float byte_value(uint32_t word, int b) {
    return __uint_as_float(0x4B400000u | ((word >> (8 * b)) & 0xFFu)) - kByteMagic;
}

// A warp's share of a finished tile: row `row` (this thread's lane), columns
// col0 .. col0 + HALF.  Two passes, so that tensor memory goes back to the
// MMAs as early as possible: the first reads every accumulator column of the
// share and keeps each plane sum as a centred residue in one byte; release()
// runs after its last load; the second folds and stores.  A residue is
// x - p rint(x RN(1/p)): for |x| < 2^24 the product is within 2/p of x / p,
// so rint is off by at most one and only where the centred residue exceeds
// p/2 - 2, which leaves |r| < p/2 + 2 <= 127.5.  C_1 of the split
// accumulators (the sum of two residues) takes one more such step (exact
// there).  The fold out_i = s_i + sum_t s_t (X^t mod P)_i runs in FP32 FMAs
// (every value below 2^17, exact) and only the k outputs take the exact
// reduction to [0, p).
template <int KP, int BN, class CF, class Release>
__device__ __forceinline__ void tile_epilogue(uint32_t tbase, int64_t row, int64_t col0,
                                              uint8_t *__restrict__ C, const TcParams &P,
                                              const float *foldf, Release release) {
    constexpr int NS = 2 * KP - 1;
    constexpr int NG = CF::HALF / 16;   // 16-column groups
    uint32_t code[NG][NS][4];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        uint32_t v[CF::NACC][16];
#pragma unroll
        for (int t = 0; t < CF::NACC; ++t) ptx::tmem_ld16(tbase + t * BN + 16 * g, v[t]);
        ptx::tmem_wait_ld();
        if (g == NG - 1) release();   // tensor memory may take the next tile's MMAs
        float s[NS][16];
#pragma unroll
        for (int t = 0; t < NS; ++t)
#pragma unroll
            for (int e = 0; e < 16; ++e) s[t][e] = 0.f;
#pragma unroll
        for (int a = 0; a < CF::NACC; ++a)
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float x = __uint_as_float(v[a][e]);
                s[CF::sum_of(a)][e] += fmaf(-P.pf, rintf(x * P.inv_pf), x);
            }
#pragma unroll
        for (int t = 0; t < NS; ++t) {
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (feeders<CF>(t) > 1) s[t][e] = fmaf(-P.pf, rintf(s[t][e] * P.inv_pf), s[t][e]);
#pragma unroll
            for (int w = 0; w < 4; ++w)
                code[g][t][w] = __byte_perm(__byte_perm(byte_code(s[t][4 * w]), byte_code(s[t][4 * w + 1]), 0x0040),
                                            __byte_perm(byte_code(s[t][4 * w + 2]), byte_code(s[t][4 * w + 3]), 0x0040),
                                            0x5410);
        }
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int64_t col = col0 + 16 * g;
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            uint32_t word[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                word[w] = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float o = byte_value(code[g][i][w], b);
#pragma unroll
                    for (int t = KP; t < NS; ++t)
                        o = fmaf(byte_value(code[g][t][w], b), foldf[(t - KP) * KP + i], o);
                    word[w] |= mod_exact_f32(__float_as_uint(o), P.pf, P.inv_pf) << (8 * b);
                }
            }
            if (row < P.m && col < P.n) {
                uint8_t *dst = C + (int64_t)i * P.c_plane + row * P.ldc + col;
                if (col + 16 <= P.n && (((uintptr_t)dst) & 15) == 0) {
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(word[0], word[1], word[2], word[3]);
                } else {
                    const int64_t nrem = P.n - col;
                    const int lim = nrem < 16 ? (int)nrem : 16;
                    for (int e = 0; e < lim; ++e) dst[e] = (uint8_t)(word[e / 4] >> (8 * (e % 4)));
                }
            }
        }
    }
}

// One CTA per output tile at a time; a stage is refilled once the MMAs that
// read it have completed (their commit arrives on the stage's "empty" barrier).
template <int KP, int BN, bool FP8>
__global__ void __launch_bounds__(kThreads, 1)
gemm_planes_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      uint8_t *__restrict__ C, const TcParams P) {
    using CF = Cfg<KP, BN>;
    const int unit0 = blockIdx.x, unit_step = gridDim.x;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + CF::STAGES * CF::STAGE);
    uint64_t *empty = full + CF::STAGES;
    uint64_t *acc_full = empty + CF::STAGES;   // MMAs of a chunk / a tile completed
    uint64_t *acc_empty = acc_full + 1;        // a drain finished
    uint64_t *tmem_free = acc_empty + 1;       // a tile's accumulators were read out
    uint64_t *mma_done = tmem_free + 1;
    uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nkb = P.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(acc_full, 1);
        ptx::mbar_init(acc_empty, 32 * kEpiWarps);
        ptx::mbar_init(tmem_free, 32 * kEpiWarps);
        ptx::mbar_init(mma_done, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, CF::TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    ptx::griddep_wait();   // the set-up above overlaps the previous kernel's tail

    auto a_tile = [&](int stage, int i) { return smem + stage * CF::STAGE + i * CF::A_TILE; };
    auto b_tile = [&](int stage, int j) {
        return smem + stage * CF::STAGE + KP * CF::A_TILE + j * CF::B_TILE;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            ptx::prefetch_tmap(&tmA);
            ptx::prefetch_tmap(&tmB);
            int64_t it = 0;   // K-blocks issued so far, over all tiles
            bool ok = true;
            for (int unit = unit0; unit < P.nunits && ok; unit += unit_step) {
                int um, tn;
                unit_coords(unit, P, um, tn);
                const int tm = um;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int stage = (int)(it % CF::STAGES);
                    if (it >= CF::STAGES) {
                        if (*abort_flag ||
                            !ptx::mbar_wait(&empty[stage], (uint32_t)((it / CF::STAGES) - 1) & 1)) {
                            ok = false;
                            break;
                        }
                    }
                    // the k A tiles and the k B tiles of this K-block
                    ptx::mbar_arrive_expect_tx(&full[stage], CF::STAGE);
                    for (int i = 0; i < KP; ++i)
                        ptx::tma_load_3d(a_tile(stage, i), &tmA, &full[stage], kb * OpT<FP8>::KE, tm * BM, i);
                    for (int j = 0; j < KP; ++j)
                        ptx::tma_load_3d(b_tile(stage, j), &tmB, &full[stage], kb * OpT<FP8>::KE, tn * BN, j);
                }
            }
            if (!ok) {
                *abort_flag = 1;
                // let the copies this thread started land before the CTA exits
                for (int64_t j = (it > CF::STAGES ? it - CF::STAGES : 0); j < it; ++j)
                    ptx::mbar_wait(&full[j % CF::STAGES], (uint32_t)(j / CF::STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc_all = OpT<FP8>::idesc(BM, KP * BN);
            const uint32_t idesc_one = OpT<FP8>::idesc(BM, BN);
            int64_t it = 0;
            int drain = 0, tcount = 0;
            bool ok = true;
            for (int unit = unit0; unit < P.nunits && ok; unit += unit_step, ++tcount) {
                if (tcount > 0) {   // the previous tile's accumulators must have been read
                    if (*abort_flag || !ptx::mbar_wait(tmem_free, (uint32_t)(tcount - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                }
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int stage = (int)(it % CF::STAGES);
                    if (*abort_flag ||
                        !ptx::mbar_wait(&full[stage], (uint32_t)(it / CF::STAGES) & 1)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t bd0 = operand_desc(b_tile(stage, 0));
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk) {
#pragma unroll
                        for (int i = 0; i < KP; ++i) {
                            const uint64_t ad = operand_desc(a_tile(stage, i)) + 2 * kk;
                            if (!CF::SPLIT && kb == 0 && kk == 0 && i > 0) {
                                // first K step of a tile: C_0..C_{i+KP-2} hold data,
                                // C_{i+KP-1} is written for the first time
#pragma unroll
                                for (int j = 0; j < KP; ++j) {
                                    const uint64_t bd = operand_desc(b_tile(stage, j));
                                    OpT<FP8>::mma(tmem_base + (i + j) * BN, ad, bd, idesc_one,
                                                  j < KP - 1 ? 1u : 0u);
                                }
                            } else {
                                OpT<FP8>::mma(tmem_base + CF::a_col(i), ad, bd0 + 2 * kk, idesc_all,
                                              (kb == 0 && kk == 0) ? 0u : 1u);
                            }
                        }
                    }
                    ptx::mma_commit(&empty[stage]);
                    if ((kb + 1) % P.chunk_kb == 0 && kb + 1 < nkb) {
                        ptx::mma_commit(acc_full);
                        if (!ptx::mbar_wait(acc_empty, (uint32_t)drain & 1)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        ++drain;
                    }
                }
                if (ok) ptx::mma_commit(acc_full);   // tile complete
            }
            if (!ok) {
                *abort_flag = 1;
                ptx::mma_commit(acc_full);   // wake the epilogue
            }
            // every MMA of this CTA has completed once mma_done flips: only
            // then may tensor memory be released
            ptx::mma_commit(mma_done);
            if (!ptx::mbar_wait(mma_done, 0)) *abort_flag = 1;
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int ew = warp - 2;
        const int quarter = warp & 3;           // TMEM lanes 32*quarter.. (warp % 4 rule)
        const int col_base = (ew / 4) * CF::HALF;   // which half of the quarter's columns
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + col_base;
        const int ndrain = nkb > 0 ? (nkb - 1) / P.chunk_kb : 0;
        float foldf[(KP - 1) * KP + 1];
#pragma unroll
        for (int x = 0; x < (KP - 1) * KP; ++x) foldf[x] = (float)P.fold[x];
        int phase = 0;
        bool ok = true;
        for (int unit = unit0; unit < P.nunits && ok; unit += unit_step) {
            int um, tn;
            unit_coords(unit, P, um, tn);
            const int tm = um;
            for (int d = 0; d < ndrain; ++d, ++phase) {
                if (!ptx::mbar_wait(acc_full, (uint32_t)phase & 1) || *abort_flag) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                drain_accumulators<CF, BN>(tbase, P);
                ptx::tc_fence_before();
                ptx::mbar_arrive(acc_empty);
            }
            if (!ok) break;
            if (!ptx::mbar_wait(acc_full, (uint32_t)phase & 1) || *abort_flag) {
                ok = false;
                break;
            }
            ++phase;
            ptx::tc_fence_after();
            const int64_t row = (int64_t)tm * BM + quarter * 32 + lane;
            const int64_t col0 = (int64_t)tn * BN + col_base;
            tile_epilogue<KP, BN, CF>(tbase, row, col0, C, P, foldf, [&] {
                ptx::tc_fence_before();
                ptx::mbar_arrive(tmem_free);
            });
        }
        if (!ok) *abort_flag = 1;
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) record_timeout(P.status, 3);
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, CF::TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// CTA-pair form (cta_group::2), k = 2, for K within one exact FP32 chunk
// (no in-place reduction).  A cluster of two CTAs on two SMs
// computes a 256 x BN unit: the leader (cluster rank 0) takes output rows
// 0..127 of the unit, the peer rows 128..255.  One MMA of M = 256 per A plane
// and 16-wide K step covers both: each CTA holds its own 128 rows of A_i and
// one half of the combined operand [B_0; B_1] (the leader B_0's tile, the
// peer B_1's), so each SM stages and reads half of the B bytes per multiply-
// add that a one-CTA tile needs.  Each CTA's tensor memory holds its rows of
// the four split accumulators [C_0 | C_1a | C_1b | C_2] (512 columns).
//   warp 0      both CTAs: TMA producer for its own tiles.  The loads of both
//               CTAs complete on the leader's "full" barrier (cta_group::2
//               TMA); the leader announces the transaction bytes of both.
//   warp 1      both CTAs allocate the pair's tensor memory; the leader's lane
//               0 issues the MMAs and commits each stage's completion to the
//               "empty" barriers, and each tile's to the "accumulators
//               ready" barriers, of both CTAs.
//   warps 2-9   both CTAs: epilogue of its own rows; every epilogue warp of
//               both CTAs arrives on the leader's "read out" barrier (one
//               arrival per warp).
// Waits are bounded; an expired wait raises the abort flag of both CTAs.
// After an abort each CTA gives in-flight copies a bounded time to land
// before the final cluster barrier, then both free tensor memory and exit.
template <int KP, int BN>
struct PairCfg {
    static_assert(KP == 2, "the pair kernel uses the split accumulators of k = 2");
    static constexpr int NACC = KP * KP;
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_ROWS = KP * BN / 2;             // this CTA's half of [B_0; B_1]
    static constexpr int B_HALF = B_ROWS * BK * 2;
    static constexpr int BOX = BN;                         // rows per B load (one plane tile)
    static constexpr int NBOX = B_ROWS / BOX;
    static constexpr int STAGE = KP * A_TILE + B_HALF;     // bytes per CTA per stage
    static constexpr int STAGES_RAW = (kSmemBudget - 2048) / STAGE;
    static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
    static constexpr int ACC_COLS = NACC * BN;
    static constexpr int a_col(int i) { return i * KP * BN; }
    static constexpr int sum_of(int a) { return (a / KP) + (a % KP); }
    static constexpr int TMEM_COLS = ACC_COLS <= 32 ? 32 : ACC_COLS <= 64 ? 64
                                   : ACC_COLS <= 128 ? 128 : ACC_COLS <= 256 ? 256 : 512;
    static constexpr int HALF = BN * 4 / kEpiWarps;
    static constexpr int CH = HALF / 32;
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
    static_assert(ACC_COLS <= 512, "accumulators exceed tensor memory");
    static_assert(KP * BN <= 256 && (KP * BN) % 16 == 0, "pair MMA N must be <= 256");
    static_assert(B_ROWS % BOX == 0 && BOX <= 256, "B half in whole loads");
    static_assert(HALF % 32 == 0, "epilogue works on 32-column chunks");
    static_assert(STAGES >= 2, "not enough shared memory for two stages");
};

// Bounded settling time after an abort: copies issued before the abort land
// within microseconds; the CTAs wait this long before leaving the cluster.
constexpr uint64_t kSettleNs = 2000000;

template <int KP, int BN, bool FP8>
__global__ void __launch_bounds__(kThreads, 1)
gemm_planes_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        uint8_t *__restrict__ C, const TcParams P) {
    using CF = PairCfg<KP, BN>;
    const uint32_t rank = ptx::cluster_ctarank();   // 0: leader, 1: peer
    const uint32_t peer = rank ^ 1u;
    const int unit0 = blockIdx.x / 2, unit_step = gridDim.x / 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + CF::STAGES * CF::STAGE);
    uint64_t *empty = full + CF::STAGES;
    uint64_t *acc_full = empty + CF::STAGES;   // a tile's MMAs completed
    uint64_t *tmem_free = acc_full + 1;        // both CTAs read a tile's accumulators out
    uint64_t *mma_done = tmem_free + 1;
    uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
    volatile uint32_t *abort_flag = (volatile uint32_t *)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nkb = P.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(acc_full, 1);
        ptx::mbar_init(tmem_free, 2 * kEpiWarps);
        ptx::mbar_init(mma_done, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc_pair(tmem_slot, CF::TMEM_COLS);
        ptx::tmem_relinquish_pair();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::cluster_sync();   // both CTAs' barriers and tensor memory exist before any remote use
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    ptx::griddep_wait();   // the set-up above overlaps the previous kernel's tail

    auto in_leader = [&](const void *x) { return ptx::mapa(ptx::smem_addr(x), 0); };
    auto in_peer = [&](const void *x) { return ptx::mapa(ptx::smem_addr(x), peer); };
    const uint32_t peer_abort = in_peer((const void *)abort_flag);
    auto abort_both = [&]() {
        *abort_flag = 1;
        ptx::st_cluster_u32(peer_abort, 1);
    };
    auto a_tile = [&](int stage, int i) { return smem + stage * CF::STAGE + i * CF::A_TILE; };
    auto b_half = [&](int stage) { return smem + stage * CF::STAGE + KP * CF::A_TILE; };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs) ----------------
            ptx::prefetch_tmap(&tmA);
            ptx::prefetch_tmap(&tmB);
            int64_t it = 0;
            bool ok = true;
            for (int unit = unit0; unit < P.nunits && ok; unit += unit_step) {
                int um, tn;
                unit_coords(unit, P, um, tn);
                const int tm = um * 2 + (int)rank;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int stage = (int)(it % CF::STAGES);
                    if (it >= CF::STAGES) {
                        if (*abort_flag ||
                            !ptx::mbar_wait_cluster(&empty[stage],
                                                    (uint32_t)((it / CF::STAGES) - 1) & 1)) {
                            ok = false;
                            break;
                        }
                    }
                    const uint32_t fb = in_leader(&full[stage]);
                    if (rank == 0) ptx::mbar_arrive_expect_tx(&full[stage], 2 * CF::STAGE);
                    for (int i = 0; i < KP; ++i)
                        ptx::tma_load_3d_pair(a_tile(stage, i), &tmA, fb, kb * OpT<FP8>::KE, tm * BM, i);
                    for (int b = 0; b < CF::NBOX; ++b) {
                        const int row = ((int)rank * CF::NBOX + b) * CF::BOX;   // in [B_0; B_1]
                        ptx::tma_load_3d_pair(b_half(stage) + b * CF::BOX * kRowBytes, &tmB, fb,
                                              kb * OpT<FP8>::KE, tn * BN + row % BN, row / BN);
                    }
                }
            }
            if (!ok) abort_both();
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- MMA issuer (leader) ----------------
            const uint32_t idesc = OpT<FP8>::idesc(2 * BM, KP * BN);
            const uint32_t peer_empty0 = in_peer(&empty[0]), peer_acc_full = in_peer(acc_full);
            auto commit_both = [&](uint64_t *bar, uint32_t peer_bar) {
                ptx::mma_commit_pair(bar);
                ptx::mma_commit_pair_at(peer_bar);
            };
            int64_t it = 0;
            int tcount = 0;
            bool ok = true;
            for (int unit = unit0; unit < P.nunits && ok; unit += unit_step, ++tcount) {
                if (tcount > 0) {   // both CTAs have read the previous tile's accumulators
                    if (*abort_flag ||
                        !ptx::mbar_wait_cluster(tmem_free, (uint32_t)(tcount - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                }
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int stage = (int)(it % CF::STAGES);
                    if (*abort_flag ||
                        !ptx::mbar_wait_cluster(&full[stage], (uint32_t)(it / CF::STAGES) & 1)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t bd = operand_desc(b_half(stage));
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk)
#pragma unroll
                        for (int i = 0; i < KP; ++i)
                            OpT<FP8>::mma_pair(tmem_base + CF::a_col(i),
                                               operand_desc(a_tile(stage, i)) + 2 * kk, bd + 2 * kk,
                                               idesc, (kb == 0 && kk == 0) ? 0u : 1u);
                    commit_both(&empty[stage], peer_empty0 + 8 * stage);
                }
                if (ok) commit_both(acc_full, peer_acc_full);   // tile complete
            }
            if (!ok) {
                abort_both();
                commit_both(acc_full, peer_acc_full);   // wake the epilogues
            }
            // every MMA has completed (in both CTAs' tensor memory) once
            // mma_done flips: only then may tensor memory be released
            ptx::mma_commit_pair(mma_done);
            if (!ptx::mbar_wait(mma_done, 0)) abort_both();
        }
    } else {
        // ---------------- epilogue (warps 2..9, both CTAs) ----------------
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int col_base = (ew / 4) * CF::HALF;
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + col_base;
        const uint32_t lead_tmem_free = in_leader(tmem_free);
        float foldf[(KP - 1) * KP + 1];
#pragma unroll
        for (int x = 0; x < (KP - 1) * KP; ++x) foldf[x] = (float)P.fold[x];
        auto ready = [&](int ph) { return ptx::mbar_wait_cluster(acc_full, (uint32_t)ph & 1); };
        auto arrive_warp = [&](uint32_t lead_bar) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive_cluster(lead_bar);
        };
        int phase = 0;
        bool ok = true;
        for (int unit = unit0; unit < P.nunits && ok; unit += unit_step) {
            int um, tn;
            unit_coords(unit, P, um, tn);
            const int tm = um * 2 + (int)rank;
            if (!ready(phase) || *abort_flag) {
                ok = false;
                break;
            }
            ++phase;
            ptx::tc_fence_after();
            const int64_t row = (int64_t)tm * BM + quarter * 32 + lane;
            const int64_t col0 = (int64_t)tn * BN + col_base;
            tile_epilogue<KP, BN, CF>(tbase, row, col0, C, P, foldf,
                                      [&] { arrive_warp(lead_tmem_free); });
        }
        if (!ok) abort_both();
    }

    ptx::tc_fence_before();
    const bool aborted = __syncthreads_or(*abort_flag != 0) != 0;
    if (aborted) {
        if (threadIdx.x == 0) {
            const uint64_t t0 = ptx::globaltimer_ns();
            while (ptx::globaltimer_ns() - t0 < kSettleNs) __nanosleep(10000);
        }
        __syncthreads();
    }
    // neither CTA leaves while the other may still arrive on its barriers,
    // copy into its shared memory or have MMAs write its tensor memory
    ptx::cluster_sync();
    if (threadIdx.x == 0 && aborted) record_timeout(P.status, 5);
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc_pair(tmem_base, CF::TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Fold-before-GEMM form.  out_j = sum_i A_i M_ij(B), where M_ij(B) is plane
// j of B X^i mod P (the columns of b's multiplication matrix): the
// reduction mod P moves in front of the contraction, which becomes one
// prime-field GEMM of m x (k n_pad) over k K, the k output planes side by
// side.  The pack step writes the operand as k planes (index i), plane i
// being the k blocks M_i0, ..., M_i,k-1 (n_pad rows each, K-major), so a
// K-block of plane i of A meets the same K-block of plane i of the operand.
// The K loop runs over (K-block, plane i) pairs, one tile of each per stage
// (all planes of a K-block before the next, so that CTAs on nearby tiles
// read the same operand K-slices at about the same time and meet in L2);
// each plane has its own accumulator (one product per K step, so the exact
// FP32 chunk is (2^24 - 2p) / h^2), and the epilogue adds the k
// accumulators and reduces mod p -- no fold, no 2k-1 plane sums.
//
// The same streaming serves the Karatsuba form for k = 2 (EPI_KARATSUBA):
// three operand plane pairs (A_0, B_0), (A_1, B_1), (A_0 + A_1, B_0 + B_1)
// (sums reduced and centred by the pack step) give D_0 = A_0 B_0,
// D_2 = A_1 B_1 and D_m, so C_1 = D_m - D_0 - D_2: three plane products
// instead of four.  The epilogue combines them and folds C_2 with X^2 mod P.
constexpr int EPI_FOLD = 0, EPI_KARATSUBA = 1;

struct FoldParams {
    int64_t m, n, n_pad, ldc, c_plane;
    int32_t tiles_m, tiles_n, units_m, nunits;
    int32_t nkbp;         // K-blocks per plane
    int32_t chunk_kb;     // K-blocks per exact FP32 chunk of one accumulator
    float pf, inv_pf;
    float x2[2];          // Karatsuba: X^2 mod P
    int *status;
};

template <int KP, int BN>
struct FoldCfg {
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = A_TILE + B_TILE;
    static constexpr int STAGES_RAW = (kSmemBudget - 2048) / STAGE;
    static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
    static constexpr int ACC_COLS = KP * BN;
    static constexpr int TMEM_COLS = ACC_COLS <= 32 ? 32 : ACC_COLS <= 64 ? 64
                                   : ACC_COLS <= 128 ? 128 : ACC_COLS <= 256 ? 256 : 512;
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
    static_assert(ACC_COLS <= 512, "accumulators exceed tensor memory");
    static_assert(BN <= 256 && BN % 16 == 0, "MMA N");
    static_assert(STAGES >= 2, "not enough shared memory for two stages");
};

template <int KP, int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 1)
gemm_fold_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    uint8_t *__restrict__ C, const FoldParams P) {
    using CF = FoldCfg<KP, BN>;
    const int unit0 = blockIdx.x, unit_step = gridDim.x;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + CF::STAGES * CF::STAGE);
    uint64_t *empty = full + CF::STAGES;
    uint64_t *acc_full = empty + CF::STAGES;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *tmem_free = acc_empty + 1;
    uint64_t *mma_done = tmem_free + 1;
    uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nkbp = P.nkbp;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(acc_full, 1);
        ptx::mbar_init(acc_empty, 32 * kEpiWarps);
        ptx::mbar_init(tmem_free, 32 * kEpiWarps);
        ptx::mbar_init(mma_done, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, CF::TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    auto a_tile = [&](int stage) { return smem + stage * CF::STAGE; };
    auto b_tile = [&](int stage) { return smem + stage * CF::STAGE + CF::A_TILE; };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: (K-block, plane) pairs ----------------
            ptx::prefetch_tmap(&tmA);
            ptx::prefetch_tmap(&tmB);
            int64_t it = 0;
            bool ok = true;
            for (int unit = unit0; unit < P.nunits && ok; unit += unit_step) {
                int um, tn;
                unit_coords(unit, P, um, tn);
                const int tm = um;
                for (int kb = 0; kb < nkbp && ok; ++kb)
                    for (int i = 0; i < KP; ++i, ++it) {
                        const int stage = (int)(it % CF::STAGES);
                        if (it >= CF::STAGES) {
                            if (*abort_flag ||
                                !ptx::mbar_wait(&empty[stage], (uint32_t)((it / CF::STAGES) - 1) & 1)) {
                                ok = false;
                                break;
                            }
                        }
                        ptx::mbar_arrive_expect_tx(&full[stage], CF::STAGE);
                        ptx::tma_load_3d(a_tile(stage), &tmA, &full[stage], kb * BK, tm * BM, i);
                        ptx::tma_load_3d(b_tile(stage), &tmB, &full[stage], kb * BK, tn * BN, i);
                    }
            }
            if (!ok) {
                *abort_flag = 1;
                for (int64_t j = (it > CF::STAGES ? it - CF::STAGES : 0); j < it; ++j)
                    ptx::mbar_wait(&full[j % CF::STAGES], (uint32_t)(j / CF::STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
            int64_t it = 0;
            int drain = 0, tcount = 0;
            bool ok = true;
            for (int unit = unit0; unit < P.nunits && ok; unit += unit_step, ++tcount) {
                if (tcount > 0) {
                    if (*abort_flag || !ptx::mbar_wait(tmem_free, (uint32_t)(tcount - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                }
                for (int kb = 0; kb < nkbp && ok; ++kb) {
                    for (int i = 0; i < KP; ++i, ++it) {
                        const int stage = (int)(it % CF::STAGES);
                        if (*abort_flag ||
                            !ptx::mbar_wait(&full[stage], (uint32_t)(it / CF::STAGES) & 1)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint64_t ad = operand_desc(a_tile(stage));
                        const uint64_t bd = operand_desc(b_tile(stage));
#pragma unroll
                        for (int kk = 0; kk < BK / UMMA_K; ++kk)
                            ptx::mma_bf16(tmem_base + i * BN, ad + 2 * kk, bd + 2 * kk, idesc,
                                          (kb == 0 && kk == 0) ? 0u : 1u);
                        ptx::mma_commit(&empty[stage]);
                    }
                    if (ok && (kb + 1) % P.chunk_kb == 0 && kb + 1 < nkbp) {
                        // exact-chunk boundary of every accumulator at once
                        ptx::mma_commit(acc_full);
                        if (!ptx::mbar_wait(acc_empty, (uint32_t)drain & 1)) {
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        ++drain;
                    }
                }
                if (ok) ptx::mma_commit(acc_full);   // tile complete
            }
            if (!ok) {
                *abort_flag = 1;
                ptx::mma_commit(acc_full);
            }
            ptx::mma_commit(mma_done);
            if (!ptx::mbar_wait(mma_done, 0)) *abort_flag = 1;
        }
    } else {
        // ---------------- epilogue (warps 2 ..) ----------------
        // kEpiWarps / 4 warps share each 32-lane quarter, splitting its columns
        constexpr int kPerQuarter = kEpiWarps / 4;
        const int quarter = warp & 3, part = (warp - 2) / 4;
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16);
        constexpr int kDrainCols = CF::ACC_COLS / kPerQuarter;   // accumulator columns reduced per warp
        constexpr int kOutCols = BN / kPerQuarter;               // output columns per warp
        static_assert(kDrainCols % 32 == 0 && kOutCols % 16 == 0, "epilogue column split");
        const int ndrain = nkbp > 0 ? (nkbp - 1) / P.chunk_kb : 0;
        int phase = 0;
        bool ok = true;
        for (int unit = unit0; unit < P.nunits && ok; unit += unit_step) {
            int um, tn;
            unit_coords(unit, P, um, tn);
            const int tm = um;
            for (int d = 0; d < ndrain; ++d, ++phase) {
                // in-place reduction of every accumulator
                if (!ptx::mbar_wait(acc_full, (uint32_t)phase & 1) || *abort_flag) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
#pragma unroll 1
                for (int c = part * kDrainCols; c < (part + 1) * kDrainCols; c += 32) {
                    uint32_t v[32];
                    ptx::tmem_ld32(tbase + c, v);
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float x = __uint_as_float(v[e]);
                        v[e] = __float_as_uint(fmaf(-P.pf, rintf(x * P.inv_pf), x));
                    }
                    ptx::tmem_st32(tbase + c, v);
                }
                ptx::tmem_wait_st();
                ptx::tc_fence_before();
                ptx::mbar_arrive(acc_empty);
            }
            if (!ok) break;
            if (!ptx::mbar_wait(acc_full, (uint32_t)phase & 1) || *abort_flag) {
                ok = false;
                break;
            }
            ++phase;
            ptx::tc_fence_after();
            const int64_t row = (int64_t)tm * BM + quarter * 32 + lane;
            const int c_begin = part * kOutCols, c_end = c_begin + kOutCols;
            if constexpr (EPI == EPI_KARATSUBA) {
#pragma unroll 1
                for (int c = c_begin; c < c_end; c += 16) {
                    float r[3][16];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        uint32_t v[16];
                        ptx::tmem_ld16(tbase + a * BN + c, v);
                        ptx::tmem_wait_ld();
                        if (c + 16 >= c_end && a == 2) {
                            ptx::tc_fence_before();
                            ptx::mbar_arrive(tmem_free);
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const float x = __uint_as_float(v[e]);
                            r[a][e] = fmaf(-P.pf, rintf(x * P.inv_pf), x);   // |.| <= 1.5 p
                        }
                    }
                    // C_0 = D_0, C_2 = D_2, C_1 = D_m - D_0 - D_2; out_i = C_i + C_2 (X^2 mod P)_i
                    uint32_t word[2][4];
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        word[0][w] = word[1][w] = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int e = 4 * w + b;
                            const float c2 = r[1][e];
                            const float o0 = fmaf(c2, P.x2[0], r[0][e]);
                            const float o1 = fmaf(c2, P.x2[1], r[2][e] - r[0][e] - r[1][e]);
                            word[0][w] |= mod_exact_f32(__float_as_uint(o0), P.pf, P.inv_pf) << (8 * b);
                            word[1][w] |= mod_exact_f32(__float_as_uint(o1), P.pf, P.inv_pf) << (8 * b);
                        }
                    }
                    const int64_t col = (int64_t)tn * BN + c;
                    if (row < P.m && col < P.n) {
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            uint8_t *dst = C + i * P.c_plane + row * P.ldc + col;
                            if (col + 16 <= P.n && (((uintptr_t)dst) & 15) == 0) {
                                *reinterpret_cast<uint4 *>(dst) =
                                    make_uint4(word[i][0], word[i][1], word[i][2], word[i][3]);
                            } else {
                                const int64_t nrem = P.n - col;
                                const int lim = nrem < 16 ? (int)nrem : 16;
                                for (int e = 0; e < lim; ++e)
                                    dst[e] = (uint8_t)(word[i][e / 4] >> (8 * (e % 4)));
                            }
                        }
                    }
                }
                continue;
            }
#pragma unroll 1
            for (int c = c_begin; c < c_end; c += 16) {
                float s[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) s[e] = 0.f;
#pragma unroll 1
                for (int a = 0; a < KP; ++a) {
                    uint32_t v[16];
                    ptx::tmem_ld16(tbase + a * BN + c, v);
                    ptx::tmem_wait_ld();
                    if (c + 16 >= c_end && a == KP - 1) {
                        ptx::tc_fence_before();
                        ptx::mbar_arrive(tmem_free);
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float x = __uint_as_float(v[e]);
                        s[e] += fmaf(-P.pf, rintf(x * P.inv_pf), x);   // |.| <= 1.5 p each
                    }
                }
                uint32_t word[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    word[w] = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        word[w] |= mod_exact_f32(__float_as_uint(s[4 * w + b]), P.pf, P.inv_pf)
                                   << (8 * b);
                }
                // output column block j = plane j (n_pad is a multiple of BN)
                const int64_t colx = (int64_t)tn * BN + c;
                const int64_t j = colx / P.n_pad, col = colx - j * P.n_pad;
                if (row < P.m && col < P.n) {
                    uint8_t *dst = C + j * P.c_plane + row * P.ldc + col;
                    if (col + 16 <= P.n && (((uintptr_t)dst) & 15) == 0) {
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(word[0], word[1], word[2], word[3]);
                    } else {
                        const int64_t nrem = P.n - col;
                        const int lim = nrem < 16 ? (int)nrem : 16;
                        for (int e = 0; e < lim; ++e) dst[e] = (uint8_t)(word[e / 4] >> (8 * (e % 4)));
                    }
                }
            }
        }
        if (!ok) *abort_flag = 1;
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) record_timeout(P.status, 4);
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, CF::TMEM_COLS);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D map over (K, rows, planes) of a k-plane operand, box (one 128-byte
// K-block row, box_rows, 1): bf16 (64 elements) or, with fp8, e4m3 bytes
// (128 elements).
int make_plane_map(CUtensorMap *map, const void *base, int64_t K, int64_t rows, int64_t ld,
                   int64_t plane_stride, uint32_t planes, uint32_t box_rows, bool fp8 = false) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return set_error(QADIC_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    const int64_t esz = fp8 ? 1 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * esz), (cuuint64_t)(plane_stride * esz)};
    const cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / esz), box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           3, const_cast<void *>(base), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           kRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(QADIC_E_INVALID, "tensor map encode failed (%d)", (int)r);
    return QADIC_OK;
}

template <int KP, int BN, bool FP8 = false>
int launch_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A, int64_t lda,
              int64_t a_plane, const void *B, int64_t ldb, int64_t b_plane, uint8_t *C,
              int64_t ldc, int64_t c_plane, cudaStream_t stream) {
    using CF = Cfg<KP, BN>;
    CUtensorMap tmA, tmB;
    int st;
    if ((st = make_plane_map(&tmA, A, K, m, lda, a_plane, KP, BM, FP8))) return st;
    if ((st = make_plane_map(&tmB, B, K, n, ldb, b_plane, KP, BN, FP8))) return st;
    constexpr int KE = OpT<FP8>::KE;
    TcParams P;
    P.m = m;
    P.n = n;
    P.ldc = ldc;
    P.c_plane = c_plane;
    P.nkb = (int32_t)((K + KE - 1) / KE);
    // exact FP32 chunk: a drained residue (|.| <= 1.5p < 2p) plus the growth
    // per K step (k h^2 with shared accumulators, h^2 with split ones) must
    // stay within 2^24
    const int64_t hh = (int64_t)f.h * f.h;
    const int64_t chunk = CF::SPLIT ? ((1ll << 24) - 2 * (int64_t)f.p) / hh : f.k_chunk_f32;
    P.chunk_kb = (int32_t)std::min<int64_t>(chunk / KE, 1 << 30);
    if (P.chunk_kb < 1) return set_error(QADIC_E_OVERFLOW, "exact FP32 chunk below one K-block");
    P.p = f.p;
    P.m32 = make_mod_small(f.p);
    P.pf = (float)f.p;
    P.inv_pf = 1.0f / (float)f.p;
    for (uint32_t i = 0; i < kMaxK * kMaxK; ++i) P.fold[i] = 0;
    for (uint32_t t = 0; t + 1 < f.k; ++t)
        for (uint32_t i = 0; i < f.k; ++i) P.fold[t * KP + i] = f.fold[t * f.k + i];
    P.status = device_status_word();
    auto kern = gemm_planes_tc_kernel<KP, BN, FP8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) !=
        cudaSuccess)
        return set_error(QADIC_E_CUDA, "tc smem attribute: %s", cudaGetErrorString(cudaGetLastError()));
    const int64_t tiles_m = (m + BM - 1) / BM, tiles_n = (n + BN - 1) / BN;
    const int64_t units_m = tiles_m;
    if (units_m * tiles_n > 0x7fffffff) return set_error(QADIC_E_INVALID, "too many tiles");
    P.tiles_m = (int32_t)tiles_m;
    P.tiles_n = (int32_t)tiles_n;
    P.units_m = (int32_t)units_m;
    P.nunits = (int32_t)(units_m * tiles_n);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = CF::SMEM;
    cfg.stream = stream;
    // persistent: one CTA per SM (one fits: 227 KB of shared memory each)
    const int units = (int)std::min<int64_t>(P.nunits, std::max(sms, 1));
    cfg.gridDim = dim3((unsigned)units);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, tmA, tmB, C, P);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(QADIC_E_CUDA, "tc launch: %s", cudaGetErrorString(e));
    }
    return QADIC_OK;
}

// CTA-pair launch: clusters of two CTAs, one pair per two SMs, persistent
// over 256 x BN units.
template <int KP, int BN, bool FP8 = false>
int launch_tc_pair(const Field &f, int64_t m, int64_t n, int64_t K, const void *A, int64_t lda,
                   int64_t a_plane, const void *B, int64_t ldb, int64_t b_plane, uint8_t *C,
                   int64_t ldc, int64_t c_plane, cudaStream_t stream) {
    using CF = PairCfg<KP, BN>;
    CUtensorMap tmA, tmB;
    int st;
    if ((st = make_plane_map(&tmA, A, K, m, lda, a_plane, KP, BM, FP8))) return st;
    if ((st = make_plane_map(&tmB, B, K, n, ldb, b_plane, KP, CF::BOX, FP8))) return st;
    constexpr int KE = OpT<FP8>::KE;
    TcParams P;
    P.m = m;
    P.n = n;
    P.ldc = ldc;
    P.c_plane = c_plane;
    P.nkb = (int32_t)((K + KE - 1) / KE);
    // split accumulators: a drained residue (|.| <= 1.5p < 2p) plus h^2 per K step
    const int64_t hh = (int64_t)f.h * f.h;
    const int64_t chunk = ((1ll << 24) - 2 * (int64_t)f.p) / hh;
    P.chunk_kb = (int32_t)std::min<int64_t>(chunk / KE, 1 << 30);
    if (P.chunk_kb < P.nkb)
        return set_error(QADIC_E_UNSUPPORTED, "pair kernel: K beyond one exact FP32 chunk");
    P.p = f.p;
    P.m32 = make_mod_small(f.p);
    P.pf = (float)f.p;
    P.inv_pf = 1.0f / (float)f.p;
    for (uint32_t i = 0; i < kMaxK * kMaxK; ++i) P.fold[i] = 0;
    for (uint32_t t = 0; t + 1 < f.k; ++t)
        for (uint32_t i = 0; i < f.k; ++i) P.fold[t * KP + i] = f.fold[t * f.k + i];
    P.status = device_status_word();
    auto kern = gemm_planes_pair_kernel<KP, BN, FP8>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) !=
        cudaSuccess)
        return set_error(QADIC_E_CUDA, "pair smem attribute: %s", cudaGetErrorString(cudaGetLastError()));
    const int64_t tiles_m = (m + BM - 1) / BM, tiles_n = (n + BN - 1) / BN;
    const int64_t units_m = (tiles_m + 1) / 2;
    if (units_m * tiles_n > 0x7fffffff) return set_error(QADIC_E_INVALID, "too many tiles");
    P.tiles_m = (int32_t)tiles_m;
    P.tiles_n = (int32_t)tiles_n;
    P.units_m = (int32_t)units_m;
    P.nunits = (int32_t)(units_m * tiles_n);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;   // the cluster shape alone for the occupancy query
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = CF::SMEM;
    cfg.stream = stream;
    int pairs = std::max(sms / 2, 1);
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0)
        pairs = std::min(pairs, clusters);
    else
        cudaGetLastError();
    pairs = (int)std::min<int64_t>(P.nunits, pairs);
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    cfg.numAttrs = 2;   // and the launch may overlap the previous kernel's tail
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, tmA, tmB, C, P);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(QADIC_E_CUDA, "pair launch: %s", cudaGetErrorString(e));
    }
    return QADIC_OK;
}

template <int KP, int BN, int EPI = EPI_FOLD>
int launch_fold(const Field &f, int64_t m, int64_t n, int64_t K, const void *A, int64_t lda,
                const void *B, int64_t ldb, uint8_t *C, int64_t ldc, cudaStream_t stream) {
    using CF = FoldCfg<KP, BN>;
    // fold: B rows are KP blocks of n_pad; Karatsuba: B rows are the n columns
    const int64_t n_pad = EPI == EPI_FOLD ? fold_n_pad(n) : n;
    const int64_t b_rows = EPI == EPI_FOLD ? KP * n_pad : n;
    CUtensorMap tmA, tmB;
    int st;
    if ((st = make_plane_map(&tmA, A, K, m, lda, m * lda, KP, BM))) return st;
    if ((st = make_plane_map(&tmB, B, K, b_rows, ldb, b_rows * ldb, KP, BN))) return st;
    FoldParams P;
    P.m = m;
    P.n = n;
    P.n_pad = n_pad;
    P.ldc = ldc;
    P.c_plane = m * ldc;
    P.nkbp = (int32_t)((K + BK - 1) / BK);
    const int64_t hh = (int64_t)f.h * f.h;
    const int64_t chunk = ((1ll << 24) - 2 * (int64_t)f.p) / (hh ? hh : 1);
    P.chunk_kb = (int32_t)std::min<int64_t>(chunk / BK, 1 << 30);
    if (P.chunk_kb < 1) return set_error(QADIC_E_OVERFLOW, "exact FP32 chunk below one K-block");
    P.pf = (float)f.p;
    P.inv_pf = 1.0f / (float)f.p;
    P.x2[0] = P.x2[1] = 0.f;
    if (EPI == EPI_KARATSUBA) {
        P.x2[0] = (float)f.fold[0];
        P.x2[1] = (float)f.fold[1];
    }
    P.status = device_status_word();
    auto kern = gemm_fold_tc_kernel<KP, BN, EPI>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) !=
        cudaSuccess)
        return set_error(QADIC_E_CUDA, "fold smem attribute: %s", cudaGetErrorString(cudaGetLastError()));
    const int64_t tiles_m = (m + BM - 1) / BM;
    const int64_t tiles_n = EPI == EPI_FOLD ? KP * n_pad / BN : (n + BN - 1) / BN;
    const int64_t units_m = tiles_m;
    if (units_m * tiles_n > 0x7fffffff) return set_error(QADIC_E_INVALID, "too many tiles");
    P.tiles_m = (int32_t)tiles_m;
    P.tiles_n = (int32_t)tiles_n;
    P.units_m = (int32_t)units_m;
    P.nunits = (int32_t)(units_m * tiles_n);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = CF::SMEM;
    cfg.stream = stream;
    const int units = (int)std::min<int64_t>(P.nunits, std::max(sms, 1));
    cfg.gridDim = dim3((unsigned)units);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, tmA, tmB, C, P);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(QADIC_E_CUDA, "fold launch: %s", cudaGetErrorString(e));
    }
    return QADIC_OK;
}

}  // namespace

bool gemm_planes_tc_supported(const Field &f) { return f.k >= 2 && f.k <= 4; }

int launch_gemm_planes_tc_strided(const Field &f, int64_t m, int64_t n, int64_t K,
                                  const void *A, int64_t lda, int64_t a_plane, const void *B,
                                  int64_t ldb, int64_t b_plane, uint8_t *C, int64_t ldc,
                                  int64_t c_plane, cudaStream_t stream, bool fp8) {
    // TMA: 16-byte aligned bases and row / plane strides of whole 16 bytes
    const int64_t e16 = fp8 ? 16 : 8;   // elements per 16 bytes
    if (lda % e16 || ldb % e16 || a_plane % e16 || b_plane % e16 || ((uintptr_t)A & 15) ||
        ((uintptr_t)B & 15))
        return set_error(QADIC_E_INVALID, "plane operands need ld %% %d == 0 and 16-byte alignment",
                         (int)e16);
    if (fp8 && f.p > 31)
        return set_error(QADIC_E_UNSUPPORTED, "e4m3 operands need p <= 31 (|c| <= 15 exact)");
    if (K == 0) {
        for (uint32_t i = 0; i < f.k; ++i)
            if (cudaMemset2DAsync(C + (size_t)i * c_plane, (size_t)ldc, 0, (size_t)n, (size_t)m,
                                  stream) != cudaSuccess)
                return set_error(QADIC_E_CUDA, "memset: %s", cudaGetErrorString(cudaGetLastError()));
        return QADIC_OK;
    }
#define QADIC_TC(KP_, BN_)                                                                            \
    (fp8 ? launch_tc<KP_, BN_, true>(f, m, n, K, A, lda, a_plane, B, ldb, b_plane, C, ldc, c_plane,    \
                                     stream)                                                          \
         : launch_tc<KP_, BN_, false>(f, m, n, K, A, lda, a_plane, B, ldb, b_plane, C, ldc, c_plane,   \
                                      stream))
    if (f.k == 2) {
        // Two tile rows or more and no in-place reduction on the way through
        // K: CTA pairs on 256-row units.  Where the exact FP32 chunk is
        // shorter than K, both SMs of a pair wait for every reduction, and
        // the one-CTA kernel measured faster (GF(251^2), n = 16384: 21.4 ms
        // against 22.3 ms).
        const int64_t ke = fp8 ? 128 : 64;   // K elements per K-block
        const int64_t hh = (int64_t)f.h * f.h;
        const int64_t chunk_kb = ((1ll << 24) - 2 * (int64_t)f.p) / hh / ke;
        if (m > BM && (K + ke - 1) / ke <= chunk_kb)
            return fp8 ? launch_tc_pair<2, 128, true>(f, m, n, K, A, lda, a_plane, B, ldb, b_plane, C,
                                                      ldc, c_plane, stream)
                       : launch_tc_pair<2, 128, false>(f, m, n, K, A, lda, a_plane, B, ldb, b_plane,
                                                       C, ldc, c_plane, stream);
        return QADIC_TC(2, 128);
    }
    if (f.k == 3) return QADIC_TC(3, 64);
    if (f.k == 4) return QADIC_TC(4, 64);
#undef QADIC_TC
    return set_error(QADIC_E_UNSUPPORTED, "no tensor-core plane kernel for k=%u", f.k);
}

int launch_gemm_planes_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                          int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                          cudaStream_t stream, bool fp8) {
    return launch_gemm_planes_tc_strided(f, m, n, K, A, lda, m * lda, B, ldb, n * ldb, C, ldc,
                                         m * ldc, stream, fp8);
}

int launch_gemm_fold_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                        int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                        cudaStream_t stream) {
    if (lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return set_error(QADIC_E_INVALID, "fold operands need ld %% 8 == 0 and 16-byte alignment");
    if (K == 0) {
        for (uint32_t i = 0; i < f.k; ++i)
            if (cudaMemset2DAsync(C + (size_t)i * m * ldc, (size_t)ldc, 0, (size_t)n, (size_t)m,
                                  stream) != cudaSuccess)
                return set_error(QADIC_E_CUDA, "memset: %s", cudaGetErrorString(cudaGetLastError()));
        return QADIC_OK;
    }
    switch (f.k) {
        case 1: return launch_fold<1, 256>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 2: return launch_fold<2, 256>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 3: return launch_fold<3, 128>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 4: return launch_fold<4, 128>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 5: return launch_fold<5, 64>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 6: return launch_fold<6, 64>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 7: return launch_fold<7, 64>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        case 8: return launch_fold<8, 64>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
        default: return set_error(QADIC_E_UNSUPPORTED, "no fold kernel for k=%u", f.k);
    }
}

int launch_gemm_karatsuba_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                             int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                             cudaStream_t stream) {
    if (f.k != 2) return set_error(QADIC_E_UNSUPPORTED, "the Karatsuba form is for k = 2");
    if (lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return set_error(QADIC_E_INVALID, "Karatsuba operands need ld %% 8 == 0 and 16-byte alignment");
    if (K == 0) {
        for (uint32_t i = 0; i < 2; ++i)
            if (cudaMemset2DAsync(C + (size_t)i * m * ldc, (size_t)ldc, 0, (size_t)n, (size_t)m,
                                  stream) != cudaSuccess)
                return set_error(QADIC_E_CUDA, "memset: %s", cudaGetErrorString(cudaGetLastError()));
        return QADIC_OK;
    }
    return launch_fold<3, 128, EPI_KARATSUBA>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
}

}  // namespace qadic
