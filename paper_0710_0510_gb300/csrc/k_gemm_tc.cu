// Coefficient-plane GEMM over GF(p^k) on the 5th-generation tensor cores.
//
// Eq. 1 written per coefficient: the product of two elements has the 2k-1
// coefficients C_t = sum_{i+j=t} A_i B_j.  For matrices the same holds with
// A_i, B_j the coefficient planes, so C = A*B over GF(p^k) is k^2 plane
// products accumulated into 2k-1 plane sums, each reduced mod p and then
// folded mod P with X^t mod P (the role of Alg. 4 lines 8-10 / Thm. 3).
//
// GB300 has no integer tcgen05 MMA (kind::i8 does not exist on sm_103a), so
// the planes are fed as bf16 holding small integers exactly (|c| <= 127 <
// 256) and accumulated in FP32 in tensor memory.  FP32 is exact while every
// partial sum stays within 2^24; the host derives the K-chunk for which that
// holds (a drained residue of magnitude <= 2p plus k K h^2, h = (p-1)/2,
// the delayed-reduction argument of Eq. 4 with a 24-bit mantissa), and at
// each chunk boundary the epilogue warps reduce the accumulators in place
// (tcgen05.ld, x - p*rint(x/p), tcgen05.st) before the MMAs continue.
//
// One CTA per 128 x BN output tile, 6 warps:
//   warp 0      TMA producer: per 64-wide K-block, the k A-plane tiles and the
//               k B-plane tiles (128-byte swizzle) into a STAGES-deep ring
//   warp 1      allocates tensor memory; one thread issues tcgen05.mma
//               (M=128, N=BN, K=16) into the 2k-1 accumulators
//   warps 2-5   epilogue: drains, then exact mod p, fold, uint8 planes out
// All waits are bounded (kSpinLimit); on expiry the kernel records
// QADIC_E_DEVICE_TIMEOUT, drains what it issued and frees tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qadic {

namespace {

constexpr int BM = 128, BK = 64, UMMA_K = 16;
constexpr int kGroupM = 16;
constexpr int kThreads = 192;
constexpr int kSmemBudget = 227 * 1024;

template <int KP, int BN>
struct Cfg {
    static constexpr int NACC = 2 * KP - 1;
    static constexpr int A_TILE = BM * BK * 2;
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE = KP * (A_TILE + B_TILE);
    static constexpr int STAGES_RAW = (kSmemBudget - 2048) / STAGE;
    static constexpr int STAGES = STAGES_RAW > 6 ? 6 : STAGES_RAW;
    static constexpr int ACC_COLS = NACC * BN;
    static constexpr int TMEM_COLS = ACC_COLS <= 32 ? 32 : ACC_COLS <= 64 ? 64
                                   : ACC_COLS <= 128 ? 128 : ACC_COLS <= 256 ? 256 : 512;
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
    static constexpr int EC = KP <= 2 ? 32 : 16;   // epilogue columns per pass
    static_assert(ACC_COLS <= 512, "accumulators exceed tensor memory");
    static_assert(KP * BN <= 256 && (KP * BN) % 16 == 0, "combined MMA N must be <= 256");
    static_assert(STAGES >= 2, "not enough shared memory for two stages");
};

struct TcParams {
    int64_t m, n, ldc;
    int32_t tiles_m, tiles_n;   // output tiles; CTAs walk them in groups of kGroupM tile rows
    int32_t nkb;          // K-blocks of 64
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

template <int KP, int BN>
__global__ void __launch_bounds__(kThreads, 1)
gemm_planes_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      uint8_t *__restrict__ C, const TcParams P) {
    using CF = Cfg<KP, BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + CF::STAGES * CF::STAGE);
    uint64_t *empty = full + CF::STAGES;
    uint64_t *acc_full = empty + CF::STAGES;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *mma_done = acc_empty + 1;
    uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // Grouped raster: consecutive CTAs cover kGroupM tile rows before moving
    // to the next tile column, so the A and B panels of the CTAs resident at
    // one time overlap and stay in L2.
    int tile_m, tile_n;
    {
        const int pid = blockIdx.x;
        const int per_group = kGroupM * P.tiles_n;
        const int first_m = (pid / per_group) * kGroupM;
        const int gm = min(P.tiles_m - first_m, kGroupM);
        const int r = pid % per_group;
        tile_m = first_m + r % gm;
        tile_n = r / gm;
    }
    const int nkb = P.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(acc_full, 1);
        ptx::mbar_init(acc_empty, 128);
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

    auto a_tile = [&](int stage, int i) { return smem + stage * CF::STAGE + i * CF::A_TILE; };
    auto b_tile = [&](int stage, int j) {
        return smem + stage * CF::STAGE + KP * CF::A_TILE + j * CF::B_TILE;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            ptx::prefetch_tmap(&tmA);
            ptx::prefetch_tmap(&tmB);
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int stage = kb % CF::STAGES;
                if (kb >= CF::STAGES) {
                    if (*abort_flag ||
                        !ptx::mbar_wait(&empty[stage], ((kb / CF::STAGES) - 1) & 1)) {
                        *abort_flag = 1;
                        break;
                    }
                }
                ptx::mbar_arrive_expect_tx(&full[stage], CF::STAGE);
                for (int i = 0; i < KP; ++i)
                    ptx::tma_load_3d(a_tile(stage, i), &tmA, &full[stage], kb * BK, tile_m * BM, i);
                for (int j = 0; j < KP; ++j)
                    ptx::tma_load_3d(b_tile(stage, j), &tmB, &full[stage], kb * BK, tile_n * BN, j);
                issued = kb + 1;
            }
            if (*abort_flag) {
                // let the copies this thread started land before the CTA exits
                for (int kb = (issued > CF::STAGES ? issued - CF::STAGES : 0); kb < issued; ++kb)
                    ptx::mbar_wait(&full[kb % CF::STAGES], (kb / CF::STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            // The KP B-plane tiles are adjacent in shared memory, so together
            // they form one K-major operand of N = KP*BN rows.  With C_t at
            // TMEM column t*BN, one MMA of A_i against [B_0; ...; B_{KP-1}]
            // at column i*BN adds A_i B_j into C_{i+j} for every j.
            const uint32_t idesc_all = ptx::idesc_bf16_f32(BM, KP * BN);
            const uint32_t idesc_one = ptx::idesc_bf16_f32(BM, BN);
            int drain = 0;
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int stage = kb % CF::STAGES;
                if (*abort_flag || !ptx::mbar_wait(&full[stage], (kb / CF::STAGES) & 1)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint64_t bd0 = ptx::smem_desc_sw128(b_tile(stage, 0));
#pragma unroll
                for (int kk = 0; kk < BK / UMMA_K; ++kk) {
#pragma unroll
                    for (int i = 0; i < KP; ++i) {
                        const uint64_t ad = ptx::smem_desc_sw128(a_tile(stage, i)) + 2 * kk;
                        if (kb == 0 && kk == 0 && i > 0) {
                            // first K step: C_0..C_{i+KP-2} already hold data,
                            // C_{i+KP-1} is written for the first time
#pragma unroll
                            for (int j = 0; j < KP; ++j) {
                                const uint64_t bd = ptx::smem_desc_sw128(b_tile(stage, j));
                                ptx::mma_bf16(tmem_base + (i + j) * BN, ad, bd, idesc_one,
                                              j < KP - 1 ? 1u : 0u);
                            }
                        } else {
                            ptx::mma_bf16(tmem_base + i * BN, ad, bd0 + 2 * kk, idesc_all,
                                          (kb == 0 && kk == 0) ? 0u : 1u);
                        }
                    }
                }
                ptx::mma_commit(&empty[stage]);
                if ((kb + 1) % P.chunk_kb == 0 && kb + 1 < nkb) {
                    ptx::mma_commit(acc_full);
                    if (!ptx::mbar_wait(acc_empty, drain & 1)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    ++drain;
                }
            }
            if (!ok) *abort_flag = 1;
            ptx::mma_commit(acc_full);   // final (or abort) completion
            // every MMA of this CTA has completed once mma_done flips: only
            // then may tensor memory be released
            ptx::mma_commit(mma_done);
            if (!ptx::mbar_wait(mma_done, 0)) *abort_flag = 1;
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int wq = warp & 3;
        const uint32_t tbase = tmem_base + ((uint32_t)(wq * 32) << 16);
        const int ndrain = nkb > 0 ? (nkb - 1) / P.chunk_kb : 0;
        bool ok = true;
        int phase = 0;
        for (int d = 0; d < ndrain; ++d, ++phase) {
            if (!ptx::mbar_wait(acc_full, phase & 1) || *abort_flag) {
                ok = false;
                break;
            }
            ptx::tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < CF::ACC_COLS; c += 32) {
                uint32_t v[32];
                ptx::tmem_ld32(tbase + c, v);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float x = __uint_as_float(v[e]);
                    const float nq = rintf(x * P.inv_pf);
                    v[e] = __float_as_uint(fmaf(-P.pf, nq, x));   // |.| <= 1.5 p, exact
                }
                ptx::tmem_st32(tbase + c, v);
            }
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            ptx::mbar_arrive(acc_empty);
        }
        if (ok) ok = ptx::mbar_wait(acc_full, phase & 1);
        if (*abort_flag) ok = false;
        if (!ok) {
            *abort_flag = 1;
        } else {
            ptx::tc_fence_after();
            const int64_t row = (int64_t)tile_m * BM + wq * 32 + lane;
            constexpr int EC = CF::EC;   // columns per pass (bounds registers)
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += EC) {
                uint32_t mu[CF::NACC][EC];
#pragma unroll
                for (int t = 0; t < CF::NACC; ++t) ptx::tmem_ld<EC>(tbase + t * BN + c0, mu[t]);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < CF::NACC; ++t)
#pragma unroll
                    for (int e = 0; e < EC; ++e) mu[t][e] = mod_exact_f32(mu[t][e], P.pf, P.inv_pf);
                const int64_t col = (int64_t)tile_n * BN + c0;
                if (row < P.m && col < P.n) {
#pragma unroll
                    for (int i = 0; i < KP; ++i) {
                        uint32_t packed[EC / 4];
#pragma unroll
                        for (int w = 0; w < EC / 4; ++w) packed[w] = 0;
#pragma unroll
                        for (int e = 0; e < EC; ++e) {
                            uint32_t o = mu[i][e];
#pragma unroll
                            for (int t = KP; t < 2 * KP - 1; ++t)
                                o = mod_small(o + mu[t][e] * P.fold[(t - KP) * KP + i], P.p, P.m32);
                            packed[e / 4] |= o << (8 * (e % 4));
                        }
                        uint8_t *dst = C + ((int64_t)i * P.m + row) * P.ldc + col;
                        if (col + EC <= P.n && (((uintptr_t)dst) & 15) == 0) {
#pragma unroll
                            for (int w = 0; w < EC / 16; ++w)
                                reinterpret_cast<uint4 *>(dst)[w] =
                                    make_uint4(packed[4 * w], packed[4 * w + 1], packed[4 * w + 2],
                                               packed[4 * w + 3]);
                        } else {
                            const int64_t nrem = P.n - col;
                            const int lim = nrem < EC ? (int)nrem : EC;
                            for (int e = 0; e < lim; ++e)
                                dst[e] = (uint8_t)(packed[e / 4] >> (8 * (e % 4)));
                        }
                    }
                }
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) record_timeout(P.status, 3);
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

// 3-D map over (K, rows, planes) of a k-plane bf16 operand, box (64, box_rows, 1).
int make_plane_map(CUtensorMap *map, const void *base, int64_t K, int64_t rows, int64_t ld,
                   uint32_t planes, uint32_t box_rows) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return set_error(QADIC_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)(rows * ld * 2)};
    const cuuint32_t box[3] = {(cuuint32_t)BK, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(QADIC_E_INVALID, "tensor map encode failed (%d)", (int)r);
    return QADIC_OK;
}

template <int KP, int BN>
int launch_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A, int64_t lda,
              const void *B, int64_t ldb, uint8_t *C, int64_t ldc, cudaStream_t stream) {
    using CF = Cfg<KP, BN>;
    CUtensorMap tmA, tmB;
    int st;
    if ((st = make_plane_map(&tmA, A, K, m, lda, KP, BM))) return st;
    if ((st = make_plane_map(&tmB, B, K, n, ldb, KP, BN))) return st;
    TcParams P;
    P.m = m;
    P.n = n;
    P.ldc = ldc;
    P.nkb = (int32_t)((K + BK - 1) / BK);
    P.chunk_kb = (int32_t)(f.k_chunk_f32 / BK);
    if (P.chunk_kb < 1) return set_error(QADIC_E_OVERFLOW, "exact FP32 chunk below one K-block");
    P.p = f.p;
    P.m32 = make_mod_small(f.p);
    P.pf = (float)f.p;
    P.inv_pf = 1.0f / (float)f.p;
    for (uint32_t i = 0; i < kMaxK * kMaxK; ++i) P.fold[i] = 0;
    for (uint32_t t = 0; t + 1 < f.k; ++t)
        for (uint32_t i = 0; i < f.k; ++i) P.fold[t * KP + i] = f.fold[t * f.k + i];
    P.status = device_status_word();
    auto kern = gemm_planes_tc_kernel<KP, BN>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) !=
        cudaSuccess)
        return set_error(QADIC_E_CUDA, "tc smem attribute: %s", cudaGetErrorString(cudaGetLastError()));
    const int64_t tiles_m = (m + BM - 1) / BM, tiles_n = (n + BN - 1) / BN;
    if (tiles_m * tiles_n > 0x7fffffff) return set_error(QADIC_E_INVALID, "too many tiles");
    P.tiles_m = (int32_t)tiles_m;
    P.tiles_n = (int32_t)tiles_n;
    kern<<<(unsigned)(tiles_m * tiles_n), kThreads, CF::SMEM, stream>>>(tmA, tmB, C, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "tc launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace

bool gemm_planes_tc_supported(const Field &f) { return f.k >= 2 && f.k <= 4; }

int launch_gemm_planes_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                          int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                          cudaStream_t stream) {
    if (lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return set_error(QADIC_E_INVALID, "plane operands need ld %% 8 == 0 and 16-byte alignment");
    if (K == 0) {
        for (uint32_t i = 0; i < f.k; ++i)
            if (cudaMemset2DAsync(C + (size_t)i * m * ldc, (size_t)ldc, 0, (size_t)n, (size_t)m,
                                  stream) != cudaSuccess)
                return set_error(QADIC_E_CUDA, "memset: %s", cudaGetErrorString(cudaGetLastError()));
        return QADIC_OK;
    }
    if (f.k == 2) return launch_tc<2, 128>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
    if (f.k == 3) return launch_tc<3, 64>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
    if (f.k == 4) return launch_tc<4, 64>(f, m, n, K, A, lda, B, ldb, C, ldc, stream);
    return set_error(QADIC_E_UNSUPPORTED, "no tensor-core plane kernel for k=%u", f.k);
}

}  // namespace qadic
