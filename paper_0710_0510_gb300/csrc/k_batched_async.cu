// Batched GF(p^k) products from operands converted once: the path that
// qadic_batched_gemm takes when its workspace has room for the converted
// operands (qadic_batched_workspace_size_fields).
//
// Launch 1 (convert_kernel, one block per piece of at most 4096 chunks of a
// product operand, largest first): the uint8 coefficient planes become
// centred operands in the workspace, each element converted once (staging
// bytes through registers converts an A tile again for every column tile of
// its product and a B tile for every row tile).  Fields with p <= 31 get fp8
// e4m3 (exact for |c| <= 15): A as K-major rows padded to 16 bytes, B
// transposed to n x K (the m16n8k32 B fragment wants K-contiguous columns).
// Larger p get bf16: A K-major, B as it is, rows padded to 8 elements.
//
// Launch 2 (async_kernel, persistent, tiles pulled with one atomicAdd each):
// operand tiles go from the converted planes to shared memory with
// cp.async (16 bytes each, zero-filled past the edges) through 2-4 stages
// (more for the smaller tiles), so that the copies of the next K-blocks run
// under the MMAs of this one; fp8 tiles take m16n8k32 e4m3 MMAs, bf16 tiles
// m16n8k16, and the exact-chunk reductions and the epilogue are those of
// the register-staged kernel (batched_tile.cuh).
//
// GF(2^8) (p = 2, k = 8) accumulates in f16: its planes hold 0 and 1, a K
// element adds at most k = 8 to an accumulator, and a chunk of at most
// 2047 / k elements (after which every accumulator is reduced to |x| <= 1)
// keeps each partial sum an integer of magnitude <= 2048, exact in f16 in
// any order of addition.  Half the accumulator registers of FP32.
#include "batched_tile.cuh"

namespace qadic {
namespace bt {

namespace {

constexpr int kConvThreads = 256;   // one thread per table entry when the table is built

// 8 consecutive bytes of a row at `src` (any alignment); only the first
// `valid` are read (none when valid <= 0), the others are zero.  In the full
// case the bytes come from aligned 32-bit loads joined by funnel shifts; every
// word loaded holds at least one of the 8 bytes, so no load leaves the buffer.
__device__ __forceinline__ void load8(const uint8_t *src, int valid, uint32_t (&w)[2]) {
    if (valid >= 8) {
        const uint32_t a = (uint32_t)((uintptr_t)src & 3);
        const uint32_t *base = reinterpret_cast<const uint32_t *>(src - a);
        if (a == 0) {
            w[0] = __ldg(base);
            w[1] = __ldg(base + 1);
        } else {
            const uint32_t x0 = __ldg(base), x1 = __ldg(base + 1), x2 = __ldg(base + 2);
            w[0] = __funnelshift_r(x0, x1, 8 * a);
            w[1] = __funnelshift_r(x1, x2, 8 * a);
        }
    } else {
        uint64_t v = 0;   // (a register: indexing w here would move it to local memory)
        for (int b = 0; b < valid; ++b) v |= (uint64_t)__ldg(src + b) << (8 * b);
        w[0] = (uint32_t)v;
        w[1] = (uint32_t)(v >> 32);
    }
}

// fp8 fields: 16-byte output chunks of e4m3 bytes.  A: rows of A as they
// are (K-major, kp bytes).  B: transposed to B^T [k][n][kp] (K-major too,
// as the m16n8k32 B fragment wants); chunk (plane, K-block of 16, column)
// with the column fastest, so that a warp's byte loads of one K row are
// consecutive.  Each thread takes kUnroll8 chunks per round and issues all
// their loads before it converts any: the launch is bound by the latency
// of those loads, so the bytes in flight per thread set its speed.
constexpr int kUnroll8 = 2;

__device__ __noinline__ void convert_fp8(const BProd &P, const BFieldParams &F, bool isB, uint32_t begin) {
    __shared__ uint8_t tab8[256];
    tab8[threadIdx.x] = fp8_bits(threadIdx.x, F);
    __syncthreads();
    const uint32_t kc = (uint32_t)P.kp / 16;   // 16-byte chunks per row of K
    uint8_t *dst = const_cast<uint8_t *>(reinterpret_cast<const uint8_t *>(isB ? P.B16 : P.A16));
    if (!isB) {
        const uint32_t total = (uint32_t)F.k * (uint32_t)P.m * kc;
        const uint32_t end = min(total, begin + kConvItemChunks);
        const Div32 div_row = make_div32_device(kc);
        for (uint32_t c0 = begin + threadIdx.x; c0 < end; c0 += kConvThreads * kUnroll8) {
            uint32_t w[kUnroll8][4];
#pragma unroll
            for (int u = 0; u < kUnroll8; ++u) {
                const uint32_t c = c0 + u * kConvThreads;
                const uint32_t r = div32(c, div_row);            // plane * m + row
                const int col = (int)(c - r * kc) * 16;
                // past the last chunk: no loads (valid <= 0), zeros
                const int valid = c < end ? P.K - col : 0;
                load8(P.A + (int64_t)r * P.lda + col, valid, *reinterpret_cast<uint32_t(*)[2]>(&w[u][0]));
                load8(P.A + (int64_t)r * P.lda + col + 8, valid - 8, *reinterpret_cast<uint32_t(*)[2]>(&w[u][2]));
            }
#pragma unroll
            for (int u = 0; u < kUnroll8; ++u) {
                const uint32_t c = c0 + u * kConvThreads;
                if (c >= end) break;
                const uint32_t r = div32(c, div_row);
                const int col = (int)(c - r * kc) * 16;
                uint4 o;
                uint32_t *ow = &o.x;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    ow[q] = (uint32_t)tab8[w[u][q] & 0xff] | ((uint32_t)tab8[(w[u][q] >> 8) & 0xff] << 8) |
                            ((uint32_t)tab8[(w[u][q] >> 16) & 0xff] << 16) | ((uint32_t)tab8[w[u][q] >> 24] << 24);
                *reinterpret_cast<uint4 *>(dst + (int64_t)r * P.kp + col) = o;
            }
        }
    } else {
        const uint32_t per_plane = kc * (uint32_t)P.n;
        const uint32_t total = (uint32_t)F.k * per_plane;
        const uint32_t end = min(total, begin + kConvItemChunks);
        const Div32 div_plane = make_div32_device(per_plane), div_n = make_div32_device((uint32_t)P.n);
        for (uint32_t c0 = begin + threadIdx.x; c0 < end; c0 += kConvThreads * kUnroll8) {
            uint32_t raw[kUnroll8][16];
#pragma unroll
            for (int u = 0; u < kUnroll8; ++u) {
                const uint32_t c = c0 + u * kConvThreads;
                const uint32_t plane = div32(c, div_plane);
                const uint32_t rem = c - plane * per_plane;
                const uint32_t kb = div32(rem, div_n);
                const uint32_t col = rem - kb * (uint32_t)P.n;
                const int k0 = (int)kb * 16;
                // rows past K, and every row of a chunk past the last: not read
                const int rows = c < end ? min(16, P.K - k0) : 0;
                const uint8_t *src = P.B + ((int64_t)plane * P.K + k0) * P.ldb + col;
#pragma unroll
                for (int i = 0; i < 16; ++i) raw[u][i] = i < rows ? __ldg(src + (int64_t)i * P.ldb) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kUnroll8; ++u) {
                const uint32_t c = c0 + u * kConvThreads;
                if (c >= end) break;
                const uint32_t plane = div32(c, div_plane);
                const uint32_t rem = c - plane * per_plane;
                const uint32_t kb = div32(rem, div_n);
                const uint32_t col = rem - kb * (uint32_t)P.n;
                const int k0 = (int)kb * 16;
                const int rows = min(16, P.K - k0);
                uint32_t ow[4] = {0, 0, 0, 0};
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const uint32_t v = i < rows ? (uint32_t)tab8[raw[u][i]] : 0u;
                    ow[i / 4] |= v << (8 * (i % 4));
                }
                *reinterpret_cast<uint4 *>(dst + ((int64_t)plane * P.n + col) * P.kp + k0) =
                    make_uint4(ow[0], ow[1], ow[2], ow[3]);
            }
        }
    }
}

__global__ void __launch_bounds__(kConvThreads) convert_kernel(const uint8_t *ws) {
    const BHeader *hdr = reinterpret_cast<const BHeader *>(ws);
    if (blockIdx.x >= hdr->nconv) return;
    // items of at most kConvItemChunks chunks, largest first, so that the
    // blocks are even and the small ones fill the end of the launch
    const ConvItem item = reinterpret_cast<const ConvItem *>(ws + hdr->order_off)[blockIdx.x];
    const int64_t prod = item.op >> 1;
    const bool isB = item.op & 1;
    const BFieldParams *fields = reinterpret_cast<const BFieldParams *>(ws + hdr->fields_off);
    const BProd &P = reinterpret_cast<const BProd *>(ws + hdr->prods_off)[prod];
    const BFieldParams &F = fields[P.field];
    if (F.fp8) {
        convert_fp8(P, F, isB, item.begin);
        return;
    }
    __shared__ uint16_t tab[256];   // byte -> centred operand bits (kConvThreads == 256)
    tab[threadIdx.x] = bf16_bits(threadIdx.x, F);
    __syncthreads();
    const int cols = isB ? P.n : P.K;
    const int64_t rows = (int64_t)F.k * (isB ? P.K : P.m);   // all k planes, one after the other
    const int ld_in = isB ? P.ldb : P.lda, ld_out = isB ? P.np : P.kp;
    const uint8_t *src = isB ? P.B : P.A;
    uint16_t *dst = const_cast<uint16_t *>(isB ? P.B16 : P.A16);
    const uint32_t per_row = (uint32_t)ld_out / 8;
    const uint32_t end = min((uint32_t)rows * per_row, item.begin + kConvItemChunks);   // <= 8 * 4096 * 512
    const Div32 div_row = make_div32_device(per_row);
    // kUnrollConv chunks per thread per round: all their loads are issued
    // before any of them is converted and stored
    constexpr int kUnrollConv = 4;
    for (uint32_t c0 = item.begin + threadIdx.x; c0 < end; c0 += kConvThreads * kUnrollConv) {
        uint32_t w[kUnrollConv][2];
#pragma unroll
        for (int u = 0; u < kUnrollConv; ++u) {
            const uint32_t c = c0 + u * kConvThreads;
            const uint32_t r = div32(c, div_row);
            const int col = (int)(c - r * per_row) * 8;
            // past the row (or past the last chunk): zeros, and tab[0] = 0
            load8(src + (int64_t)r * ld_in + col, c < end ? cols - col : 0, w[u]);
        }
#pragma unroll
        for (int u = 0; u < kUnrollConv; ++u) {
            const uint32_t c = c0 + u * kConvThreads;
            if (c >= end) break;
            const uint32_t r = div32(c, div_row);
            const int col = (int)(c - r * per_row) * 8;
            uint4 o;
            o.x = (uint32_t)tab[w[u][0] & 0xff] | ((uint32_t)tab[(w[u][0] >> 8) & 0xff] << 16);
            o.y = (uint32_t)tab[(w[u][0] >> 16) & 0xff] | ((uint32_t)tab[w[u][0] >> 24] << 16);
            o.z = (uint32_t)tab[w[u][1] & 0xff] | ((uint32_t)tab[(w[u][1] >> 8) & 0xff] << 16);
            o.w = (uint32_t)tab[(w[u][1] >> 16) & 0xff] | ((uint32_t)tab[w[u][1] >> 24] << 16);
            *reinterpret_cast<uint4 *>(dst + (int64_t)r * ld_out + col) = o;
        }
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies of one K-block of operand tiles into a stage: A_s [KP][BM][LDA],
// B_s [KP][BK][LDB], 16-byte pieces; a piece outside the product (rows past
// m, K-rows past K, columns past the padded row) is zero-filled (source size
// 0, the source pointer then only names the buffer's first element).
template <int KP, typename T>
__device__ __forceinline__ void issue_stage(const BProd &P, uint16_t *As, uint16_t *Bs, int row0,
                                            int col0, int k0) {
    constexpr int A_PER_ROW = T::BK / 8, B_PER_ROW = T::BN / 8;
    constexpr int A_CH = KP * T::BM * A_PER_ROW;
    constexpr int B_CH = KP * T::BK * B_PER_ROW;
#pragma unroll
    for (int s = 0; s < (A_CH + B_CH + kThreads - 1) / kThreads; ++s) {
        const int c = threadIdx.x + s * kThreads;
        if (c < A_CH) {
            const int part = c % A_PER_ROW, r = (c / A_PER_ROW) % T::BM, i = c / (A_PER_ROW * T::BM);
            const int gr = row0 + r, gk = k0 + part * 8;
            const bool ok = gr < P.m && gk < P.kp;
            const uint16_t *src = ok ? P.A16 + ((int64_t)i * P.m + gr) * P.kp + gk : P.A16;
            cp_async16((uint32_t)__cvta_generic_to_shared(As + (i * T::BM + r) * T::LDA + part * 8),
                       src, ok ? 16u : 0u);
        } else if (c < A_CH + B_CH) {
            const int cb = c - A_CH;
            const int part = cb % B_PER_ROW, r = (cb / B_PER_ROW) % T::BK, j = cb / (B_PER_ROW * T::BK);
            const int gk = k0 + r, gc = col0 + part * 8;
            const bool ok = gk < P.K && gc < P.np;
            const uint16_t *src = ok ? P.B16 + ((int64_t)j * P.K + gk) * P.np + gc : P.B16;
            cp_async16((uint32_t)__cvta_generic_to_shared(Bs + (j * T::BK + r) * T::LDB + part * 8),
                       src, ok ? 16u : 0u);
        }
    }
}

template <int KP, int BM, int BN, int BK, bool F16>
__device__ __forceinline__ void run_tile_async(const BProd &P, const BFieldParams &F, int tm, int tn,
                                               uint8_t *smem) {
    using T = TileCfg<KP, BM, BN, BK>;
    constexpr int NS = T::NSTAGE;
    constexpr int kStage = T::SMEM / 2;               // 16-bit elements per stage
    constexpr int kAElems = KP * T::BM * T::LDA;
    uint16_t *S = reinterpret_cast<uint16_t *>(smem);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int wm = warp / 2, wn = warp % 2;
    const int row0 = tm * T::BM, col0 = tn * T::BN;

    AccArray<T, F16> acc;
    acc_zero<T, F16>(acc);
    const int nkb = (P.K + BK - 1) / BK;
    const int chunk_blocks = max(1, (F16 ? F.chunk_k16 : F.chunk_k) / BK);
    __syncthreads();   // the previous tile's reads of every stage are done
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {   // K-blocks 0 .. NS-2 in flight
        if (s < nkb) issue_stage<KP, T>(P, S + s * kStage, S + s * kStage + kAElems, row0, col0, s * BK);
        cp_async_commit();
    }
    for (int kb = 0; kb < nkb; ++kb) {
        uint16_t *As = S + (kb % NS) * kStage;
        const int nxt = kb + NS - 1;   // refills the stage read in iteration kb - 1
        if (nxt < nkb) {
            uint16_t *An = S + (nxt % NS) * kStage;
            issue_stage<KP, T>(P, An, An + kAElems, row0, col0, nxt * BK);
        }
        cp_async_commit();       // (empty near the end: keeps the group count uniform)
        cp_async_wait<NS - 1>(); // all but the NS - 1 newest groups: stage kb has landed
        __syncthreads();
#pragma unroll 1
        for (int ks = 0; ks < BK / 16; ++ks)
            tile_mma_step<KP, T, F16>(acc, As, As + kAElems, ks, wm, wn, lane);
        if ((kb + 1) % chunk_blocks == 0 && kb + 1 < nkb) tile_chunk_reduce<T, F16>(acc, F);
        __syncthreads();         // stage kb read by every warp before it is refilled
    }
    tile_epilogue<KP, T, F16>(acc, P, F, row0, col0, wm, wn, lane);
}

// fp8 operand tiles: A [KP][BM][LDA] and B^T [KP][BN][LDB] bytes, 16-byte
// pieces, zero-filled outside the product.
template <int KP, typename T8>
__device__ __forceinline__ void issue_stage8(const BProd &P, uint8_t *As, uint8_t *Bs, int row0, int col0,
                                             int k0) {
    constexpr int PER_ROW = T8::BK / 16;
    constexpr int A_CH = KP * T8::BM * PER_ROW;
    constexpr int B_CH = KP * T8::BN * PER_ROW;
    const uint8_t *A8 = reinterpret_cast<const uint8_t *>(P.A16);
    const uint8_t *B8 = reinterpret_cast<const uint8_t *>(P.B16);
#pragma unroll
    for (int s = 0; s < (A_CH + B_CH + kThreads - 1) / kThreads; ++s) {
        const int c = threadIdx.x + s * kThreads;
        if (c < A_CH) {
            const int part = c % PER_ROW, r = (c / PER_ROW) % T8::BM, i = c / (PER_ROW * T8::BM);
            const int gr = row0 + r, gk = k0 + part * 16;
            const bool ok = gr < P.m && gk < P.kp;
            const uint8_t *src = ok ? A8 + ((int64_t)i * P.m + gr) * P.kp + gk : A8;
            cp_async16((uint32_t)__cvta_generic_to_shared(As + (i * T8::BM + r) * T8::LDA + part * 16), src,
                       ok ? 16u : 0u);
        } else if (c < A_CH + B_CH) {
            const int cb = c - A_CH;
            const int part = cb % PER_ROW, r = (cb / PER_ROW) % T8::BN, j = cb / (PER_ROW * T8::BN);
            const int gn = col0 + r, gk = k0 + part * 16;
            const bool ok = gn < P.n && gk < P.kp;
            const uint8_t *src = ok ? B8 + ((int64_t)j * P.n + gn) * P.kp + gk : B8;
            cp_async16((uint32_t)__cvta_generic_to_shared(Bs + (j * T8::BN + r) * T8::LDB + part * 16), src,
                       ok ? 16u : 0u);
        }
    }
}

template <int KP, int BM, int BN, int BK, bool F16>
__device__ __forceinline__ void run_tile_async8(const BProd &P, const BFieldParams &F, int tm, int tn,
                                                uint8_t *smem) {
    using T8 = TileCfg8<KP, BM, BN, BK>;
    using T = typename T8::W;
    constexpr int NS = T8::NSTAGE;
    constexpr int kStage = T8::SMEM;
    constexpr int kABytes = KP * T8::BM * T8::LDA;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int wm = warp / 2, wn = warp % 2;
    const int row0 = tm * T8::BM, col0 = tn * T8::BN;

    AccArray<T, F16> acc;
    acc_zero<T, F16>(acc);
    const int nkb = (P.K + T8::BK - 1) / T8::BK;
    const int chunk_blocks = max(1, (F16 ? F.chunk_k16 : F.chunk_k) / T8::BK);
    __syncthreads();   // the previous tile's reads of every stage are done
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
        if (s < nkb) issue_stage8<KP, T8>(P, smem + s * kStage, smem + s * kStage + kABytes, row0, col0, s * T8::BK);
        cp_async_commit();
    }
    for (int kb = 0; kb < nkb; ++kb) {
        uint8_t *As = smem + (kb % NS) * kStage;
        const int nxt = kb + NS - 1;
        if (nxt < nkb) {
            uint8_t *An = smem + (nxt % NS) * kStage;
            issue_stage8<KP, T8>(P, An, An + kABytes, row0, col0, nxt * T8::BK);
        }
        cp_async_commit();
        cp_async_wait<NS - 1>();
        __syncthreads();
#pragma unroll 1
        for (int ks = 0; ks < T8::BK / 32; ++ks)
            tile_mma_step8<KP, T8, F16>(acc, As, As + kABytes, ks, wm, wn, lane);
        if ((kb + 1) % chunk_blocks == 0 && kb + 1 < nkb) tile_chunk_reduce<T, F16>(acc, F);
        __syncthreads();
    }
    tile_epilogue<KP, T, F16>(acc, P, F, row0, col0, wm, wn, lane);
}

template <int KP, bool F16>
__device__ __noinline__ void run_tile_async8_cfg(int cfg, const BProd &P, const BFieldParams &F, int tm,
                                                 int tn, uint8_t *smem) {
    constexpr bool kSmall = KP <= 2, kMid = KP > 2 && KP <= 4;
    constexpr TileShape c0 = kSmall ? kShapesK2[0] : kMid ? kShapesK4[0] : kShapesK8[0];
    constexpr TileShape c1 = kSmall ? kShapesK2[1] : kMid ? kShapesK4[1] : kShapesK8[1];
    constexpr TileShape c2 = kSmall ? kShapesK2[2] : kMid ? kShapesK4[2] : kShapesK8[2];
    constexpr TileShape c3 = kSmall ? kShapesK2[3] : kMid ? kShapesK4[3] : kShapesK8[3];
    constexpr TileShape c4 = kSmall ? kShapesK2[4] : kMid ? kShapesK4[4] : kShapesK8[4];
    switch (cfg) {
        case 1: run_tile_async8<KP, c1.bm, c1.bn, c1.bk, F16>(P, F, tm, tn, smem); break;
        case 2: run_tile_async8<KP, c2.bm, c2.bn, c2.bk, F16>(P, F, tm, tn, smem); break;
        case 3: run_tile_async8<KP, c3.bm, c3.bn, c3.bk, F16>(P, F, tm, tn, smem); break;
        case 4:
            if constexpr (num_cfgs(KP) > 4) {
                run_tile_async8<KP, c4.bm, c4.bn, c4.bk, F16>(P, F, tm, tn, smem);
                break;
            }
            [[fallthrough]];
        default: run_tile_async8<KP, c0.bm, c0.bn, c0.bk, F16>(P, F, tm, tn, smem); break;
    }
}

// Not inlined: each (k, F16) is register-allocated on its own.
template <int KP, bool F16>
__device__ __noinline__ void run_tile_async_cfg(int cfg, const BProd &P, const BFieldParams &F,
                                                int tm, int tn, uint8_t *smem) {
    constexpr bool kSmall = KP <= 2, kMid = KP > 2 && KP <= 4;
    constexpr TileShape c0 = kSmall ? kShapesK2[0] : kMid ? kShapesK4[0] : kShapesK8[0];
    constexpr TileShape c1 = kSmall ? kShapesK2[1] : kMid ? kShapesK4[1] : kShapesK8[1];
    constexpr TileShape c2 = kSmall ? kShapesK2[2] : kMid ? kShapesK4[2] : kShapesK8[2];
    constexpr TileShape c3 = kSmall ? kShapesK2[3] : kMid ? kShapesK4[3] : kShapesK8[3];
    constexpr TileShape c4 = kSmall ? kShapesK2[4] : kMid ? kShapesK4[4] : kShapesK8[4];
    switch (cfg) {
        case 1: run_tile_async<KP, c1.bm, c1.bn, c1.bk, F16>(P, F, tm, tn, smem); break;
        case 2: run_tile_async<KP, c2.bm, c2.bn, c2.bk, F16>(P, F, tm, tn, smem); break;
        case 3: run_tile_async<KP, c3.bm, c3.bn, c3.bk, F16>(P, F, tm, tn, smem); break;
        case 4:
            if constexpr (num_cfgs(KP) > 4) {
                run_tile_async<KP, c4.bm, c4.bn, c4.bk, F16>(P, F, tm, tn, smem);
                break;
            }
            [[fallthrough]];
        default: run_tile_async<KP, c0.bm, c0.bn, c0.bk, F16>(P, F, tm, tn, smem); break;
    }
}

__global__ void __launch_bounds__(kThreads, 5) async_kernel(uint8_t *ws) {
    extern __shared__ __align__(128) uint8_t smem[];   // the stages of the largest tile in the list
    __shared__ int s_tile;
    BHeader *hdr = reinterpret_cast<BHeader *>(ws);
    const BFieldParams *fields = reinterpret_cast<const BFieldParams *>(ws + hdr->fields_off);
    const BProd *prods = reinterpret_cast<const BProd *>(ws + hdr->prods_off);
    const BTile *tiles = reinterpret_cast<const BTile *>(ws + hdr->tiles_off);
    const int ntiles = hdr->ntiles;
    while (true) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&hdr->counter, 1u);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= ntiles) break;
        const BTile tile = tiles[t];
        const BProd &P = prods[tile.prod];
        const BFieldParams &F = fields[P.field];
        if (F.fp8) {
            switch (F.k) {
                case 1: run_tile_async8_cfg<1, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                case 2: run_tile_async8_cfg<2, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                case 3: run_tile_async8_cfg<3, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                case 4: run_tile_async8_cfg<4, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                case 5: run_tile_async8_cfg<5, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                case 6: run_tile_async8_cfg<6, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                case 7: run_tile_async8_cfg<7, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
                default:
                    if (F.f16) run_tile_async8_cfg<8, true>(P.cfg, P, F, tile.tm, tile.tn, smem);
                    else run_tile_async8_cfg<8, false>(P.cfg, P, F, tile.tm, tile.tn, smem);
                    break;
            }
            continue;
        }
        switch (F.k) {
            case 1: run_tile_async_cfg<1, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            case 2: run_tile_async_cfg<2, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            case 3: run_tile_async_cfg<3, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            case 4: run_tile_async_cfg<4, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            case 5: run_tile_async_cfg<5, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            case 6: run_tile_async_cfg<6, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            case 7: run_tile_async_cfg<7, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
            default: run_tile_async_cfg<8, false>(P.cfg, P, F, tile.tm, tile.tn, smem); break;
        }
    }
}

}  // namespace

size_t async_smem_bytes(uint32_t k, int cfg, bool fp8) {
    const size_t stage = fp8 ? tile_smem_bytes8(k, cfg) : tile_smem_bytes(k, cfg);
    return async_stages(stage) * stage;
}

int prepare_async_kernel() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        size_t most = 0;
        for (uint32_t k = 1; k <= kMaxK; ++k)
            for (int c = 0; c < num_cfgs(k); ++c)
                most = std::max(most, std::max(async_smem_bytes(k, c, false), async_smem_bytes(k, c, true)));
        err = cudaFuncSetAttribute(async_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    });
    if (err != cudaSuccess)
        return set_error(QADIC_E_CUDA, "batched smem attribute: %s", cudaGetErrorString(err));
    return QADIC_OK;
}

int64_t async_grid(size_t smem, int64_t ntiles) {
    int64_t grid = resident_blocks(async_kernel, kThreads, smem);
    if (ntiles < grid) grid = std::max<int64_t>(1, ntiles);
    return grid;
}

int launch_convert(const uint8_t *ws, int64_t nitems, cudaStream_t stream) {
    convert_kernel<<<(unsigned)nitems, kConvThreads, 0, stream>>>(ws);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "batched convert launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

int launch_async(uint8_t *ws, int64_t grid, size_t smem, cudaStream_t stream) {
    async_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(ws);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "batched launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace bt
}  // namespace qadic
