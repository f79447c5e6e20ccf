// Batched GF(p^k) products on the 5th-generation tensor cores: the path that
// qadic_batched_gemm takes when its workspace has room for the converted
// operands (qadic_batched_workspace_size_fields).  Per product the math is
// the plane form of Alg. 4: C_t = sum_{i+j=t} A_i B_j over the coefficient
// planes, each C_t reduced mod p, then folded with X^t mod P.
//
// Launch 1 (tc_convert_kernel): the uint8 planes become centred operands in
// the workspace, each element converted once, already cut into the blocks
// the product kernel copies: for every product, operand and 32-byte K-block
// (32 fp8 elements for p <= 31, which e4m3 holds exactly, else 16 bf16), the
// k planes of one 128-row tile of A (rows rounded up to 8) or one BN-column
// tile of B^T, one after the other, each plane in the K-major no-swizzle
// layout of the MMA operand descriptors: 8-row x 16-byte core matrices,
// the two of a row group's K-block adjacent (128 B apart), row groups 256 B
// apart.  Only the K padding is written as zeros: rows of A beyond m and
// columns of B beyond n produce outputs that are never stored.
//
// Launch 2 (tc_products_kernel, persistent, one CTA per SM, tiles taken in
// a fixed stride over the cost-ordered list of tile records, each role
// reading its next record while it works on the current one):
//   warp 0      producer: two cp.async.bulk copies per K-block (the A
//               planes, the B planes) into a ring of stages
//   warp 1      allocates 512 tensor-memory columns (two accumulator
//               buffers of 256); one thread issues tcgen05.mma: per K-block
//               one MMA of M = 128, N = k BN per A plane, A_i against
//               [B_0; ...; B_{k-1}], so C_t sits at column t BN of the buffer
//               (k = 2: split sums [C_0 | C_1a | C_1b | C_2], one product per
//               accumulator per K step)
//   warps 2-9   epilogue in two groups of four warps (one per 32-lane quarter
//               of tensor memory), group g taking the tiles of buffer g:
//               in-place reductions at exact-chunk boundaries, then the
//               tile's plane sums mod p, the fold and the byte stores, while
//               the other group works on the previous tile and the MMAs fill
//               the buffer it released.
// Waits are bounded; on expiry the kernel records QADIC_E_DEVICE_TIMEOUT,
// lets its copies land and frees tensor memory.
#include "batched_tile.cuh"
#include "tc_ptx.cuh"

namespace qadic {
namespace bt {

namespace {

constexpr int kTcEpiWarps = 8;
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr int kTcConvThreads = 256;
constexpr int kTcMaxStages = 8;
constexpr int kTcSmemBudget = 227 * 1024;

// ---------------------------------------------------------------- convert --

// `valid` (<= 16) consecutive bytes of a row at `src`, any alignment; the
// rest zero.
__device__ __forceinline__ void load16(const uint8_t *src, int valid, uint32_t (&w)[4]) {
    if (valid >= 16) {
        const uint32_t a = (uint32_t)((uintptr_t)src & 3);
        const uint32_t *base = reinterpret_cast<const uint32_t *>(src - a);
        if (a == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = __ldg(base + q);
        } else {
            uint32_t x[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) x[q] = __ldg(base + q);
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = __funnelshift_r(x[q], x[q + 1], 8 * a);
        }
    } else {
        uint32_t v[4] = {0, 0, 0, 0};
#pragma unroll
        for (int b = 0; b < 16; ++b)
            if (b < valid) v[b / 4] |= (uint32_t)__ldg(src + b) << (8 * (b % 4));
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = v[q];
    }
}

// 16 output bytes from up to 16 input bytes (fp8: one byte each) or up to 8
// (bf16: two bytes each), through the byte -> operand table.
__device__ __forceinline__ uint4 convert16(const uint32_t (&w)[4], bool fp8, const uint8_t *tab8,
                                           const uint16_t *tab16) {
    uint4 o;
    uint32_t *ow = &o.x;
    if (fp8) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            ow[q] = (uint32_t)tab8[w[q] & 0xff] | ((uint32_t)tab8[(w[q] >> 8) & 0xff] << 8) |
                    ((uint32_t)tab8[(w[q] >> 16) & 0xff] << 16) | ((uint32_t)tab8[w[q] >> 24] << 24);
    } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            ow[2 * q] = (uint32_t)tab16[w[q] & 0xff] | ((uint32_t)tab16[(w[q] >> 8) & 0xff] << 16);
            ow[2 * q + 1] = (uint32_t)tab16[(w[q] >> 16) & 0xff] | ((uint32_t)tab16[w[q] >> 24] << 16);
        }
    }
    return o;
}

__global__ void __launch_bounds__(kTcConvThreads) tc_convert_kernel(const uint8_t *ws) {
    const BHeader *hdr = reinterpret_cast<const BHeader *>(ws);
    if (blockIdx.x >= hdr->nconv) return;
    const ConvItem item = reinterpret_cast<const ConvItem *>(ws + hdr->order_off)[blockIdx.x];
    const BProd &P = reinterpret_cast<const BProd *>(ws + hdr->prods_off)[item.op >> 1];
    const BFieldParams &F = reinterpret_cast<const BFieldParams *>(ws + hdr->fields_off)[P.field];
    const bool isB = item.op & 1;
    const bool fp8 = F.fp8 != 0;
    __shared__ uint8_t tab8[256];
    __shared__ uint16_t tab16[256];
    if (fp8) tab8[threadIdx.x] = fp8_bits(threadIdx.x, F);
    else tab16[threadIdx.x] = bf16_bits(threadIdx.x, F);
    __syncthreads();
    const uint32_t k = F.k, KS = (uint32_t)P.kp;
    const int epc = fp8 ? 16 : 8;            // input elements per 16-byte chunk
    const int epb = 2 * epc;                 // per 32-byte K-block
    uint8_t *base = const_cast<uint8_t *>(reinterpret_cast<const uint8_t *>(isB ? P.B16 : P.A16));
    if (!isB) {
        // A chunks in the order of the blocks: [row tile][K-block][plane]
        // [row group][half][row in group], so chunk c is at byte 16 c
        const uint32_t m = (uint32_t)P.m;
        const uint32_t nfull = m / 128, rows8_last = ((m - nfull * 128) + 7) / 8 * 8;
        const uint32_t per_full = KS * k * 256;
        const uint32_t total = nfull * per_full + KS * k * rows8_last * 2;
        const uint32_t end = min(total, item.begin + kConvItemChunks);
        const Div32 d_full = make_div32_device(per_full);
        for (uint32_t c = item.begin + threadIdx.x; c < end; c += kTcConvThreads) {
            const uint32_t tm = div32(c, d_full);
            uint32_t rem = c - tm * per_full;
            const uint32_t rows8 = tm < nfull ? 128 : rows8_last;
            const uint32_t per_ks = k * rows8 * 2;
            const uint32_t ks = rem / per_ks;
            rem -= ks * per_ks;
            const uint32_t i = rem / (rows8 * 2);
            rem -= i * rows8 * 2;
            const uint32_t g = rem / 16, q = (rem / 8) % 2, r8 = rem % 8;
            const uint32_t R = tm * 128 + g * 8 + r8;
            const int e0 = (int)(ks * epb + q * epc);
            const int valid = R < m ? min(epc, P.K - e0) : 0;
            uint32_t w[4];
            load16(P.A + ((int64_t)i * m + R) * P.lda + e0, valid, w);
            *reinterpret_cast<uint4 *>(base + (size_t)c * 16) = convert16(w, fp8, tab8, tab16);
        }
    } else {
        // B chunks [plane][K-block][half][column]: a warp's byte loads of one
        // K row are consecutive columns
        const uint32_t n = (uint32_t)P.n, BN = (uint32_t)tc_bn(k);
        const uint32_t per_plane = KS * 2 * n, total = k * per_plane;
        const uint32_t end = min(total, item.begin + kConvItemChunks);
        const Div32 d_plane = make_div32_device(per_plane), d_2n = make_div32_device(2 * n),
                    d_n = make_div32_device(n);
        for (uint32_t c = item.begin + threadIdx.x; c < end; c += kTcConvThreads) {
            const uint32_t j = div32(c, d_plane);
            uint32_t rem = c - j * per_plane;
            const uint32_t ks = div32(rem, d_2n);
            rem -= ks * 2 * n;
            const uint32_t q = div32(rem, d_n), col = rem - q * n;
            const int e0 = (int)(ks * epb + q * epc);
            const int valid = min(epc, P.K - e0);
            const uint8_t *src = P.B + ((int64_t)j * P.K + e0) * P.ldb + col;
            uint32_t v[4] = {0, 0, 0, 0};
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (e < epc && e < valid) v[e / 4] |= (uint32_t)__ldg(src + (int64_t)e * P.ldb) << (8 * (e % 4));
            const uint32_t tn = col / BN, cc = col - tn * BN;
            uint8_t *dst = base + ((size_t)tn * KS + ks) * (k * BN * 32) + (size_t)j * BN * 32 +
                           (cc / 8) * 256 + q * 128 + (cc % 8) * 16;
            *reinterpret_cast<uint4 *>(dst) = convert16(v, fp8, tab8, tab16);
        }
    }
}

// --------------------------------------------------------------- products --

// K-major, no-swizzle operand descriptor: 8-row x 16-byte core matrices,
// leading (K-direction) byte offset 128, stride (row-group) byte offset 256.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            ptx::smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(ptx::smem_addr(bar))
        : "memory");
}

// The same in pieces of at most 32 KB (sizes and addresses stay multiples
// of 16 bytes).
__device__ __forceinline__ void bulk_copy_split(void *dst, const void *src, uint32_t bytes,
                                                uint64_t *bar) {
    constexpr uint32_t kPiece = 32768;
    for (uint32_t off = 0; off < bytes; off += kPiece)
        bulk_copy(static_cast<uint8_t *>(dst) + off, static_cast<const uint8_t *>(src) + off,
                  bytes - off < kPiece ? bytes - off : kPiece, bar);
}

// 32 lanes x 8 columns of 32-bit data.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// 32 lanes x 4 columns.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_zero4(uint32_t taddr) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%1,%1,%1};" ::"r"(taddr), "r"(0u)
                 : "memory");
}

template <int CW>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&v)[CW]) {
    if constexpr (CW == 8) tmem_ld8(taddr, v);
    else tmem_ld4(taddr, v);
}

template <int CW>
__device__ __forceinline__ void tmem_zero_cols(uint32_t taddr);

__device__ __forceinline__ void tmem_zero8(uint32_t taddr) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
                 "r"(0u)
                 : "memory");
}

template <int CW>
__device__ __forceinline__ void tmem_zero_cols(uint32_t taddr) {
    if constexpr (CW == 8) tmem_zero8(taddr);
    else tmem_zero4(taddr);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7])
                 : "memory");
}

// The tile record at t (48 bytes, three independent 16-byte loads); t past
// the end gives a record that is never used.
__device__ __forceinline__ TcRec tc_rec(const uint8_t *ws, const BHeader *hdr, int t, int ntiles) {
    TcRec r;
    if (t < ntiles) {
        const uint4 *src = reinterpret_cast<const uint4 *>(ws + hdr->tiles_off) + 3 * (size_t)t;
        uint4 *dst = reinterpret_cast<uint4 *>(&r);
        dst[0] = __ldg(src);
        dst[1] = __ldg(src + 1);
        dst[2] = __ldg(src + 2);
    }
    return r;
}

// In-place reduction of accumulator columns [c0, c0 + w) of accumulators
// 0 .. nacc-1 (x -> x - p rint(x / p), exact).
__device__ __forceinline__ void tc_drain(uint32_t tacc, int nacc, int bn, int c0, int w, float pf,
                                         float inv_pf) {
    for (int a = 0; a < nacc; ++a)
        for (int c = c0; c < c0 + w; c += 8) {
            uint32_t v[8];
            tmem_ld8(tacc + a * bn + c, v);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float x = __uint_as_float(v[e]);
                v[e] = __float_as_uint(fmaf(-pf, rintf(x * inv_pf), x));
            }
            tmem_st8(tacc + a * bn + c, v);
        }
    ptx::tmem_wait_st();
}

// o mod p for an integer-valued float |o| < 2^23 and 3 <= p < 256, on the
// full-rate FP32 pipe: t = o / p rounded to an integer by adding and
// subtracting 1.5 * 2^23 (|o / p| < 2^22), possibly one off, r = o - p t
// exact and within (-2p, 2p), one correction each way, and the integer r
// read off the bits of r + 2^23.
__device__ __forceinline__ uint32_t tc_mod(float o, float pf, float inv_pf) {
    const float t = __fadd_rn(__fmaf_rn(o, inv_pf, 12582912.0f), -12582912.0f);
    float r = __fmaf_rn(-pf, t, o);
    if (r < 0.f) r += pf;
    if (r >= pf) r -= pf;
    return __float_as_uint(r + 8388608.0f) & 0xffu;
}

// Stores 8 columns of one output plane for the warp's 32 rows: lane r holds
// row r's 8 bytes in (lo, hi).  Store j writes byte lane % 8 of row
// lane / 8 + 4 j, taken from that row's lane by two shuffles, so that each
// store instruction covers 8 consecutive bytes of each of 4 rows (the rows
// of a plane start at any byte, so the stores are bytes; with one row per
// lane each instruction would touch 32 rows).  Shuffles, not a shared-memory
// exchange: a warp barrier between exchange steps would also wait for this
// warp's global stores already in flight.  p0 = the lane's byte of row
// (lane / 8) in this plane; rows_left, cols_left: valid rows and columns
// from the first of these.
__device__ __forceinline__ void store_rows8(const uint8_t *p0, int64_t step4, int rows_left,
                                            int cols_left, uint32_t lo, uint32_t hi, int lane) {
    uint8_t *p = const_cast<uint8_t *>(p0);
    const uint32_t sh = 8u * (lane & 3);
    const bool col_ok = (lane & 7) < cols_left;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int src = (lane >> 3) + 4 * j;   // the row this store writes
        const uint32_t wl = __shfl_sync(0xffffffffu, lo, src);
        const uint32_t wh = __shfl_sync(0xffffffffu, hi, src);
        const uint8_t v = (uint8_t)(((lane & 4) ? wh : wl) >> sh);
        if (col_ok && src < rows_left) *p = v;
        p += step4;
    }
}

// Spreads the low 4 bits of x to the low bit of each byte (bit b -> byte b):
// the partial products of x by 1 + 2^7 + 2^14 + 2^21 do not overlap.
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return ((x & 0xFu) * 0x00204081u) & 0x01010101u; }

// A warp's share of a finished tile: its 32 rows from row0 (tile-relative),
// columns [c0, c0 + w) of the tile, 8 at a time; each accumulator is zeroed
// once read.  release() once the last columns have been read.
template <int KP, bool P2, class Release>
__device__ __forceinline__ void tc_epilogue(uint32_t tacc, const TcRec &T,
                                            const BFieldParams &F, int row0, int c0, int w,
                                            Release release) {
    constexpr int NACC = KP == 2 ? 4 : 2 * KP - 1;
    constexpr int BN = tc_bn(KP);
    // tile-relative coordinates: rows [0, T.rows), columns [0, T.cols)
    const int lane = threadIdx.x & 31;
    const int rows_left = T.rows - row0;
    const int64_t ldc = T.ldc, c_plane = T.c_plane;
    const int64_t step4 = 4 * ldc;
    // this lane's byte of row (row0 + lane / 8), column lane % 8 of a chunk
    const uint8_t *const lane_base = T.c + (int64_t)(row0 + (lane >> 3)) * ldc + (lane & 7);
    if constexpr (P2) {
        // GF(2^k): C_t mod 2 for the 8 columns as an 8-bit mask m_t (the
        // low bit of x + 1.5 * 2^23 is the parity of an integer-valued float
        // of magnitude < 2^22), the fold mod P as XORs of the masks of the
        // t >= k whose row X^t mod P has bit i, output plane i = mask bits as
        // bytes.  The accumulators are read NB at a time.
        constexpr int NB = NACC < 8 ? NACC : 8;
        uint32_t fold2[KP > 1 ? KP - 1 : 1];
#pragma unroll
        for (int t = 0; t + 1 < KP; ++t) fold2[t] = F.fold2[t];
        for (int c = c0; c < c0 + w; c += 8) {
            uint32_t mt[2 * KP - 1];
#pragma unroll
            for (int t = 0; t < 2 * KP - 1; ++t) mt[t] = 0;
#pragma unroll
            for (int a0 = 0; a0 < NACC; a0 += NB) {
                uint32_t v[NB][8];
#pragma unroll
                for (int x = 0; x < NB; ++x)
                    if (a0 + x < NACC) tmem_ld8(tacc + (a0 + x) * BN + c, v[x]);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int x = 0; x < NB; ++x)
                    if (a0 + x < NACC) tmem_zero8(tacc + (a0 + x) * BN + c);
                if (a0 + NB >= NACC && c + 8 >= c0 + w) release();
#pragma unroll
                for (int x = 0; x < NB; ++x) {
                    const int a = a0 + x;
                    if (a >= NACC) break;
                    const int t = KP == 2 ? (a / 2) + (a % 2) : a;
                    uint32_t msk = 0;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        msk |= (__float_as_uint(__uint_as_float(v[x][e]) + 12582912.0f) & 1u) << e;
                    mt[t] ^= msk;
                }
            }
            if (rows_left <= 0 || c >= T.cols) continue;   // the same for the whole warp
            const int cols_left = T.cols - c;
#pragma unroll
            for (int i = 0; i < KP; ++i) {
                uint32_t o = mt[i];
#pragma unroll
                for (int t = KP; t < 2 * KP - 1; ++t)
                    o ^= mt[t] & (0u - ((fold2[t - KP] >> i) & 1u));
                store_rows8(lane_base + (int64_t)i * c_plane + c, step4, rows_left, cols_left,
                            spread4(o), spread4(o >> 4), lane);
            }
        }
    } else {
        const float pf = F.pf, inv_pf = F.inv_pf;
        constexpr int NF = KP <= 4 ? (KP - 1) * KP : 1;
        float foldf[NF > 0 ? NF : 1];
        if constexpr (KP <= 4) {
#pragma unroll
            for (int x = 0; x < NF; ++x) foldf[x] = (float)F.fold[x];
        }
        // Where the raw plane sums are small enough, the fold runs on them
        // directly (one reduction per output instead of one per accumulator):
        // a K-element adds at most k h^2 to a plane sum (2 h^2 with the split
        // sums of k = 2), and each output adds up at most 1 + (k-1)(p-1)
        // plane sums times a coefficient below p; all of it exact in FP32
        // below 2^23.
        const double kel = (double)T.ks * (F.fp8 ? 32 : 16);
        const double hh = (double)F.h * F.h;
        const bool direct = kel * hh * (KP == 2 ? 2 : KP) * (1.0 + (KP - 1) * (double)(F.p - 1)) < 8388608.0;
        // columns per tensor-memory read: 4 for k >= 4 (up to 15
        // accumulators, then their sums, live at once), else 8
        constexpr int CW = KP >= 5 ? 4 : 8;
        for (int c = c0; c < c0 + w; c += 8) {
            const bool active = rows_left > 0 && c < T.cols;   // the same for the whole warp
            uint32_t lo[KP], hi[KP];
#pragma unroll
            for (int i = 0; i < KP; ++i) lo[i] = hi[i] = 0;
#pragma unroll
            for (int h = 0; h < 8 / CW; ++h) {
                const int cc = c + h * CW;
                // plane sums C_t of these columns (k = 2: C_1 = C_1a + C_1b),
                // each accumulator reduced first unless the fold is exact on
                // the raw sums
                float sum[2 * KP - 1][CW];
                {
                    uint32_t v[NACC][CW];
#pragma unroll
                    for (int a = 0; a < NACC; ++a) tmem_ld_cols<CW>(tacc + a * BN + cc, v[a]);
                    ptx::tmem_wait_ld();
#pragma unroll
                    for (int a = 0; a < NACC; ++a) tmem_zero_cols<CW>(tacc + a * BN + cc);
                    if (h + 1 == 8 / CW && c + 8 >= c0 + w) release();
#pragma unroll
                    for (int a = 0; a < NACC; ++a) {
                        const int t = KP == 2 ? (a / 2) + (a % 2) : a;
#pragma unroll
                        for (int e = 0; e < CW; ++e) {
                            const float x = __uint_as_float(v[a][e]);
                            const float y = direct ? x : fmaf(-pf, rintf(x * inv_pf), x);
                            if (KP == 2 && a == 2) sum[t][e] += y;
                            else sum[t][e] = y;
                        }
                    }
                }
                if (!active) continue;
#pragma unroll
                for (int i = 0; i < KP; ++i) {
#pragma unroll
                    for (int e = 0; e < CW; ++e) {
                        float o = sum[i][e];
#pragma unroll
                        for (int t = KP; t < 2 * KP - 1; ++t) {
                            const float fv = KP <= 4 ? foldf[(KP <= 4 ? (t - KP) * KP + i : 0)]
                                                     : (float)F.fold[(t - KP) * KP + i];
                            o = fmaf(sum[t][e], fv, o);
                        }
                        const uint32_t b = tc_mod(o, pf, inv_pf);
                        const int pos = h * CW + e;
                        if (pos < 4) lo[i] |= b << (8 * pos);
                        else hi[i] |= b << (8 * (pos - 4));
                    }
                }
            }
            if (!active) continue;
            const int cols_left = T.cols - c;
#pragma unroll
            for (int i = 0; i < KP; ++i)
                store_rows8(lane_base + (int64_t)i * c_plane + c, step4, rows_left, cols_left, lo[i],
                            hi[i], lane);
        }
    }
}

template <class Release>
__device__ __forceinline__ void tc_epilogue_k(uint32_t tacc, const TcRec &T, const BFieldParams &F,
                                           int row, int c0, int w, Release release) {
    // GF(2^k) (the parity path) and the other fields (FP32 reductions) are
    // separate functions, each with its own register allocation
    if (F.p == 2) {
        switch (T.k) {
            case 1: tc_epilogue<1, true>(tacc, T, F, row, c0, w, release); break;
            case 2: tc_epilogue<2, true>(tacc, T, F, row, c0, w, release); break;
            case 3: tc_epilogue<3, true>(tacc, T, F, row, c0, w, release); break;
            case 4: tc_epilogue<4, true>(tacc, T, F, row, c0, w, release); break;
            case 5: tc_epilogue<5, true>(tacc, T, F, row, c0, w, release); break;
            case 6: tc_epilogue<6, true>(tacc, T, F, row, c0, w, release); break;
            case 7: tc_epilogue<7, true>(tacc, T, F, row, c0, w, release); break;
            default: tc_epilogue<8, true>(tacc, T, F, row, c0, w, release); break;
        }
        return;
    }
    switch (T.k) {
        case 1: tc_epilogue<1, false>(tacc, T, F, row, c0, w, release); break;
        case 2: tc_epilogue<2, false>(tacc, T, F, row, c0, w, release); break;
        case 3: tc_epilogue<3, false>(tacc, T, F, row, c0, w, release); break;
        case 4: tc_epilogue<4, false>(tacc, T, F, row, c0, w, release); break;
        case 5: tc_epilogue<5, false>(tacc, T, F, row, c0, w, release); break;
        case 6: tc_epilogue<6, false>(tacc, T, F, row, c0, w, release); break;
        case 7: tc_epilogue<7, false>(tacc, T, F, row, c0, w, release); break;
        default: tc_epilogue<8, false>(tacc, T, F, row, c0, w, release); break;
    }
}

// K-blocks of a tile per ring stage: as many as one slot holds (the
// converted blocks of consecutive K-blocks are contiguous, so a stage is one
// bulk copy per operand: nkb A blocks, then nkb B blocks).
__device__ __forceinline__ int tc_stage_kblocks(int slot_bytes, uint32_t ab, uint32_t bb) {
    const int c = slot_bytes / (int)(ab + bb);
    return c > 1 ? c : 1;
}

// The K loop of one tile on the MMA thread: per K-block one MMA per A
// plane, A_i against [B_0; ...; B_{k-1}] into the accumulators at column
// a_col(i) of the buffer, which the epilogue zeroed after reading the tile
// before last (every MMA accumulates).  The ring position (s, round) and the
// drain count of the buffer advance here.
template <int KP, bool FP8>
__device__ __noinline__ bool tc_mma_tile(uint32_t d0, uint8_t *smem, int slot_bytes, int stages,
                                         int &s, uint32_t &round, int rows8, int ks_n, int chunk,
                                         uint64_t *full, uint64_t *empty, uint64_t *acc_full_b,
                                         uint64_t *acc_empty_b, int &drains,
                                         volatile int *abort_flag) {
    constexpr int BN = tc_bn(KP);
    const uint32_t idesc = FP8 ? ptx::idesc_e4m3_f32(128, KP * BN) : ptx::idesc_bf16_f32(128, KP * BN);
    const uint32_t ab = (uint32_t)(KP * rows8 * 32), bb = (uint32_t)(KP * BN * 32);
    const uint64_t astep = (uint64_t)((uint32_t)rows8 * 32) >> 4;   // descriptor units of 16 bytes
    const int cap = tc_stage_kblocks(slot_bytes, ab, bb);
    uint32_t sa = ptx::smem_addr(smem + (size_t)s * slot_bytes);
    const uint32_t slot_u = (uint32_t)slot_bytes;
    const uint32_t sa0 = ptx::smem_addr(smem);
    int to_drain = chunk;
    for (int kb = 0; kb < ks_n;) {
        const int nkb = ks_n - kb < cap ? ks_n - kb : cap;
        if (*abort_flag || !ptx::mbar_wait(&full[s], round & 1)) return false;
        ptx::tc_fence_after();
        const uint32_t sb = sa + (uint32_t)nkb * ab;
        for (int j = 0; j < nkb; ++j, ++kb) {
            const uint64_t ad = desc_kmajor(sa + (uint32_t)j * ab), bd = desc_kmajor(sb + (uint32_t)j * bb);
#pragma unroll
            for (int i = 0; i < KP; ++i) {
                const uint32_t col = KP <= 2 ? (uint32_t)(i * KP * BN) : (uint32_t)(i * BN);
                if constexpr (FP8) ptx::mma_e4m3(d0 + col, ad + i * astep, bd, idesc, 1u);
                else ptx::mma_bf16(d0 + col, ad + i * astep, bd, idesc, 1u);
            }
            if (--to_drain == 0 && kb + 1 < ks_n) {
                // an exact chunk ends inside or at the end of this stage: the
                // epilogue reduces in place before the next K-block's MMAs
                to_drain = chunk;
                ptx::mma_commit(acc_full_b);
                if (!ptx::mbar_wait(acc_empty_b, (uint32_t)drains & 1)) return false;
                ++drains;
                ptx::tc_fence_after();
            }
        }
        ptx::mma_commit(&empty[s]);
        if (++s == stages) {
            s = 0;
            ++round;
            sa = sa0;
        } else {
            sa += slot_u;
        }
    }
    return true;
}

// Called once the warp's last accumulator columns of the tile have been
// read (and zeroed, tmem_zero8): the zeros land, then the buffer goes back
// to the MMAs.  The tensor-memory waits are warp-collective, so after them
// one lane speaks for the warp (one arrival per warp: per-lane arrivals on
// one barrier serialise).
struct Releaser {
    uint64_t *bar;
    __device__ void operator()() const {
        ptx::tmem_wait_st();
        ptx::tc_fence_before();
        if ((threadIdx.x & 31) == 0) ptx::mbar_arrive(bar);
    }
};

__global__ void __launch_bounds__(kTcThreads, 1)
tc_products_kernel(const uint8_t *__restrict__ ws, int slot_bytes, int stages,
                   int *status) {
    const BHeader *hdr = reinterpret_cast<const BHeader *>(ws);
    const int ntiles = hdr->ntiles, nfields = hdr->nfields;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *full = (uint64_t *)(smem + (size_t)stages * slot_bytes);
    uint64_t *empty = full + kTcMaxStages;
    uint64_t *acc_full = empty + kTcMaxStages;   // [2] MMAs of a chunk / a tile completed
    uint64_t *acc_empty = acc_full + 2;          // [2] a drain finished
    uint64_t *tmem_free = acc_empty + 2;         // [2] a tile's accumulators were read out
    uint64_t *mma_done = tmem_free + 2;
    uint32_t *tmem_slot = (uint32_t *)(mma_done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    BFieldParams *sF = reinterpret_cast<BFieldParams *>(smem + (size_t)stages * slot_bytes + 256);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    {
        // the field parameters, copied once into shared memory
        const uint32_t *src = reinterpret_cast<const uint32_t *>(ws + hdr->fields_off);
        uint32_t *dst = reinterpret_cast<uint32_t *>(sF);
        const int words = nfields * (int)(sizeof(BFieldParams) / 4);
        for (int x = threadIdx.x; x < words; x += kTcThreads) dst[x] = src[x];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&acc_full[b], 1);
            ptx::mbar_init(&acc_empty[b], kTcEpiWarps / 2);   // one arrival per warp of a group
            ptx::mbar_init(&tmem_free[b], kTcEpiWarps / 2);
        }
        ptx::mbar_init(mma_done, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    auto slot_at = [&](int s) { return smem + (size_t)s * slot_bytes; };
    const int t0 = blockIdx.x, tstep = gridDim.x;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer ----------------
            // ring position kept as (stage, round): no division by the
            // run-time stage count on the per-K-block path
            int s = 0;
            uint32_t round = 0;
            int64_t it = 0;
            bool ok = true;
            TcRec T = tc_rec(ws, hdr, t0, ntiles);
            for (int t = t0; t < ntiles && ok; t += tstep) {
                const TcRec Tn = tc_rec(ws, hdr, t + tstep, ntiles);   // in flight meanwhile
                const uint32_t ab = (uint32_t)(T.k * T.rows8 * 32), bb = (uint32_t)(T.k * tc_bn(T.k) * 32);
                const int cap = tc_stage_kblocks(slot_bytes, ab, bb);
                const uint8_t *a0 = T.a;
                const uint8_t *b0 = T.b;
                for (int kb = 0; kb < T.ks; ++it) {
                    const int nkb = T.ks - kb < cap ? T.ks - kb : cap;
                    if (round > 0) {
                        if (*abort_flag || !ptx::mbar_wait(&empty[s], (round - 1) & 1)) {
                            ok = false;
                            break;
                        }
                    }
                    ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)nkb * (ab + bb));
                    bulk_copy_split(slot_at(s), a0 + (size_t)kb * ab, (uint32_t)nkb * ab, &full[s]);
                    bulk_copy_split(slot_at(s) + (size_t)nkb * ab, b0 + (size_t)kb * bb,
                                    (uint32_t)nkb * bb, &full[s]);
                    kb += nkb;
                    if (++s == stages) {
                        s = 0;
                        ++round;
                    }
                }
                T = Tn;
            }
            if (!ok) {
                *abort_flag = 1;
                for (int64_t j = (it > stages ? it - stages : 0); j < it; ++j)
                    ptx::mbar_wait(&full[j % stages], (uint32_t)(j / stages) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int s = 0;
            uint32_t round = 0;
            int tcount = 0, drains0 = 0, drains1 = 0;
            bool ok = true;
            TcRec T = tc_rec(ws, hdr, t0, ntiles);
            for (int t = t0; t < ntiles && ok; t += tstep, ++tcount) {
                const TcRec Tn = tc_rec(ws, hdr, t + tstep, ntiles);
                const int b = tcount & 1;
                // this buffer was zeroed: at the start, or after the epilogue
                // read out the tile before last
                if (*abort_flag ||
                    !ptx::mbar_wait(&tmem_free[b], (uint32_t)(tcount >> 1) & 1)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d0 = tmem_base + 256u * b;
                const bool fp8 = sF[T.field].fp8 != 0;
                const int chunk = sF[T.field].tc_chunk_ks;
                int &drains = b ? drains1 : drains0;
#define QADIC_TC_MMA(KP_)                                                                         \
    ok = fp8 ? tc_mma_tile<KP_, true>(d0, smem, slot_bytes, stages, s, round, T.rows8,                \
                                      T.ks, chunk, full, empty, &acc_full[b], &acc_empty[b],        \
                                      drains, abort_flag)                                           \
             : tc_mma_tile<KP_, false>(d0, smem, slot_bytes, stages, s, round, T.rows8,               \
                                       T.ks, chunk, full, empty, &acc_full[b], &acc_empty[b],       \
                                       drains, abort_flag)
                switch (T.k) {
                    case 1: QADIC_TC_MMA(1); break;
                    case 2: QADIC_TC_MMA(2); break;
                    case 3: QADIC_TC_MMA(3); break;
                    case 4: QADIC_TC_MMA(4); break;
                    case 5: QADIC_TC_MMA(5); break;
                    case 6: QADIC_TC_MMA(6); break;
                    case 7: QADIC_TC_MMA(7); break;
                    default: QADIC_TC_MMA(8); break;
                }
#undef QADIC_TC_MMA
                if (ok) ptx::mma_commit(&acc_full[b]);   // tile complete
                T = Tn;
            }
            if (!ok) {
                *abort_flag = 1;
                ptx::mma_commit(&acc_full[0]);   // wake the epilogue
                ptx::mma_commit(&acc_full[1]);
            }
            ptx::mma_commit(mma_done);
            if (!ptx::mbar_wait(mma_done, 0)) *abort_flag = 1;
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int ew = warp - 2;
        const int quarter = warp & 3, part = ew / 4;   // part: the group, and its buffer
        {
            // the group's buffer starts at zero: every MMA accumulates
            const uint32_t tz = tmem_base + ((uint32_t)(quarter * 32) << 16) + 256u * part;
            for (int c = 0; c < 256; c += 8) tmem_zero8(tz + c);
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            if (lane == 0) ptx::mbar_arrive(&tmem_free[part]);
        }
        int phase0 = 0, phase1 = 0;
        int tcount = part;
        bool ok = true;
        TcRec T = tc_rec(ws, hdr, t0 + part * tstep, ntiles);
        for (int t = t0 + part * tstep; t < ntiles && ok; t += 2 * tstep, tcount += 2) {
            const TcRec Tn = tc_rec(ws, hdr, t + 2 * tstep, ntiles);
            const int b = tcount & 1;
            const uint32_t tacc = tmem_base + 256u * b + ((uint32_t)(quarter * 32) << 16);
            const BFieldParams &F = sF[T.field];
            const int bn = tc_bn(T.k);
            const int w = bn, c0 = 0;
            const int nacc = T.k == 2 ? 4 : 2 * T.k - 1;
            const int ndrain = T.ndrain;
            auto ready = [&]() {
                const bool r = ptx::mbar_wait(&acc_full[b], (uint32_t)(b ? phase1 : phase0) & 1);
                if (b) ++phase1;
                else ++phase0;
                return r && !*abort_flag;
            };
            for (int d = 0; d < ndrain; ++d) {
                if (!ready()) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                tc_drain(tacc, nacc, bn, c0, w, F.pf, F.inv_pf);
                ptx::tc_fence_before();
                if (lane == 0) ptx::mbar_arrive(&acc_empty[b]);
            }
            if (!ok) break;
            if (!ready()) {
                ok = false;
                break;
            }
            ptx::tc_fence_after();
            tc_epilogue_k(tacc, T, F, quarter * 32, c0, w, Releaser{&tmem_free[b]});
            T = Tn;
        }
        if (!ok) *abort_flag = 1;
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) record_timeout(status, 7);
    if (warp == 1) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 512);
    }
}

}  // namespace

// Stage layout for the fields of a launch: every stage holds the A planes of
// the largest k (k x 128 rows x 32 bytes) and one B tile (k BN = 128 rows).
// Ring stages for the widest field degree present: three when a K-block of
// A takes 20 KB or more (k >= 5), else four; each slot as large as the
// budget allows (several K-blocks of the smaller degrees per stage), and at
// least one K-block of the widest degree.
int tc_stage_layout(uint32_t kmax, int *slot_bytes, int *stages) {
    const int one = (int)kmax * 4096 + 4096;
    const int reserve = 256 + kMaxFields * (int)sizeof(BFieldParams);
    const int s = kmax >= 5 ? 3 : 4;
    const int slot = (kTcSmemBudget - reserve - 128) / s / 256 * 256;
    if (slot < one) return set_error(QADIC_E_UNSUPPORTED, "batched tcgen05 stages do not fit");
    *slot_bytes = slot;
    *stages = s;
    return QADIC_OK;
}

// Dynamic shared memory of a launch: the stages and the barriers, and at
// least half of the SM's shared memory, so that no two CTAs share an SM
// (each allocates all 512 tensor-memory columns).
size_t tc_smem_bytes(int slot_bytes, int stages) {
    const size_t need = 128 + (size_t)stages * slot_bytes + 256 + kMaxFields * sizeof(BFieldParams);
    return std::max<size_t>(need, kTcSmemBudget / 2 + 1024);
}

int prepare_tc_kernel() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(tc_products_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kTcSmemBudget);
    });
    if (err != cudaSuccess)
        return set_error(QADIC_E_CUDA, "batched tcgen05 smem attribute: %s", cudaGetErrorString(err));
    return QADIC_OK;
}

int64_t tc_grid(int64_t ntiles) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max<int64_t>(1, std::min<int64_t>(ntiles, std::max(sms, 1)));
}

int launch_tc_convert(const uint8_t *ws, int64_t nitems, cudaStream_t stream) {
    if (nitems <= 0) return QADIC_OK;
    tc_convert_kernel<<<(unsigned)nitems, kTcConvThreads, 0, stream>>>(ws);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "tc convert launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

int launch_tc_products(const uint8_t *ws, int64_t grid, int slot_bytes, int stages,
                       int *status, cudaStream_t stream) {
    tc_products_kernel<<<(unsigned)grid, kTcThreads, tc_smem_bytes(slot_bytes, stages), stream>>>(
        ws, slot_bytes, stages, status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "tc products launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace bt
}  // namespace qadic
