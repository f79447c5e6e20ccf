// Many independent GF(p^k) products in one persistent launch.
//
// Each product C = A B is the coefficient-plane form of Eq. 1: 2k-1 plane
// sums C_t = sum_{i+j=t} A_i B_j, reduced mod p and folded mod P with
// X^t mod P.  The host lays a work list into the caller's workspace: field
// parameters, product descriptors and one entry per output tile, sorted by
// field and decreasing work, so thousands of uneven products (m, n, K in
// [16, 256], several fields) share one launch.  Two kernels run it:
//
//   * with room in the workspace for converted operands, the tensor-core
//     path of k_batched_tc.cu: one conversion launch, then a persistent
//     tcgen05 kernel over 128-row tiles (fp8 or bf16 operands, FP32
//     accumulators in tensor memory);
//   * with the work list alone (and in the allocation-free entry point), the
//     register-staged kernel below: uint8 coefficient tiles staged in shared
//     memory as centred bf16 (exact small integers), multiplied with
//     warp-level mma.sync (m16n8k16, bf16 -> f32), accumulated exactly in
//     FP32 registers (at each exact chunk the accumulators are reduced mod p
//     in place), then reduced mod p, folded and written as uint8 planes; a
//     grid of (SMs x resident blocks) CTAs pulls tiles with one atomicAdd each.
//
// The register-staged kernel's tile shape (BM x BN) and K-block size BK are
// picked per k from a short list of candidates whose 2k-1 accumulator sets
// fit in registers: index 0 by default, or whichever qadic_batched_autotune
// measured fastest on the caller's own batch (qadic_batched_select_tiles
// sets one by hand).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "batched_tile.cuh"

namespace qadic {

namespace {

using namespace bt;

// 16 consecutive bytes of a row starting at `src` (any alignment); only the
// first `valid` (<= 16) are read, the others are zero.  In the full case the
// bytes come from aligned 32-bit loads joined by funnel shifts; every word
// loaded holds at least one of the 16 bytes, so no load leaves the buffer.
__device__ __forceinline__ void load16(const uint8_t *src, int valid, uint32_t (&w)[4]) {
    if (valid >= 16) {
        const uint32_t a = (uint32_t)((uintptr_t)src & 3);
        const uint32_t *base = reinterpret_cast<const uint32_t *>(src - a);
        if (a == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = __ldg(base + i);
        } else {
            uint32_t x[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) x[i] = __ldg(base + i);
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = __funnelshift_r(x[i], x[i + 1], 8 * a);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = 0;
        for (int b = 0; b < valid; ++b) w[b >> 2] |= (uint32_t)__ldg(src + b) << (8 * (b & 3));
    }
}

// Tile staging: chunks of 16 coefficients (one row segment of one plane).
template <int KP, typename T>
struct Stager {
    static constexpr int BK = T::BK;
    static constexpr int A_CH = KP * T::BM * (BK / 16);
    static constexpr int B_CH = KP * BK * (T::BN / 16);
    static constexpr int PER_THREAD = (A_CH + B_CH + kThreads - 1) / kThreads;

    uint32_t raw[PER_THREAD][4];

    __device__ __forceinline__ void load(const BProd &P, int row0, int col0, int k0) {
#pragma unroll
        for (int s = 0; s < PER_THREAD; ++s) {
            const int c = threadIdx.x + s * kThreads;
            if (c < A_CH) {
                const int part = c % (BK / 16), r = (c / (BK / 16)) % T::BM,
                          i = c / ((BK / 16) * T::BM);
                const int gr = row0 + r, gk = k0 + part * 16;
                const int valid = gr < P.m ? min(16, max(0, P.K - gk)) : 0;
                load16(P.A + ((int64_t)i * P.m + gr) * P.lda + gk, valid, raw[s]);
            } else if (c < A_CH + B_CH) {
                const int cb = c - A_CH;
                const int part = cb % (T::BN / 16), r = (cb / (T::BN / 16)) % BK,
                          j = cb / ((T::BN / 16) * BK);
                const int gk = k0 + r, gc = col0 + part * 16;
                const int valid = gk < P.K ? min(16, max(0, P.n - gc)) : 0;
                load16(P.B + ((int64_t)j * P.K + gk) * P.ldb + gc, valid, raw[s]);
            }
        }
    }

    // bytes -> centred bf16 through the 256-entry table, 32-byte stores
    __device__ __forceinline__ void store(uint16_t *As, uint16_t *Bs, const uint16_t *tab) const {
#pragma unroll
        for (int s = 0; s < PER_THREAD; ++s) {
            const int c = threadIdx.x + s * kThreads;
            uint32_t o[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t w = raw[s][q];
                o[2 * q] = (uint32_t)tab[w & 0xff] | ((uint32_t)tab[(w >> 8) & 0xff] << 16);
                o[2 * q + 1] = (uint32_t)tab[(w >> 16) & 0xff] | ((uint32_t)tab[w >> 24] << 16);
            }
            uint16_t *dst = nullptr;
            if (c < A_CH) {
                const int part = c % (BK / 16), r = (c / (BK / 16)) % T::BM,
                          i = c / ((BK / 16) * T::BM);
                dst = As + (i * T::BM + r) * T::LDA + part * 16;
            } else if (c < A_CH + B_CH) {
                const int cb = c - A_CH;
                const int part = cb % (T::BN / 16), r = (cb / (T::BN / 16)) % BK,
                          j = cb / ((T::BN / 16) * BK);
                dst = Bs + (j * BK + r) * T::LDB + part * 16;
            }
            if (dst) {
                uint4 *d4 = reinterpret_cast<uint4 *>(dst);
                d4[0] = make_uint4(o[0], o[1], o[2], o[3]);
                d4[1] = make_uint4(o[4], o[5], o[6], o[7]);
            }
        }
    }
};

template <int KP, int BM, int BN, int BK>
__device__ __forceinline__ void run_tile(const BProd &P, const BFieldParams &F, int tm, int tn,
                                      uint8_t *smem, const uint16_t *tab) {
    using T = TileCfg<KP, BM, BN, BK>;
    uint16_t *As = reinterpret_cast<uint16_t *>(smem);   // [KP][BM][LDA]
    uint16_t *Bs = As + KP * T::BM * T::LDA;             // [KP][BK][LDB]
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int wm = warp / 2, wn = warp % 2;
    const int row0 = tm * T::BM, col0 = tn * T::BN;

    AccArray<T> acc;
    acc_zero<T>(acc);
    const int nkb = (P.K + BK - 1) / BK;
    const int chunk_blocks = max(1, F.chunk_k / BK);
    Stager<KP, T> stage;
    stage.load(P, row0, col0, 0);
    for (int kb = 0; kb < nkb; ++kb) {
        __syncthreads();   // previous tile/step finished reading shared memory
        stage.store(As, Bs, tab);
        __syncthreads();
        if (kb + 1 < nkb) stage.load(P, row0, col0, (kb + 1) * BK);   // in flight during the MMAs
#pragma unroll 1
        for (int ks = 0; ks < BK / 16; ++ks) tile_mma_step<KP, T>(acc, As, Bs, ks, wm, wn, lane);
        if ((kb + 1) % chunk_blocks == 0 && kb + 1 < nkb) tile_chunk_reduce<T>(acc, F);
    }
    tile_epilogue<KP, T>(acc, P, F, row0, col0, wm, wn, lane);
}

// Not inlined: each k is register-allocated on its own (its configurations
// are branches of one function) instead of inside one kernel body holding
// all eight.
template <int KP>
__device__ __noinline__ void run_tile_cfg(int cfg, const BProd &P, const BFieldParams &F, int tm,
                                             int tn, uint8_t *smem, const uint16_t *tab) {
    constexpr bool kSmall = KP <= 2, kMid = KP > 2 && KP <= 4;
    constexpr TileShape c0 = kSmall ? kShapesK2[0] : kMid ? kShapesK4[0] : kShapesK8[0];
    constexpr TileShape c1 = kSmall ? kShapesK2[1] : kMid ? kShapesK4[1] : kShapesK8[1];
    constexpr TileShape c2 = kSmall ? kShapesK2[2] : kMid ? kShapesK4[2] : kShapesK8[2];
    constexpr TileShape c3 = kSmall ? kShapesK2[3] : kMid ? kShapesK4[3] : kShapesK8[3];
    constexpr TileShape c4 = kSmall ? kShapesK2[4] : kMid ? kShapesK4[4] : kShapesK8[4];
    switch (cfg) {
        case 1: run_tile<KP, c1.bm, c1.bn, c1.bk>(P, F, tm, tn, smem, tab); break;
        case 2: run_tile<KP, c2.bm, c2.bn, c2.bk>(P, F, tm, tn, smem, tab); break;
        case 3: run_tile<KP, c3.bm, c3.bn, c3.bk>(P, F, tm, tn, smem, tab); break;
        case 4:
            if constexpr (num_cfgs(KP) > 4) {
                run_tile<KP, c4.bm, c4.bn, c4.bk>(P, F, tm, tn, smem, tab);
                break;
            }
            [[fallthrough]];
        default: run_tile<KP, c0.bm, c0.bn, c0.bk>(P, F, tm, tn, smem, tab); break;
    }
}

__global__ void __launch_bounds__(kThreads, 5) batched_kernel(uint8_t *ws) {
    extern __shared__ __align__(16) uint8_t smem[];   // sized for the largest tile in the list
    __shared__ uint16_t tab[256];   // input byte -> centred bf16 bits, for field s_field
    __shared__ int s_tile, s_field;
    BHeader *hdr = reinterpret_cast<BHeader *>(ws);
    const BFieldParams *fields = reinterpret_cast<const BFieldParams *>(ws + hdr->fields_off);
    const BProd *prods = reinterpret_cast<const BProd *>(ws + hdr->prods_off);
    const BTile *tiles = reinterpret_cast<const BTile *>(ws + hdr->tiles_off);
    const int ntiles = hdr->ntiles;
    if (threadIdx.x == 0) s_field = -1;
    while (true) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&hdr->counter, 1u);
        __syncthreads();
        const int t = s_tile;
        const int cur_field = s_field;
        __syncthreads();
        if (t >= ntiles) break;
        const BTile tile = tiles[t];
        // descriptors stay in global memory (read-only, L1-cached) and are
        // read where used instead of being copied into registers
        const BProd &P = prods[tile.prod];
        const BFieldParams &F = fields[P.field];
        if (P.field != cur_field) {   // block-uniform
            for (int b = threadIdx.x; b < 256; b += kThreads)
                tab[b] = bf16_bits((uint32_t)b, F);
            if (threadIdx.x == 0) s_field = P.field;
            // run_tile's first __syncthreads orders these writes before any use
        }
        switch (F.k) {
            case 1: run_tile_cfg<1>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            case 2: run_tile_cfg<2>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            case 3: run_tile_cfg<3>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            case 4: run_tile_cfg<4>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            case 5: run_tile_cfg<5>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            case 6: run_tile_cfg<6>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            case 7: run_tile_cfg<7>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
            default: run_tile_cfg<8>(P.cfg, P, F, tile.tm, tile.tn, smem, tab); break;
        }
    }
}

// Selected configuration per k (process-wide: every device runs the same
// kernel), -1 = default.
std::mutex g_tiles_mu;
int g_tile_choice[kMaxK + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};

int tile_choice(uint32_t k) {
    std::lock_guard<std::mutex> lock(g_tiles_mu);
    const int c = (k <= kMaxK) ? g_tile_choice[k] : -1;
    return c < 0 ? 0 : c;
}

void field_params(const Field &f, BFieldParams &F) {
    F.p = f.p;
    F.k = f.k;
    F.h = f.h;
    F.m32 = make_mod_small(f.p);
    F.pf = (float)f.p;
    F.inv_pf = 1.0f / (float)f.p;
    F.chunk_k = (int32_t)std::min<int64_t>(f.k_chunk_f32, 1 << 30);
    // Tensor-core path: p <= 31 runs on fp8 e4m3 operands (exact for
    // |centred| <= 15), the rest on bf16.
    F.fp8 = fp8_field(f.p);
    // Tensor-core path: FP32 accumulators exact while |sum| <= 2^24; a drained
    // residue is below 2p and a K element adds at most h^2 to an accumulator
    // of k = 1 or of the split k = 2 layout, k h^2 with shared accumulators
    // (p = 2: the planes hold 0 and 1, h = 1).
    {
        const int64_t hh = (int64_t)f.h * f.h;
        const int64_t growth = (f.k <= 2 ? 1 : (int64_t)f.k) * hh;
        const int64_t elems = ((1ll << 24) - 2 * (int64_t)f.p) / growth;
        F.tc_chunk_ks = (int32_t)std::min<int64_t>(elems / (F.fp8 ? 32 : 16), 1 << 30);
    }
    for (uint32_t t = 0; t + 1 < f.k; ++t) {
        F.fold2[t] = 0;
        for (uint32_t c = 0; c < f.k; ++c) {
            F.fold[t * f.k + c] = f.fold[t * f.k + c];
            F.fold2[t] |= (uint8_t)((f.fold[t * f.k + c] & 1u) << c);
        }
    }
}

int field_cfg(const Field &f) {
    const int c = tile_choice(f.k);
    return f.k_chunk_f32 >= tile_shape_of(f.k, c).bk ? c : 0;
}

uint64_t tile_cost(const qadic_gemm_desc &d, uint32_t k, int cfg) {
    const TileShape t = tile_shape_of(k, cfg);
    return (uint64_t)t.bm * t.bn * (uint64_t)(((d.K + t.bk - 1) / t.bk) * t.bk) * k * k;
}

// Opt the kernel in to the largest dynamic shared memory any candidate needs.
int prepare_kernel(size_t smem) {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        size_t most = 0;
        for (uint32_t k = 1; k <= kMaxK; ++k)
            for (int c = 0; c < num_cfgs(k); ++c) most = std::max(most, tile_smem_bytes(k, c));
        err = cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)most);
    });
    (void)smem;
    if (err != cudaSuccess)
        return set_error(QADIC_E_CUDA, "batched smem attribute: %s", cudaGetErrorString(err));
    return QADIC_OK;
}

int64_t grid_for(int dev, size_t smem, int64_t ntiles) {
    (void)dev;
    int64_t grid = resident_blocks(batched_kernel, kThreads, smem);
    if (ntiles < grid) grid = std::max<int64_t>(1, ntiles);
    return grid;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t fields_off, prods_off, tiles_off, order_off, conv_off, total;
};

// Work list (header, fields, products, tiles), then, for the converted-
// operand kernels, conv_bytes of 16-bit operands.
Layout layout_for(int64_t count, int64_t ntiles, size_t conv_bytes = 0, int64_t conv_items = 0,
                  size_t tile_bytes = sizeof(BTile)) {
    Layout L;
    L.fields_off = kHeaderBytes;
    L.prods_off = align_up(L.fields_off + kMaxFields * sizeof(BFieldParams), 256);
    L.tiles_off = align_up(L.prods_off + count * sizeof(BProd), 256);
    L.order_off = align_up(L.tiles_off + ntiles * tile_bytes, 256);
    L.conv_off = align_up(L.order_off + conv_items * sizeof(ConvItem), 256);
    L.total = L.conv_off + conv_bytes;
    return L;
}

int32_t round8(int32_t x) { return (x + 7) / 8 * 8; }
int32_t round16(int32_t x) { return (x + 15) / 16 * 16; }

// The tensor-core path's converted operands (k_batched_tc.cu): per product,
// 32-byte K-blocks (32 fp8 or 16 bf16 elements); A as k planes of 128-row
// tiles (rows rounded up to 8), B^T as k planes of BN-column tiles, each
// operand starting on a 256-byte boundary.
int32_t tc_kblocks(const qadic_gemm_desc &d, const Field &f) {
    const int32_t e = fp8_field(f.p) ? 32 : 16;
    return (d.K + e - 1) / e;
}
size_t tc_a_bytes(const qadic_gemm_desc &d, const Field &f) {
    return (size_t)f.k * round8(d.m) * 32 * tc_kblocks(d, f);
}
size_t tc_b_bytes(const qadic_gemm_desc &d, const Field &f) {
    const int32_t bn = tc_bn(f.k);
    return (size_t)f.k * bn * 32 * tc_kblocks(d, f) * ((d.n + bn - 1) / bn);
}
size_t conv_bytes_of(const qadic_gemm_desc &d, const Field &f) {
    return align_up(tc_a_bytes(d, f), 256) + align_up(tc_b_bytes(d, f), 256);
}

// 16-byte output chunks the conversion writes for product d's operands (A:
// all of its blocks; B: the valid columns only) and the items they make.
uint64_t chunks_a(const qadic_gemm_desc &d, const Field &f) { return tc_a_bytes(d, f) / 16; }
uint64_t chunks_b(const qadic_gemm_desc &d, const Field &f) {
    return (uint64_t)f.k * tc_kblocks(d, f) * 2 * d.n;
}
int64_t tc_tiles_of(const qadic_gemm_desc &d, const Field &f) {
    const int32_t bn = tc_bn(f.k);
    return (int64_t)((d.m + 127) / 128) * ((d.n + bn - 1) / bn);
}
int64_t conv_items_of(const qadic_gemm_desc &d, const Field &f) {
    return (int64_t)((chunks_a(d, f) + kConvItemChunks - 1) / kConvItemChunks +
                     (chunks_b(d, f) + kConvItemChunks - 1) / kConvItemChunks);
}

// The work queue's tile counter and tile count are 32-bit signed integers,
// and so are the byte offsets of the list's sections (below 2^31 with
// 8-byte tiles and at most 2^24 products).
constexpr int64_t kMaxQueueTiles = (int64_t)1 << 27;

int64_t max_tiles(const qadic_gemm_desc *descs, int64_t count) {
    int64_t t = 0;
    for (int64_t i = 0; i < count; ++i)
        t += (int64_t)((descs[i].m + 31) / 32) * ((descs[i].n + 15) / 16);   // smallest tile 32 x 16
    return t;
}

// Cached CUDA graphs of {counter reset, [operand conversion,] persistent
// kernel}, keyed by the call's exact arguments (descriptors, field ids,
// workspace, stream, tile configurations, path).  A graph replays whatever work list its workspace holds,
// so each entry keeps the list it was built with, and a hit re-uploads it
// when another list was written to the same workspace in between.
struct GraphEntry {
    std::vector<uint8_t> key;
    cudaGraphExec_t exec;
    std::vector<uint8_t> list;   // the uploaded bytes of the work list
    uint64_t id;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
constexpr size_t kMaxGraphs = 32;
uint64_t g_next_list_id = 1;
std::map<void *, uint64_t> g_ws_list;   // workspace -> id of the list it holds

// One non-blocking stream per device, used only to capture graphs.
cudaStream_t capture_stream(int dev) {
    static std::mutex mu;
    static cudaStream_t streams[64] = {nullptr};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

}  // namespace

size_t batched_workspace_size(const qadic_gemm_desc *descs, int64_t count) {
    if (!descs || count <= 0) return 0;
    return layout_for(count, max_tiles(descs, count)).total;
}

size_t batched_workspace_size_fields(const Field *const *fields, int32_t nfields,
                                     const qadic_gemm_desc *descs, int64_t count) {
    if (!descs || !fields || count <= 0 || nfields < 1) return 0;
    size_t conv = 0;
    int64_t items = 0, tc_tiles = 0;
    for (int64_t i = 0; i < count; ++i) {
        const qadic_gemm_desc &d = descs[i];
        if (d.field < 0 || d.field >= nfields || !fields[d.field] || d.m < 1 || d.n < 1 || d.K < 1)
            return 0;
        conv += conv_bytes_of(d, *fields[d.field]);
        items += conv_items_of(d, *fields[d.field]);
        tc_tiles += tc_tiles_of(d, *fields[d.field]);
    }
    return layout_for(count, tc_tiles, conv, items, sizeof(TcRec)).total;
}

int launch_batched(const Field *const *fields, int32_t nfields, const qadic_gemm_desc *descs,
                   int64_t count, void *workspace, size_t ws_bytes, bool use_graph,
                   cudaStream_t stream) {
    if (nfields < 1 || nfields > kMaxFields)
        return set_error(QADIC_E_INVALID, "nfields must be in [1, %d]", kMaxFields);
    if (count > (1 << 24)) return set_error(QADIC_E_INVALID, "too many products");
    int dev = -1;
    cudaGetDevice(&dev);
    for (int32_t i = 0; i < nfields; ++i) {
        if (!fields[i]) return set_error(QADIC_E_INVALID, "field %d is NULL", i);
        if (fields[i]->device != dev)
            return set_error(QADIC_E_INVALID, "field %d lives on another device", i);
    }
    for (int64_t i = 0; i < count; ++i) {
        const qadic_gemm_desc &d = descs[i];
        if (d.field < 0 || d.field >= nfields)
            return set_error(QADIC_E_INVALID, "desc %lld: field index out of range", (long long)i);
        if (d.m < 1 || d.n < 1 || d.K < 1 || d.m > 4096 || d.n > 4096 || d.K > 4096)
            return set_error(QADIC_E_INVALID, "desc %lld: sizes must be in [1, 4096]", (long long)i);
        if (!d.A || !d.B || !d.C) return set_error(QADIC_E_INVALID, "desc %lld: NULL", (long long)i);
        if (d.lda < d.K || d.ldb < d.n || d.ldc < d.n)
            return set_error(QADIC_E_INVALID, "desc %lld: leading dimension too small",
                             (long long)i);
        const Field &f = *fields[d.field];
        if (f.k_chunk_f32 < kMinBK)
            return set_error(QADIC_E_OVERFLOW, "exact FP32 chunk below one K-block (p=%u k=%u)",
                             f.p, f.k);
    }
    const int64_t tile_bound = max_tiles(descs, count);
    if (tile_bound > kMaxQueueTiles)
        return set_error(QADIC_E_INVALID,
                         "the batch has up to %lld output tiles; the work queue indexes at most %lld",
                         (long long)tile_bound, (long long)kMaxQueueTiles);
    size_t conv = 0;
    int64_t conv_items = 0, tc_tiles = 0;
    for (int64_t i = 0; i < count; ++i) {
        conv += conv_bytes_of(descs[i], *fields[descs[i].field]);
        conv_items += conv_items_of(descs[i], *fields[descs[i].field]);
        tc_tiles += tc_tiles_of(descs[i], *fields[descs[i].field]);
    }
    // converted operands when the workspace holds them, else bytes staged through registers
    const Layout L_conv = layout_for(count, tc_tiles, conv, conv_items, sizeof(TcRec));
    const Layout L_list = layout_for(count, tile_bound);
    if (!workspace || ws_bytes < L_list.total)
        return set_error(QADIC_E_NOMEM, "workspace %zu < %zu bytes", ws_bytes, L_list.total);
    if (((uintptr_t)workspace) & 255) return set_error(QADIC_E_INVALID, "workspace must be 256-byte aligned");
    const bool converted = ws_bytes >= L_conv.total;
    const Layout L = converted ? L_conv : L_list;
    int cfgs[kMaxFields];
    size_t smem = 0;
    uint32_t kmax = 1;
    for (int32_t i = 0; i < nfields; ++i) {
        cfgs[i] = field_cfg(*fields[i]);
        smem = std::max(smem, tile_smem_bytes(fields[i]->k, cfgs[i]));
    }
    for (int64_t i = 0; i < count; ++i) kmax = std::max(kmax, fields[descs[i].field]->k);
    int tc_slot = 0, tc_stages = 0;
    int st = QADIC_OK;
    if (converted) {
        if ((st = tc_stage_layout(kmax, &tc_slot, &tc_stages)) != QADIC_OK) return st;
        st = prepare_tc_kernel();
    } else {
        st = prepare_kernel(smem);
    }
    if (st != QADIC_OK) return st;

    // graph cache lookup
    std::vector<uint8_t> key;
    if (use_graph) {
        key.resize(sizeof(int64_t) + count * sizeof(qadic_gemm_desc) + nfields * sizeof(uint64_t) +
                   2 * sizeof(void *) + nfields * sizeof(int) + 1);
        uint8_t *kp = key.data();
        *kp++ = converted ? 1 : 0;
        std::memcpy(kp, &count, sizeof(int64_t));
        kp += sizeof(int64_t);
        std::memcpy(kp, descs, count * sizeof(qadic_gemm_desc));
        kp += count * sizeof(qadic_gemm_desc);
        // fields by their never-reused ids: a destroyed field's address may
        // come back for another field, whose graph must not be replayed
        for (int32_t i = 0; i < nfields; ++i) {
            std::memcpy(kp, &fields[i]->uid, sizeof(uint64_t));
            kp += sizeof(uint64_t);
        }
        std::memcpy(kp, &workspace, sizeof(void *));
        kp += sizeof(void *);
        std::memcpy(kp, &stream, sizeof(void *));
        kp += sizeof(void *);
        std::memcpy(kp, cfgs, nfields * sizeof(int));   // the tile configurations in use
        std::lock_guard<std::mutex> lock(g_graph_mu);
        for (auto &g : g_graphs)
            if (g.key == key) {
                auto it = g_ws_list.find(workspace);
                if (it == g_ws_list.end() || it->second != g.id) {
                    if (cudaMemcpyAsync(workspace, g.list.data(), g.list.size(),
                                        cudaMemcpyHostToDevice, stream) != cudaSuccess)
                        return set_error(QADIC_E_CUDA, "work list upload: %s",
                                         cudaGetErrorString(cudaGetLastError()));
                    g_ws_list[workspace] = g.id;
                }
                if (cudaGraphLaunch(g.exec, stream) != cudaSuccess)
                    return set_error(QADIC_E_CUDA, "graph launch: %s",
                                     cudaGetErrorString(cudaGetLastError()));
                return QADIC_OK;
            }
    }

    // host-built work list
    std::vector<uint8_t> host(L.conv_off, 0);
    std::vector<BTile> tiles;
    std::vector<uint64_t> cost;
    tiles.reserve(tile_bound);
    BFieldParams *fp = reinterpret_cast<BFieldParams *>(host.data() + L.fields_off);
    for (int32_t i = 0; i < nfields; ++i) field_params(*fields[i], fp[i]);
    BProd *pp = reinterpret_cast<BProd *>(host.data() + L.prods_off);
    size_t conv_at = L.conv_off;
    for (int64_t i = 0; i < count; ++i) {
        const qadic_gemm_desc &d = descs[i];
        BProd &P = pp[i];
        P.A = d.A;
        P.B = d.B;
        P.C = d.C;
        P.m = d.m;
        P.n = d.n;
        P.K = d.K;
        P.lda = d.lda;
        P.ldb = d.ldb;
        P.ldc = d.ldc;
        P.field = d.field;
        P.cfg = cfgs[d.field];
        const uint32_t k = fields[d.field]->k;
        TileShape ts = tile_shape_of(k, P.cfg);
        uint64_t c = tile_cost(d, k, P.cfg);
        if (converted) {
            // tensor-core path: kp = 32-byte K-blocks; A16 / B16 = the
            // operands in the blocked layout of k_batched_tc.cu
            const Field &f = *fields[d.field];
            P.kp = tc_kblocks(d, f);
            P.np = tc_bn(k);
            P.A16 = reinterpret_cast<const uint16_t *>((uint8_t *)workspace + conv_at);
            conv_at += align_up(tc_a_bytes(d, f), 256);
            P.B16 = reinterpret_cast<const uint16_t *>((uint8_t *)workspace + conv_at);
            conv_at += align_up(tc_b_bytes(d, f), 256);
            ts = TileShape{128, tc_bn(k), 32};
            c = (uint64_t)k * k * 128 * tc_bn(k) * 32 * P.kp;   // MMA work of a tile
        }
        for (int tm = 0; tm * ts.bm < d.m; ++tm)
            for (int tn = 0; tn * ts.bn < d.n; ++tn) {
                tiles.push_back(BTile{(int32_t)i, (int16_t)tm, (int16_t)tn});
                cost.push_back(c);
            }
    }
    // Tiles field by field (the field with the most work first), decreasing
    // cost within a field: all SMs then run one field's code at a time
    // (tiles of different fields interleaved kept the instruction cache
    // missing), and the cheapest tiles of the smallest field fill the end.
    std::vector<double> field_work(nfields, 0.0);
    for (size_t i = 0; i < tiles.size(); ++i) field_work[pp[tiles[i].prod].field] += (double)cost[i];
    std::vector<int> field_rank(nfields);
    {
        std::vector<int> fo(nfields);
        for (int32_t i = 0; i < nfields; ++i) fo[i] = i;
        std::stable_sort(fo.begin(), fo.end(), [&](int a, int b) { return field_work[a] > field_work[b]; });
        for (int32_t r = 0; r < nfields; ++r) field_rank[fo[r]] = r;
    }
    std::vector<int64_t> order(tiles.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int64_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const int fa = field_rank[pp[tiles[a].prod].field], fb = field_rank[pp[tiles[b].prod].field];
        if (fa != fb) return fa < fb;
        return cost[a] > cost[b];
    });
    if (converted) {
        TcRec *rp = reinterpret_cast<TcRec *>(host.data() + L.tiles_off);
        int32_t chunk_ks[kMaxFields];
        for (int32_t i = 0; i < nfields; ++i) chunk_ks[i] = fp[i].tc_chunk_ks;
        for (size_t i = 0; i < order.size(); ++i) {
            const BTile &t = tiles[order[i]];
            const BProd &P = pp[t.prod];
            const uint32_t k = fields[P.field]->k;
            const int32_t bn = tc_bn(k);
            const int32_t rows = std::min(128, P.m - 128 * t.tm);
            TcRec r;
            r.a = reinterpret_cast<const uint8_t *>(P.A16) + (size_t)t.tm * P.kp * k * 4096;
            r.b = reinterpret_cast<const uint8_t *>(P.B16) + (size_t)t.tn * P.kp * k * bn * 32;
            r.c = P.C + (int64_t)t.tm * 128 * P.ldc + (int64_t)t.tn * bn;
            r.c_plane = (int64_t)P.m * P.ldc;
            r.ldc = P.ldc;
            r.rows = (int16_t)rows;
            r.cols = (int16_t)std::min(bn, P.n - bn * t.tn);
            r.ks = (int16_t)P.kp;
            r.rows8 = (int16_t)((rows + 7) / 8 * 8);
            r.ndrain = (int16_t)((P.kp - 1) / chunk_ks[P.field]);
            r.field = (uint8_t)P.field;
            r.k = (uint8_t)k;
            rp[i] = r;
        }
    } else {
        BTile *tp = reinterpret_cast<BTile *>(host.data() + L.tiles_off);
        for (size_t i = 0; i < order.size(); ++i) tp[i] = tiles[order[i]];
    }
    BHeader *hdr = reinterpret_cast<BHeader *>(host.data());
    hdr->counter = 0;
    hdr->ntiles = (int32_t)tiles.size();
    hdr->nprod = (int32_t)count;
    hdr->nfields = nfields;
    hdr->fields_off = (uint32_t)L.fields_off;
    hdr->prods_off = (uint32_t)L.prods_off;
    hdr->tiles_off = (uint32_t)L.tiles_off;
    hdr->order_off = (uint32_t)L.order_off;
    size_t used = L.tiles_off + tiles.size() * (converted ? sizeof(TcRec) : sizeof(BTile));
    if (converted) {
        // conversion items of at most kConvItemChunks chunks, by decreasing size
        std::vector<ConvItem> items;
        std::vector<uint32_t> size;
        items.reserve(conv_items);
        size.reserve(conv_items);
        for (int64_t i = 0; i < count; ++i) {
            const Field &fi = *fields[descs[i].field];
            const uint64_t n_ops[2] = {chunks_a(descs[i], fi), chunks_b(descs[i], fi)};
            for (int op = 0; op < 2; ++op)
                for (uint64_t b = 0; b < n_ops[op]; b += kConvItemChunks) {
                    items.push_back(ConvItem{(uint32_t)(2 * i + op), (uint32_t)b});
                    size.push_back((uint32_t)std::min<uint64_t>(kConvItemChunks, n_ops[op] - b));
                }
        }
        std::vector<int64_t> ord(items.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int64_t)i;
        std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return size[a] > size[b]; });
        ConvItem *ip = reinterpret_cast<ConvItem *>(host.data() + L.order_off);
        for (size_t i = 0; i < ord.size(); ++i) ip[i] = items[ord[i]];
        hdr->nconv = (uint32_t)items.size();
        used = L.order_off + items.size() * sizeof(ConvItem);
    }
    if (cudaMemcpyAsync(workspace, host.data(), used, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "work list upload: %s", cudaGetErrorString(cudaGetLastError()));
    {
        std::lock_guard<std::mutex> lock(g_graph_mu);
        g_ws_list[workspace] = 0;   // an uncached list: no cached graph owns this workspace
    }

    const int64_t grid = converted ? tc_grid((int64_t)tiles.size())
                                   : grid_for(dev, smem, (int64_t)tiles.size());
    int *status = device_status_word();
    // {convert, products} or {products}; the tile counter starts at zero
    auto enqueue = [&](cudaStream_t s) -> int {
        if (converted) {
            const int cs = launch_tc_convert((const uint8_t *)workspace, conv_items, s);
            if (cs != QADIC_OK) return cs;
            return launch_tc_products((const uint8_t *)workspace, grid, tc_slot, tc_stages,
                                      status, s);
        }
        batched_kernel<<<(unsigned)grid, kThreads, smem, s>>>((uint8_t *)workspace);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "batched launch: %s", cudaGetErrorString(e));
        return QADIC_OK;
    };

    if (!use_graph) return enqueue(stream);
    // Capture {counter reset, kernel} on a private stream (the caller's may
    // be the legacy default stream, which cannot be captured; capturing runs
    // nothing), then launch the graph on the caller's stream.  The work list
    // uploaded above stays in the workspace for every replay.
    cudaStream_t cap = capture_stream(dev);
    if (!cap) return set_error(QADIC_E_CUDA, "no capture stream");
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "begin capture: %s", cudaGetErrorString(cudaGetLastError()));
    cudaMemsetAsync(workspace, 0, sizeof(uint32_t), cap);
    const int qs = enqueue(cap);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
    if (qs != QADIC_OK || le != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (qs != QADIC_OK) return qs;
        return set_error(QADIC_E_CUDA, "capture: %s", cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return set_error(QADIC_E_CUDA, "instantiate: %s", cudaGetErrorString(ie));
    if (cudaGraphLaunch(exec, stream) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return set_error(QADIC_E_CUDA, "graph launch: %s", cudaGetErrorString(cudaGetLastError()));
    }
    std::lock_guard<std::mutex> lock(g_graph_mu);
    if (g_graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    const uint64_t id = g_next_list_id++;
    host.resize(used);
    g_graphs.push_back(GraphEntry{std::move(key), exec, std::move(host), id});
    g_ws_list[workspace] = id;
    return QADIC_OK;
}

int batched_tile_configs(uint32_t k, qadic_tile_config *out, int32_t capacity, int32_t *n) {
    if (k < 1 || k > kMaxK) return set_error(QADIC_E_INVALID, "k outside [1, %u]", kMaxK);
    if (!n || (capacity > 0 && !out)) return set_error(QADIC_E_INVALID, "NULL output");
    *n = num_cfgs(k);
    for (int32_t c = 0; c < std::min<int32_t>(capacity, *n); ++c) {
        const TileShape t = tile_shape_of(k, c);
        out[c].bm = t.bm;
        out[c].bn = t.bn;
        out[c].bk = t.bk;
        out[c].smem_bytes = (int32_t)tile_smem_bytes(k, c);
    }
    return QADIC_OK;
}

int batched_select_tiles(uint32_t k, int32_t index) {
    if (k < 1 || k > kMaxK) return set_error(QADIC_E_INVALID, "k outside [1, %u]", kMaxK);
    if (index < -1 || index >= num_cfgs(k))
        return set_error(QADIC_E_INVALID, "configuration %d outside [-1, %d)", index, num_cfgs(k));
    std::lock_guard<std::mutex> lock(g_tiles_mu);
    g_tile_choice[k] = index;
    return QADIC_OK;
}

int batched_selected_tiles(uint32_t k, int32_t *index) {
    if (k < 1 || k > kMaxK) return set_error(QADIC_E_INVALID, "k outside [1, %u]", kMaxK);
    if (!index) return set_error(QADIC_E_INVALID, "NULL output");
    *index = tile_choice(k);
    return QADIC_OK;
}

// For each k present (largest total work first), time every candidate on
// this batch -- one graph capture as warm-up, then `reps` graph replays
// between CUDA events -- and keep the fastest before tuning the next k.
// The candidates are the register-staged kernel's tile shapes: tuning runs
// that kernel (the workspace is offered with its work-list size only), which
// the batched call uses when the workspace holds no converted operands and
// the allocation-free call always; the tensor-core path's tiles follow from
// the tensor-memory budget per k (tc_bn).
int autotune_batched(const Field *const *fields, int32_t nfields, const qadic_gemm_desc *descs,
                     int64_t count, void *workspace, size_t ws_bytes, int32_t reps,
                     int32_t *chosen, cudaStream_t stream) {
    if (reps < 1 || reps > 1000) return set_error(QADIC_E_INVALID, "reps outside [1, 1000]");
    ws_bytes = std::min(ws_bytes, batched_workspace_size(descs, count));
    if (nfields < 1 || nfields > kMaxFields)
        return set_error(QADIC_E_INVALID, "nfields must be in [1, %d]", kMaxFields);
    double work[kMaxK + 1] = {0};
    for (int64_t i = 0; i < count; ++i) {
        const qadic_gemm_desc &d = descs[i];
        if (d.field < 0 || d.field >= nfields || !fields[d.field])
            return set_error(QADIC_E_INVALID, "desc %lld: field index out of range", (long long)i);
        const double k = fields[d.field]->k;
        work[(int)k] += k * k * (double)d.m * d.n * d.K;
    }
    std::vector<uint32_t> ks;
    for (uint32_t k = 1; k <= kMaxK; ++k)
        if (work[k] > 0) ks.push_back(k);
    std::stable_sort(ks.begin(), ks.end(), [&](uint32_t a, uint32_t b) { return work[a] > work[b]; });
    for (uint32_t k = 0; k <= kMaxK; ++k) chosen[k] = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return set_error(QADIC_E_CUDA, "event: %s", cudaGetErrorString(cudaGetLastError()));
    }
    int st = QADIC_OK;
    for (uint32_t k : ks) {
        int best = 0;
        float best_ms = 0.f;
        bool have = false;
        for (int c = 0; c < num_cfgs(k) && st == QADIC_OK; ++c) {
            // a candidate deeper than some field's exact chunk would fall back to 0
            bool fits = true;
            for (int32_t i = 0; i < nfields; ++i)
                if (fields[i]->k == k && fields[i]->k_chunk_f32 < tile_shape_of(k, c).bk) fits = false;
            if (!fits) continue;
            batched_select_tiles(k, c);
            st = launch_batched(fields, nfields, descs, count, workspace, ws_bytes, true, stream);
            if (st != QADIC_OK) break;
            cudaEventRecord(e0, stream);
            for (int32_t r = 0; r < reps && st == QADIC_OK; ++r)
                st = launch_batched(fields, nfields, descs, count, workspace, ws_bytes, true, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = set_error(QADIC_E_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!have || ms < best_ms) {
                best = c;
                best_ms = ms;
                have = true;
            }
        }
        batched_select_tiles(k, best);
        chosen[k] = best;
        if (st != QADIC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace qadic

// ------------------------------------------------------------------------
// Allocation-free variant of qadic_batched_gemm.
//
// The work list lives in a fixed device array that belongs to this library
// instead of in a caller-provided workspace, and the host side builds it in
// a fixed host array, so a call allocates no memory of any kind.  Every
// device that loads the library keeps the array until the process exits.
// All calls share it: the header (tile counter included) is rewritten by
// every call, and two calls whose kernels overlap on the GPU race on it.
namespace qadic {

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;   // 8 MiB

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
alignas(256) uint8_t g_noalloc_host[kNoAllocScratchBytes];
void *g_noalloc_dev[64] = {nullptr};
// One event per device, recorded after each upload of the host array; the
// next call waits for the last one before it rewrites the array, since a
// copy from pageable memory need not have read all of it when
// cudaMemcpyAsync returns (on a system whose GPU reads host page tables,
// the copy may read the array in place).
cudaEvent_t g_noalloc_uploaded[64] = {nullptr};
cudaEvent_t g_noalloc_pending = nullptr;

// Set-up, once per device with that device current: the device address of
// the array (the symbol's name is only a host-side stand-in) and the upload
// event.
int noalloc_device_ptr(int dev, void **out) {
    if (dev < 0 || dev >= 64) return set_error(QADIC_E_INVALID, "device index %d", dev);
    if (!g_noalloc_dev[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return set_error(QADIC_E_CUDA, "scratch address: %s", cudaGetErrorString(e));
        cudaEvent_t ev = nullptr;
        const cudaError_t e2 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e2 != cudaSuccess)
            return set_error(QADIC_E_CUDA, "upload event: %s", cudaGetErrorString(e2));
        g_noalloc_uploaded[dev] = ev;
        g_noalloc_dev[dev] = ptr;
    }
    *out = g_noalloc_dev[dev];
    return QADIC_OK;
}

}  // namespace

int launch_batched_noalloc(const Field *const *fields, int32_t nfields,
                           const qadic_gemm_desc *descs, int64_t count, cudaStream_t stream) {
    if (nfields < 1 || nfields > kMaxFields)
        return set_error(QADIC_E_INVALID, "nfields must be in [1, %d]", kMaxFields);
    if (count > (1 << 24)) return set_error(QADIC_E_INVALID, "too many products");
    int dev = -1;
    cudaGetDevice(&dev);
    for (int32_t i = 0; i < nfields; ++i) {
        if (!fields[i]) return set_error(QADIC_E_INVALID, "field %d is NULL", i);
        if (fields[i]->device != dev)
            return set_error(QADIC_E_INVALID, "field %d lives on another device", i);
    }
    for (int64_t i = 0; i < count; ++i) {
        const qadic_gemm_desc &d = descs[i];
        if (d.field < 0 || d.field >= nfields)
            return set_error(QADIC_E_INVALID, "desc %lld: field index out of range", (long long)i);
        if (d.m < 1 || d.n < 1 || d.K < 1 || d.m > 4096 || d.n > 4096 || d.K > 4096)
            return set_error(QADIC_E_INVALID, "desc %lld: sizes must be in [1, 4096]", (long long)i);
        if (!d.A || !d.B || !d.C) return set_error(QADIC_E_INVALID, "desc %lld: NULL", (long long)i);
        if (d.lda < d.K || d.ldb < d.n || d.ldc < d.n)
            return set_error(QADIC_E_INVALID, "desc %lld: leading dimension too small",
                             (long long)i);
        if (fields[d.field]->k_chunk_f32 < kMinBK)
            return set_error(QADIC_E_OVERFLOW, "exact FP32 chunk below one K-block");
    }
    int cfgs[kMaxFields];
    size_t smem = 0;
    for (int32_t i = 0; i < nfields; ++i) {
        cfgs[i] = field_cfg(*fields[i]);
        smem = std::max(smem, tile_smem_bytes(fields[i]->k, cfgs[i]));
    }
    const int64_t tile_bound = max_tiles(descs, count);
    if (tile_bound > kMaxQueueTiles)
        return set_error(QADIC_E_INVALID,
                         "the batch has up to %lld output tiles; the work queue indexes at most %lld",
                         (long long)tile_bound, (long long)kMaxQueueTiles);
    int st0 = prepare_kernel(smem);
    if (st0 != QADIC_OK) return st0;
    const Layout L = layout_for(count, tile_bound);
    if (L.total > kNoAllocScratchBytes)
        return set_error(QADIC_E_INVALID,
                         "work list of %zu bytes exceeds the %zu-byte fixed scratch of the "
                         "allocation-free entry point; use qadic_batched_gemm with a workspace",
                         L.total, kNoAllocScratchBytes);

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    void *dptr = nullptr;
    int st = noalloc_device_ptr(dev, &dptr);
    if (st != QADIC_OK) return st;

    // the previous call's upload must have read the host array before it changes
    if (g_noalloc_pending) {
        const cudaError_t e = cudaEventSynchronize(g_noalloc_pending);
        if (e != cudaSuccess)
            return set_error(QADIC_E_CUDA, "previous upload: %s", cudaGetErrorString(e));
        g_noalloc_pending = nullptr;
    }
    uint8_t *host = g_noalloc_host;
    std::memset(host, 0, L.tiles_off);
    BFieldParams *fp = reinterpret_cast<BFieldParams *>(host + L.fields_off);
    for (int32_t i = 0; i < nfields; ++i) field_params(*fields[i], fp[i]);
    BProd *pp = reinterpret_cast<BProd *>(host + L.prods_off);
    BTile *tp = reinterpret_cast<BTile *>(host + L.tiles_off);
    int64_t nt = 0;
    for (int64_t i = 0; i < count; ++i) {
        const qadic_gemm_desc &d = descs[i];
        BProd &P = pp[i];
        P.A = d.A;
        P.B = d.B;
        P.C = d.C;
        P.m = d.m;
        P.n = d.n;
        P.K = d.K;
        P.lda = d.lda;
        P.ldb = d.ldb;
        P.ldc = d.ldc;
        P.field = d.field;
        P.cfg = cfgs[d.field];
        const TileShape ts = tile_shape_of(fields[d.field]->k, P.cfg);
        for (int tm = 0; tm * ts.bm < d.m; ++tm)
            for (int tn = 0; tn * ts.bn < d.n; ++tn) tp[nt++] = BTile{(int32_t)i, (int16_t)tm, (int16_t)tn};
    }
    // largest tiles first; std::sort works in place
    auto cost = [&](const BTile &t) {
        const qadic_gemm_desc &d = descs[t.prod];
        return tile_cost(d, fields[d.field]->k, cfgs[d.field]);
    };
    std::sort(tp, tp + nt, [&](const BTile &a, const BTile &b) {
        const uint64_t ca = cost(a), cb = cost(b);
        if (ca != cb) return ca > cb;
        if (a.prod != b.prod) return a.prod < b.prod;
        return a.tm != b.tm ? a.tm < b.tm : a.tn < b.tn;
    });
    BHeader *hdr = reinterpret_cast<BHeader *>(host);
    hdr->counter = 0;   // every call starts the tile counter from zero
    hdr->ntiles = (int32_t)nt;
    hdr->nprod = (int32_t)count;
    hdr->nfields = nfields;
    hdr->fields_off = (uint32_t)L.fields_off;
    hdr->prods_off = (uint32_t)L.prods_off;
    hdr->tiles_off = (uint32_t)L.tiles_off;
    const size_t used = L.tiles_off + (size_t)nt * sizeof(BTile);
    if (cudaMemcpyAsync(dptr, host, used, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "work list upload: %s", cudaGetErrorString(cudaGetLastError()));
    if (cudaEventRecord(g_noalloc_uploaded[dev], stream) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "upload event: %s", cudaGetErrorString(cudaGetLastError()));
    g_noalloc_pending = g_noalloc_uploaded[dev];
    const int64_t grid = grid_for(dev, smem, nt);
    batched_kernel<<<(unsigned)grid, kThreads, smem, stream>>>((uint8_t *)dptr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "batched launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace qadic

using namespace qadic;

extern "C" int qadic_batched_gemm_noalloc(const qadic_field *const *fields, int32_t nfields,
                                          const qadic_gemm_desc *descs, int64_t count,
                                          void *stream) {
    if (count < 0) return set_error(QADIC_E_INVALID, "negative count");
    if (count == 0) return QADIC_OK;
    if (!fields || !descs) return set_error(QADIC_E_INVALID, "NULL fields or descs");
    if (nfields < 1 || nfields > 64) return set_error(QADIC_E_INVALID, "nfields outside [1, 64]");
    const Field *fs[64];
    for (int32_t i = 0; i < nfields; ++i) {
        if (!fields[i]) return set_error(QADIC_E_INVALID, "field %d is NULL", i);
        fs[i] = field_of(fields[i]);
    }
    return launch_batched_noalloc(fs, nfields, descs, count, (cudaStream_t)stream);
}

extern "C" int qadic_batched_tile_configs(uint32_t k, qadic_tile_config *out, int32_t capacity,
                                          int32_t *count) {
    return batched_tile_configs(k, out, capacity, count);
}

extern "C" int qadic_batched_select_tiles(uint32_t k, int32_t index) {
    return batched_select_tiles(k, index);
}

extern "C" int qadic_batched_selected_tiles(uint32_t k, int32_t *index) {
    return batched_selected_tiles(k, index);
}

extern "C" int qadic_batched_autotune(const qadic_field *const *fields, int32_t nfields,
                                      const qadic_gemm_desc *descs, int64_t count, void *workspace,
                                      size_t ws_bytes, int32_t reps, int32_t *chosen,
                                      void *stream) {
    if (count < 1) return set_error(QADIC_E_INVALID, "nothing to tune");
    if (!fields || !descs || !chosen) return set_error(QADIC_E_INVALID, "NULL argument");
    if (nfields < 1 || nfields > 64) return set_error(QADIC_E_INVALID, "nfields outside [1, 64]");
    const Field *fs[64];
    for (int32_t i = 0; i < nfields; ++i) {
        if (!fields[i]) return set_error(QADIC_E_INVALID, "field %d is NULL", i);
        fs[i] = field_of(fields[i]);
    }
    return autotune_batched(fs, nfields, descs, count, workspace, ws_bytes, reps, chosen,
                            (cudaStream_t)stream);
}
