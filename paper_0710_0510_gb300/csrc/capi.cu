// C ABI entry points of libqadic (declared in include/qadic.h): argument
// and bound checks on the host, field lifetime, dispatch to the kernels.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "qadic_internal.h"

struct qadic_field {
    qadic::Field f;
};

namespace qadic {

namespace {
thread_local std::string t_last_error;

__device__ int g_status_word;   // bounded-wait status (one per device)

std::mutex g_status_mu;
int *g_status_ptr[64] = {nullptr};

// The device allocator for field tables (qadic_set_device_allocator).
int default_alloc(void **ptr, size_t bytes, void *) {
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) return QADIC_OK;
    cudaGetLastError();
    *ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? QADIC_E_NOMEM : QADIC_E_CUDA;
}

void default_free(void *ptr, size_t, void *) { cudaFree(ptr); }

struct Allocator {
    qadic_alloc_fn alloc = default_alloc;
    qadic_free_fn free_fn = default_free;
    void *ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

Allocator current_allocator() {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc;
}

template <class T>
int alloc_table(const Allocator &a, T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return QADIC_OK;
    void *p = nullptr;
    const int st = a.alloc(&p, src.size() * sizeof(T), a.ctx);
    if (st != QADIC_OK || !p) {
        *dst = nullptr;
        return set_error(st == QADIC_E_CUDA ? QADIC_E_CUDA : QADIC_E_NOMEM,
                         "device allocation of %zu bytes for a field table failed (status %d)",
                         src.size() * sizeof(T), st);
    }
    *dst = (T *)p;
    return QADIC_OK;
}

template <class T>
int copy_table(T *dst, const std::vector<T> &src) {
    if (src.empty()) return QADIC_OK;
    if (cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return set_error(QADIC_E_CUDA, "table upload failed: %s",
                         cudaGetErrorString(cudaGetLastError()));
    return QADIC_OK;
}

template <class T>
void free_table(Field &f, T *&p, const std::vector<T> &src) {
    if (p && f.table_free) f.table_free(p, src.size() * sizeof(T), f.table_ctx);
    p = nullptr;
}

void free_tables(Field &f) {
    free_table(f, f.d_antilog, f.antilog);
    free_table(f, f.d_log_f64, f.log_f64);
    free_table(f, f.d_log_centred, f.log_centred);
    free_table(f, f.d_tab_L, f.tab_L);
    free_table(f, f.d_tab_H, f.tab_H);
    free_table(f, f.d_fold, f.fold);
}

// Every device table from the allocator, then the uploads.
int upload_tables(Field &f) {
    const Allocator a = current_allocator();
    f.table_free = a.free_fn;
    f.table_ctx = a.ctx;
    int st;
    if ((st = alloc_table(a, &f.d_antilog, f.antilog)) ||
        (st = alloc_table(a, &f.d_log_f64, f.log_f64)) ||
        (st = alloc_table(a, &f.d_log_centred, f.log_centred)) ||
        (st = alloc_table(a, &f.d_tab_L, f.tab_L)) || (st = alloc_table(a, &f.d_tab_H, f.tab_H)) ||
        (st = alloc_table(a, &f.d_fold, f.fold)))
        return st;
    if (cudaGetDevice(&f.device) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
    if ((st = copy_table(f.d_antilog, f.antilog)) || (st = copy_table(f.d_log_f64, f.log_f64)) ||
        (st = copy_table(f.d_log_centred, f.log_centred)) || (st = copy_table(f.d_tab_L, f.tab_L)) ||
        (st = copy_table(f.d_tab_H, f.tab_H)) || (st = copy_table(f.d_fold, f.fold)))
        return st;
    return QADIC_OK;
}

// One non-blocking stream per device for the host copies of qadic_matmul_host.
// Library-owned non-blocking streams per device (index 0: copies, 1: packs
// of later row blocks in qadic_matmul_host).
cudaStream_t side_stream(int dev, int which = 0) {
    static std::mutex mu;
    static cudaStream_t streams[64][3] = {};
    if (dev < 0 || dev >= 64 || which < 0 || which > 2) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    cudaStream_t &st = streams[dev][which];
    if (!st && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
    }
    return st;
}

bool on_device(const Field &f) {
    if (f.device < 0) return false;
    int dev = -1;
    cudaGetDevice(&dev);
    return dev == f.device;
}

}  // namespace

const Field *field_of(const qadic_field *handle) { return handle ? &handle->f : nullptr; }

int set_error(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return status;
}

int *device_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_status_mu);
    if (!g_status_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_status_word) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_status_ptr[dev] = (int *)ptr;
    }
    return g_status_ptr[dev];
}

}  // namespace qadic

using namespace qadic;

extern "C" {

int qadic_field_init(qadic_field **out, uint32_t p, uint32_t k, const uint32_t *poly,
                     uint32_t flags) {
    if (!out) return set_error(QADIC_E_INVALID, "out is NULL");
    if (flags & ~QADIC_FIELD_HOST_ONLY) return set_error(QADIC_E_INVALID, "unknown flags");
    qadic_field *h = new (std::nothrow) qadic_field();
    if (!h) return set_error(QADIC_E_NOMEM, "host allocation failed");
    int st = build_field(h->f, p, k, poly);
    if (st != QADIC_OK) {
        delete h;
        return st;
    }
    static std::atomic<uint64_t> next_uid{1};
    h->f.uid = next_uid.fetch_add(1);
    if (flags & QADIC_FIELD_HOST_ONLY) {
        h->f.device = -1;
        *out = h;
        return QADIC_OK;
    }
    Field &f = h->f;
    if ((st = upload_tables(f)) != QADIC_OK) {
        free_tables(f);
        delete h;
        return st;
    }
    if (!device_status_word()) {
        free_tables(f);
        delete h;
        return set_error(QADIC_E_CUDA, "status word unavailable");
    }
    *out = h;
    return QADIC_OK;
}

int qadic_set_device_allocator(qadic_alloc_fn alloc, qadic_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return set_error(QADIC_E_INVALID, "alloc and free_fn must both be given or both be NULL");
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (!alloc) {
        g_alloc = Allocator();
    } else {
        g_alloc.alloc = alloc;
        g_alloc.free_fn = free_fn;
        g_alloc.ctx = ctx;
    }
    return QADIC_OK;
}

int qadic_field_destroy(qadic_field *field) {
    if (!field) return QADIC_OK;
    if (field->f.device < 0) {
        delete field;
        return QADIC_OK;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != field->f.device) cudaSetDevice(field->f.device);
    free_tables(field->f);
    if (prev >= 0 && prev != field->f.device) cudaSetDevice(prev);
    delete field;
    return QADIC_OK;
}

int qadic_field_info(const qadic_field *field, qadic_info *out) {
    if (!field || !out) return set_error(QADIC_E_INVALID, "NULL argument");
    const Field &f = field->f;
    std::memset(out, 0, sizeof(*out));
    out->p = f.p;
    out->k = f.k;
    for (uint32_t i = 0; i <= f.k; ++i) out->poly[i] = f.poly[i];
    for (uint32_t i = 0; i < f.k; ++i) out->generator[i] = f.gen[i];
    out->order = f.order;
    out->zero_code = f.order - 1;
    out->log_bytes = f.order <= 256 ? 1 : 2;
    out->log2_q = f.log2_q;
    out->n_q = f.n_q;
    out->k_max_int32 = f.k_max_int32;
    out->k_chunk_f32 = f.k_chunk_f32;
    return QADIC_OK;
}

int qadic_pack(const qadic_field *field, int in_fmt, const void *in, int64_t rows, int64_t cols,
               int64_t ld_in, int out_fmt, void *out, int64_t ld_out, void *stream) {
    if (!field) return set_error(QADIC_E_INVALID, "field is NULL");
    const Field &f = field->f;
    if (!on_device(f)) return set_error(QADIC_E_INVALID, "field lives on another device");
    if (rows < 0 || cols < 0) return set_error(QADIC_E_INVALID, "negative size");
    if (rows == 0 || cols == 0) return QADIC_OK;
    if (!in || !out) return set_error(QADIC_E_INVALID, "NULL data pointer");
    if (ld_in < cols) return set_error(QADIC_E_INVALID, "ld_in < cols");
    const int64_t out_minor =
        (out_fmt == QADIC_FMT_OPERAND_B || out_fmt == QADIC_FMT_OPERAND_B_FOLD ||
         out_fmt == QADIC_FMT_OPERAND_B_KARA || out_fmt == QADIC_FMT_OPERAND_B_E4M3) ? rows : cols;
    if (ld_out < out_minor) return set_error(QADIC_E_INVALID, "ld_out too small");
    if (out_fmt == QADIC_FMT_QADIC_F64 && f.n_q == 0)
        return set_error(QADIC_E_OVERFLOW, "Eq. 2 admits no q-adic block for p=%u k=%u", f.p, f.k);
    if (out_fmt == QADIC_FMT_OPERAND_A || out_fmt == QADIC_FMT_OPERAND_B ||
        out_fmt == QADIC_FMT_OPERAND_B_FOLD || out_fmt == QADIC_FMT_OPERAND_A_KARA ||
        out_fmt == QADIC_FMT_OPERAND_B_KARA) {
        if (ld_out % 8 != 0 || ((uintptr_t)out & 15) != 0)
            return set_error(QADIC_E_INVALID, "operand output needs ld %% 8 == 0 and 16B alignment");
    }
    if (out_fmt == QADIC_FMT_OPERAND_A_E4M3 || out_fmt == QADIC_FMT_OPERAND_B_E4M3) {
        if (ld_out % 16 != 0 || ((uintptr_t)out & 15) != 0)
            return set_error(QADIC_E_INVALID, "e4m3 operand output needs ld %% 16 == 0 and 16B alignment");
    }
    return launch_pack(f, in_fmt, in, rows, cols, ld_in, out_fmt, out, ld_out,
                       (cudaStream_t)stream);
}

int qadic_gemm(const qadic_field *field, int path, int64_t m, int64_t n, int64_t K, const void *A,
               int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc, void *workspace,
               size_t ws_bytes, void *stream) {
    (void)workspace;
    (void)ws_bytes;
    if (!field) return set_error(QADIC_E_INVALID, "field is NULL");
    const Field &f = field->f;
    if (!on_device(f)) return set_error(QADIC_E_INVALID, "field lives on another device");
    if (m < 0 || n < 0 || K < 0) return set_error(QADIC_E_INVALID, "negative size");
    if (m == 0 || n == 0) return QADIC_OK;
    if (!C) return set_error(QADIC_E_INVALID, "C is NULL");
    if (ldc < n) return set_error(QADIC_E_INVALID, "ldc < n");
    if (K > 0 && (!A || !B)) return set_error(QADIC_E_INVALID, "NULL operand");
    cudaStream_t s = (cudaStream_t)stream;
    if (path == QADIC_PATH_FP64_QADIC) {
        if (f.n_q == 0)
            return set_error(QADIC_E_OVERFLOW, "Eq. 2 admits no q-adic block for p=%u k=%u", f.p,
                             f.k);
        if (f.k > 4) return set_error(QADIC_E_UNSUPPORTED, "FP64 path supports k <= 4");
        if (lda < K || ldb < n) return set_error(QADIC_E_INVALID, "lda < K or ldb < n");
        return launch_gemm_f64(f, m, n, K, (const double *)A, lda, (const double *)B, ldb, C, ldc,
                               s);
    }
    if (path == QADIC_PATH_PLANES || path == QADIC_PATH_PLANES_E4M3) {
        if (lda < K || ldb < K) return set_error(QADIC_E_INVALID, "lda or ldb < K");
        if (!gemm_planes_tc_supported(f))
            return set_error(QADIC_E_UNSUPPORTED, "no tensor-core plane kernel for k=%u", f.k);
        return launch_gemm_planes_tc(f, m, n, K, A, lda, B, ldb, C, ldc, s,
                                     path == QADIC_PATH_PLANES_E4M3);
    }
    if (path == QADIC_PATH_FOLD) {
        if (lda < K || ldb < K) return set_error(QADIC_E_INVALID, "lda or ldb < K");
        if (f.k > 8) return set_error(QADIC_E_UNSUPPORTED, "no fold kernel for k=%u", f.k);
        return launch_gemm_fold_tc(f, m, n, K, A, lda, B, ldb, C, ldc, s);
    }
    if (path == QADIC_PATH_KARATSUBA) {
        if (lda < K || ldb < K) return set_error(QADIC_E_INVALID, "lda or ldb < K");
        if (f.k != 2) return set_error(QADIC_E_UNSUPPORTED, "the Karatsuba form is for k = 2");
        return launch_gemm_karatsuba_tc(f, m, n, K, A, lda, B, ldb, C, ldc, s);
    }
    return set_error(QADIC_E_INVALID, "unknown path %d", path);
}

static size_t align256_(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of the two packed operands of qadic_matmul (bf16 rows padded to a
// multiple of 8 elements, so every layout meets the 16-byte TMA rules).
static size_t packed_bytes(const Field &f, int path, int64_t m, int64_t n, int64_t K,
                           size_t *a_bytes) {
    const size_t K8 = (size_t)((K + 7) / 8 * 8);
    size_t a = 0, b = 0;
    switch (path) {
        case QADIC_PATH_FP64_QADIC: a = 8 * (size_t)m * K; b = 8 * (size_t)K * n; break;
        case QADIC_PATH_PLANES: a = 2 * (size_t)f.k * m * K8; b = 2 * (size_t)f.k * n * K8; break;
        case QADIC_PATH_FOLD:
            a = 2 * (size_t)f.k * m * K8;
            b = 2 * (size_t)f.k * f.k * (size_t)fold_n_pad(n) * K8;
            break;
        case QADIC_PATH_KARATSUBA: a = 6 * (size_t)m * K8; b = 6 * (size_t)n * K8; break;
        case QADIC_PATH_PLANES_E4M3: {   // one byte per element, rows padded to 16
            const size_t K16 = (size_t)((K + 15) / 16 * 16);
            a = (size_t)f.k * m * K16;
            b = (size_t)f.k * n * K16;
            break;
        }
        default: return 0;
    }
    if (a_bytes) *a_bytes = align256_(a);
    return align256_(a) + align256_(b);
}

// Both operands in one call; e4m3 selects the fp8 operand formats.
static int pack_operands(const qadic_field *field, int in_fmt, const void *A, int64_t m, int64_t K,
                         int64_t lda_in, void *outA, int64_t lda_out, const void *B, int64_t n,
                         int64_t ldb_in, void *outB, int64_t ldb_out, void *stream, bool e4m3) {
    if (!field) return set_error(QADIC_E_INVALID, "field is NULL");
    const Field &f = field->f;
    if (!on_device(f)) return set_error(QADIC_E_INVALID, "field lives on another device");
    if (m < 0 || n < 0 || K < 0) return set_error(QADIC_E_INVALID, "negative size");
    if (e4m3 && f.p > 31)
        return set_error(QADIC_E_UNSUPPORTED, "e4m3 operands need p <= 31 (|c| <= 15 exact)");
    if (m == 0 || n == 0 || K == 0) return QADIC_OK;
    if (!A || !B || !outA || !outB) return set_error(QADIC_E_INVALID, "NULL data pointer");
    if (lda_in < K || ldb_in < n) return set_error(QADIC_E_INVALID, "ld_in too small");
    const int64_t lo = e4m3 ? 16 : 8;
    if (lda_out < K || ldb_out < K || lda_out % lo || ldb_out % lo || ((uintptr_t)outA & 15) ||
        ((uintptr_t)outB & 15))
        return set_error(QADIC_E_INVALID, "operand outputs need ld >= K, ld %% %d == 0, 16B alignment",
                         (int)lo);
    const int fa = e4m3 ? QADIC_FMT_OPERAND_A_E4M3 : QADIC_FMT_OPERAND_A;
    const int fb = e4m3 ? QADIC_FMT_OPERAND_B_E4M3 : QADIC_FMT_OPERAND_B;
    if (in_fmt == QADIC_FMT_LOG) {
        int st = qadic_pack(field, in_fmt, A, m, K, lda_in, fa, outA, lda_out, stream);
        if (st != QADIC_OK) return st;
        return qadic_pack(field, in_fmt, B, K, n, ldb_in, fb, outB, ldb_out, stream);
    }
    if (in_fmt != QADIC_FMT_COEFF_U8 && in_fmt != QADIC_FMT_INT8_PLANES)
        return set_error(QADIC_E_INVALID, "input format %d", in_fmt);
    return launch_pack_pair(f, in_fmt, A, m, K, lda_in, outA, lda_out, B, n, ldb_in, outB, ldb_out,
                            (cudaStream_t)stream, e4m3);
}

int qadic_pack_operands(const qadic_field *field, int in_fmt, const void *A, int64_t m, int64_t K,
                        int64_t lda_in, void *outA, int64_t lda_out, const void *B, int64_t n,
                        int64_t ldb_in, void *outB, int64_t ldb_out, void *stream) {
    return pack_operands(field, in_fmt, A, m, K, lda_in, outA, lda_out, B, n, ldb_in, outB, ldb_out,
                         stream, false);
}

int qadic_pack_operands_e4m3(const qadic_field *field, int in_fmt, const void *A, int64_t m,
                             int64_t K, int64_t lda_in, void *outA, int64_t lda_out, const void *B,
                             int64_t n, int64_t ldb_in, void *outB, int64_t ldb_out, void *stream) {
    return pack_operands(field, in_fmt, A, m, K, lda_in, outA, lda_out, B, n, ldb_in, outB, ldb_out,
                         stream, true);
}

size_t qadic_matmul_device_workspace_size(const qadic_field *field, int path, int64_t m, int64_t n,
                                          int64_t K) {
    if (!field || m < 0 || n < 0 || K < 0) return 0;
    return packed_bytes(field->f, path, m, n, K, nullptr);
}

int qadic_matmul(const qadic_field *field, int path, int in_fmt, int64_t m, int64_t n, int64_t K,
                 const void *A, int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                 void *workspace, size_t ws_bytes, void *stream) {
    if (!field) return set_error(QADIC_E_INVALID, "field is NULL");
    const Field &f = field->f;
    if (!on_device(f)) return set_error(QADIC_E_INVALID, "field lives on another device");
    if (m < 0 || n < 0 || K < 0) return set_error(QADIC_E_INVALID, "negative size");
    if (in_fmt != QADIC_FMT_LOG && in_fmt != QADIC_FMT_COEFF_U8 && in_fmt != QADIC_FMT_INT8_PLANES)
        return set_error(QADIC_E_INVALID, "input format %d", in_fmt);
    if (path < QADIC_PATH_FP64_QADIC || path > QADIC_PATH_PLANES_E4M3)
        return set_error(QADIC_E_INVALID, "unknown path %d", path);
    if (path == QADIC_PATH_PLANES_E4M3 && f.p > 31)
        return set_error(QADIC_E_UNSUPPORTED, "e4m3 operands need p <= 31 (|c| <= 15 exact)");
    size_t a_bytes = 0;
    const size_t need = packed_bytes(f, path, m, n, K, &a_bytes);
    if (m == 0 || n == 0) return QADIC_OK;
    if (need > 0 && (!workspace || ws_bytes < need))
        return set_error(QADIC_E_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
    if (((uintptr_t)workspace) & 255) return set_error(QADIC_E_INVALID, "workspace must be 256-byte aligned");
    char *pA = (char *)workspace, *pB = pA ? pA + a_bytes : nullptr;
    const int64_t K8 = (K + 7) / 8 * 8;
    int st;
    if (!C || ldc < n) return set_error(QADIC_E_INVALID, "C is NULL or ldc < n");
    if (K == 0) {   // empty sums: C = 0
        for (uint32_t i = 0; i < f.k; ++i)
            if (cudaMemset2DAsync(C + (size_t)i * m * ldc, (size_t)ldc, 0, (size_t)n, (size_t)m,
                                  (cudaStream_t)stream) != cudaSuccess)
                return set_error(QADIC_E_CUDA, "memset: %s", cudaGetErrorString(cudaGetLastError()));
        return QADIC_OK;
    }
    // (bf16 rows are K8 long; the tensor maps' inner extent is K, so the pad
    // columns are never read)
    if (path == QADIC_PATH_PLANES) {
        if (!gemm_planes_tc_supported(f))
            return set_error(QADIC_E_UNSUPPORTED, "no tensor-core plane kernel for k=%u", f.k);
        if (!A || !B) return set_error(QADIC_E_INVALID, "NULL operand");
        if (lda < K || ldb < n) return set_error(QADIC_E_INVALID, "lda < K or ldb < n");
        if ((st = qadic_pack_operands(field, in_fmt, A, m, K, lda, pA, K8, B, n, ldb, pB, K8,
                                      stream)))
            return st;
        return qadic_gemm(field, path, m, n, K, pA, K8, pB, K8, C, ldc, nullptr, 0, stream);
    }
    int fa, fb;
    int64_t la, lb;
    switch (path) {
        case QADIC_PATH_FP64_QADIC: fa = fb = QADIC_FMT_QADIC_F64; la = K; lb = n; break;
        case QADIC_PATH_PLANES_E4M3: {
            // both operands by one launch where the inputs allow it
            if (!gemm_planes_tc_supported(f))
                return set_error(QADIC_E_UNSUPPORTED, "no tensor-core plane kernel for k=%u", f.k);
            if (!A || !B) return set_error(QADIC_E_INVALID, "NULL operand");
            if (lda < K || ldb < n) return set_error(QADIC_E_INVALID, "lda < K or ldb < n");
            const int64_t K16 = (K + 15) / 16 * 16;
            if ((st = qadic_pack_operands_e4m3(field, in_fmt, A, m, K, lda, pA, K16, B, n, ldb, pB,
                                               K16, stream)))
                return st;
            return qadic_gemm(field, path, m, n, K, pA, K16, pB, K16, C, ldc, nullptr, 0, stream);
        }
        case QADIC_PATH_FOLD: fa = QADIC_FMT_OPERAND_A; fb = QADIC_FMT_OPERAND_B_FOLD; la = lb = K8; break;
        default: fa = QADIC_FMT_OPERAND_A_KARA; fb = QADIC_FMT_OPERAND_B_KARA; la = lb = K8; break;
    }
    if ((st = qadic_pack(field, in_fmt, A, m, K, lda, fa, pA, la, stream))) return st;
    if ((st = qadic_pack(field, in_fmt, B, K, n, ldb, fb, pB, lb, stream))) return st;
    return qadic_gemm(field, path, m, n, K, pA, la, pB, lb, C, ldc, nullptr, 0, stream);
}

static size_t in_elem_bytes(const Field &f, int fmt) {
    if (fmt == QADIC_FMT_LOG) return f.order <= 256 ? 1 : 2;
    if (fmt == QADIC_FMT_COEFF_U8 || fmt == QADIC_FMT_INT8_PLANES) return f.k;
    return 0;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t qadic_matmul_workspace_size(const qadic_field *field, int path, int in_fmt, int64_t m,
                                   int64_t n, int64_t K) {
    if (!field || m < 0 || n < 0 || K < 0) return 0;
    const Field &f = field->f;
    const size_t eb = in_elem_bytes(f, in_fmt);
    if (!eb) return 0;
    size_t ws = align256(eb * m * K) + align256(eb * K * n) + align256((size_t)f.k * m * n);
    if (path == QADIC_PATH_FP64_QADIC)
        ws += align256(8 * (size_t)m * K) + align256(8 * (size_t)K * n);
    else
        ws += align256(2 * (size_t)f.k * m * K) + align256(2 * (size_t)f.k * n * K);
    return ws;
}

namespace {

// The plane path's host pipeline with B cut into four column blocks as well
// as A into row blocks (n a multiple of 512 and at least 1024, m >= 512):
// the first GEMM needs one quarter of B and the first rows of A, so it
// starts after about a fifth of the inputs have crossed the link instead of
// all of B.  Copies in on `side` (B_0, A_0, then the other blocks of B, then
// those of A), packs on `side2` as each block lands, the block GEMMs on `s`
// (each one round of 256 x 128 output units on the SM pairs), each block of
// C back on `d2h` while the next is computed, the last on `s`.
int matmul_host_blocked(const qadic_field *field, const Field &f, int in_fmt, int64_t m, int64_t n,
                        int64_t K, const void *A_host, const void *B_host, uint8_t *C_host, char *dA,
                        char *dB, uint8_t *dC, char *pA, char *pB, uint32_t planes, size_t esz,
                        cudaStream_t s, cudaStream_t side, cudaStream_t side2, cudaStream_t d2h,
                        int sms) {
    constexpr int NCB = 4, kMaxRows = 4;
    const int64_t nc = n / NCB;
    const int64_t unit_rows = 256, um = (m + unit_rows - 1) / unit_rows;
    const int64_t tn = (nc + 127) / 128, cl = std::max(1, sms / 2);
    int64_t ub = std::max<int64_t>(1, cl / tn);
    if ((um + ub - 1) / ub > kMaxRows) ub = (um + kMaxRows - 1) / kMaxRows;
    const int nrb = (int)((um + ub - 1) / ub);
    int64_t rows[kMaxRows] = {0}, r0[kMaxRows] = {0};
    for (int i = 0; i < nrb; ++i) {
        r0[i] = (int64_t)i * ub * unit_rows;
        rows[i] = std::min<int64_t>(ub * unit_rows, m - r0[i]);
    }
    constexpr int kEvents = 1 + 2 * NCB + 2 * kMaxRows + kMaxRows * NCB + 2;
    cudaEvent_t ev[kEvents] = {};
    for (auto &e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return set_error(QADIC_E_CUDA, "event: %s", cudaGetErrorString(cudaGetLastError()));
        }
    cudaEvent_t *ev_bc = ev + 1, *ev_bp = ev + 1 + NCB, *ev_ac = ev + 1 + 2 * NCB,
                *ev_ap = ev + 1 + 2 * NCB + kMaxRows, *ev_g = ev + 1 + 2 * NCB + 2 * kMaxRows;
    cudaEvent_t &ev_start = ev[0], &ev_join = ev[kEvents - 2], &ev_d2h = ev[kEvents - 1];
    auto cleanup = [&](int status) {
        for (auto &x : ev) cudaEventDestroy(x);   // released once their work completes
        return status;
    };
    auto cuda_fail = [&](const char *what) {
        return cleanup(set_error(QADIC_E_CUDA, "%s: %s", what, cudaGetErrorString(cudaGetLastError())));
    };
    const size_t c_plane = (size_t)m * n;
    auto dA_blk = [&](int i) { return dA + (size_t)planes * r0[i] * K * esz; };
    auto pA_blk = [&](int i) { return pA + 2 * (size_t)f.k * r0[i] * K; };
    auto pB_blk = [&](int j) { return pB + 2 * (size_t)f.k * nc * K * j; };
    auto copy_b = [&](int j) -> cudaError_t {   // columns j nc .. j nc + nc - 1 of every plane
        for (uint32_t i = 0; i < planes; ++i) {
            const size_t off = ((size_t)i * K * n + (size_t)j * nc) * esz;
            const cudaError_t e = cudaMemcpy2DAsync(dB + off, n * esz, (const char *)B_host + off,
                                                    n * esz, nc * esz, K, cudaMemcpyHostToDevice, side);
            if (e != cudaSuccess) return e;
        }
        return cudaEventRecord(ev_bc[j], side);
    };
    auto copy_a = [&](int b) -> cudaError_t {   // rows r0[b] .., each plane a block of its own
        for (uint32_t i = 0; i < planes; ++i) {
            const cudaError_t e = cudaMemcpyAsync(
                dA_blk(b) + (size_t)i * rows[b] * K * esz,
                (const char *)A_host + ((size_t)i * m + r0[b]) * K * esz, (size_t)rows[b] * K * esz,
                cudaMemcpyHostToDevice, side);
            if (e != cudaSuccess) return e;
        }
        return cudaEventRecord(ev_ac[b], side);
    };
    // every side stream starts after the work already queued on `stream`
    if (cudaEventRecord(ev_start, s) || cudaStreamWaitEvent(side, ev_start, 0) ||
        cudaStreamWaitEvent(side2, ev_start, 0) || cudaStreamWaitEvent(d2h, ev_start, 0))
        return cuda_fail("stream order");
    if (copy_b(0) || copy_a(0)) return cuda_fail("H2D copy");
    for (int j = 1; j < NCB; ++j)
        if (copy_b(j)) return cuda_fail("H2D copy");
    for (int b = 1; b < nrb; ++b)
        if (copy_a(b)) return cuda_fail("H2D copy");
    // packs in the order the blocks land
    auto pack_b = [&](int j) -> int {
        if (cudaStreamWaitEvent(side2, ev_bc[j], 0)) return cuda_fail("wait");
        const int st = qadic_pack(field, in_fmt, dB + (size_t)j * nc * esz, K, nc, n,
                                  QADIC_FMT_OPERAND_B, pB_blk(j), K, side2);
        if (st != QADIC_OK) return cleanup(st);
        return cudaEventRecord(ev_bp[j], side2) ? cuda_fail("event") : QADIC_OK;
    };
    auto pack_a = [&](int b) -> int {
        if (cudaStreamWaitEvent(side2, ev_ac[b], 0)) return cuda_fail("wait");
        const int st = qadic_pack(field, in_fmt, dA_blk(b), rows[b], K, K, QADIC_FMT_OPERAND_A,
                                  pA_blk(b), K, side2);
        if (st != QADIC_OK) return cleanup(st);
        return cudaEventRecord(ev_ap[b], side2) ? cuda_fail("event") : QADIC_OK;
    };
    int st;
    if ((st = pack_b(0)) != QADIC_OK || (st = pack_a(0)) != QADIC_OK) return st;
    for (int j = 1; j < NCB; ++j)
        if ((st = pack_b(j)) != QADIC_OK) return st;
    for (int b = 1; b < nrb; ++b)
        if ((st = pack_a(b)) != QADIC_OK) return st;
    // block GEMMs; each block of C goes back while the next is computed
    for (int b = 0; b < nrb; ++b)
        for (int j = 0; j < NCB; ++j) {
            const bool last = b + 1 == nrb && j + 1 == NCB;
            if ((j == 0 && cudaStreamWaitEvent(s, ev_ap[b], 0)) ||
                (b == 0 && cudaStreamWaitEvent(s, ev_bp[j], 0)))
                return cuda_fail("wait");
            if ((st = launch_gemm_planes_tc_strided(f, rows[b], nc, K, pA_blk(b), K,
                                                    (int64_t)rows[b] * K, pB_blk(j), K,
                                                    (int64_t)nc * K, dC + r0[b] * n + (int64_t)j * nc,
                                                    n, (int64_t)c_plane, s)) != QADIC_OK)
                return cleanup(st);
            cudaStream_t cs = last ? s : d2h;
            if (!last && (cudaEventRecord(ev_g[b * NCB + j], s) ||
                          cudaStreamWaitEvent(d2h, ev_g[b * NCB + j], 0)))
                return cuda_fail("event");
            for (uint32_t i = 0; i < f.k; ++i) {
                const size_t off = i * c_plane + (size_t)r0[b] * n + (size_t)j * nc;
                if (cudaMemcpy2DAsync(C_host + off, n, dC + off, n, nc, rows[b],
                                      cudaMemcpyDeviceToHost, cs))
                    return cuda_fail("D2H copy");
            }
        }
    // join: `stream` also waits for the side streams' copies
    if (cudaEventRecord(ev_join, side) || cudaStreamWaitEvent(s, ev_join, 0) ||
        cudaEventRecord(ev_d2h, d2h) || cudaStreamWaitEvent(s, ev_d2h, 0))
        return cuda_fail("join");
    return cleanup(QADIC_OK);
}

}  // namespace

int qadic_matmul_host(const qadic_field *field, int path, int in_fmt, int64_t m, int64_t n,
                      int64_t K, const void *A_host, const void *B_host, uint8_t *C_host,
                      void *workspace, size_t ws_bytes, void *stream) {
    if (!field) return set_error(QADIC_E_INVALID, "field is NULL");
    const Field &f = field->f;
    const size_t need = qadic_matmul_workspace_size(field, path, in_fmt, m, n, K);
    if (!need) return set_error(QADIC_E_INVALID, "bad format or size");
    if (!workspace || ws_bytes < need)
        return set_error(QADIC_E_NOMEM, "workspace %zu < %zu bytes", ws_bytes, need);
    if (!A_host || !B_host || !C_host) return set_error(QADIC_E_INVALID, "NULL host pointer");
    if (path == QADIC_PATH_PLANES && (K % 8 != 0))
        return set_error(QADIC_E_INVALID, "plane path needs K %% 8 == 0 for dense operands");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t eb = in_elem_bytes(f, in_fmt);
    char *w = (char *)workspace;
    char *dA = w;
    w += align256(eb * m * K);
    char *dB = w;
    w += align256(eb * K * n);
    uint8_t *dC = (uint8_t *)w;
    w += align256((size_t)f.k * m * n);
    char *pA = w;
    w += align256((path == QADIC_PATH_FP64_QADIC ? 8 : 2 * (size_t)f.k) * m * K);
    char *pB = w;
    if (path != QADIC_PATH_FP64_QADIC && path != QADIC_PATH_PLANES)
        return set_error(QADIC_E_INVALID, "unknown path %d", path);
    if (path == QADIC_PATH_PLANES && !gemm_planes_tc_supported(f))
        return set_error(QADIC_E_UNSUPPORTED, "no tensor-core plane kernel for k=%u", f.k);

    // Overlap.  The inputs go host -> device on a side stream, B first and
    // then A in row blocks; B and the first block are packed on `stream`,
    // later blocks on a second side stream as soon as they land (a pack
    // block fits beside the GEMM's CTA on an SM), and the plane GEMM runs
    // per block.  Each block of C goes back to the host on a third stream
    // while the next one is computed (the link carries both directions at
    // once).  A block is as many 256-row unit rows as one round of 256 x 128
    // output units on the SM pairs takes, so the GEMMs can start on the
    // first small block and follow the copies, at most kMaxBlocks blocks.
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t side = side_stream(dev, 0), side2 = side_stream(dev, 1), d2h = side_stream(dev, 2);
    if (!side || !side2 || !d2h) return set_error(QADIC_E_CUDA, "no side stream");
    if (path == QADIC_PATH_PLANES && m >= 512 && n >= 1024 && n % 512 == 0) {
        const bool planar_in = in_fmt != QADIC_FMT_LOG;
        return matmul_host_blocked(field, f, in_fmt, m, n, K, A_host, B_host, C_host, dA, dB, dC, pA,
                                   pB, planar_in ? f.k : 1, planar_in ? 1 : eb, s, side, side2, d2h,
                                   sms);
    }
    constexpr int kMaxBlocks = 8;
    int64_t rows[kMaxBlocks] = {m};
    int nblk = 1;
    if (path == QADIC_PATH_PLANES && m >= 512) {
        const int64_t unit_rows = 256, um = (m + unit_rows - 1) / unit_rows;
        const int64_t tn = (n + 127) / 128, cl = std::max(1, sms / 2);
        int64_t ub = std::max<int64_t>(1, cl / tn);          // unit rows per block: one round
        if ((um + ub - 1) / ub > kMaxBlocks) ub = (um + kMaxBlocks - 1) / kMaxBlocks;
        const int64_t nb = (um + ub - 1) / ub;
        if (nb >= 2) {
            nblk = (int)nb;
            for (int b = 0; b < nblk; ++b)
                rows[b] = std::min<int64_t>(ub * unit_rows, m - (int64_t)b * ub * unit_rows);
        }
    }
    constexpr int kEvents = 2 + 3 * kMaxBlocks + 2;
    cudaEvent_t ev[kEvents] = {};
    for (auto &e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return set_error(QADIC_E_CUDA, "event: %s", cudaGetErrorString(cudaGetLastError()));
        }
    cudaEvent_t &ev_start = ev[0], &ev_b = ev[1], &ev_join = ev[kEvents - 2], &ev_d2h = ev[kEvents - 1];
    cudaEvent_t *ev_copied = ev + 2, *ev_packed = ev + 2 + kMaxBlocks, *ev_gemm = ev + 2 + 2 * kMaxBlocks;
    auto cleanup = [&](int status) {
        for (auto &x : ev) cudaEventDestroy(x);   // released once their work completes
        return status;
    };
    auto cuda_fail = [&](const char *what) {
        return cleanup(set_error(QADIC_E_CUDA, "%s: %s", what, cudaGetErrorString(cudaGetLastError())));
    };
    const size_t c_plane = (size_t)m * n;
    // Host A is `planes` planes of m x K elements of `esz` bytes; the device
    // copy holds block b's rows as planes of their own, blocks back to back.
    const bool planar = in_fmt != QADIC_FMT_LOG;
    const uint32_t planes = planar ? f.k : 1;
    const size_t esz = planar ? 1 : eb;
    const size_t pa_elem = path == QADIC_PATH_FP64_QADIC ? 8 : 2 * (size_t)f.k;
    int64_t r0[kMaxBlocks] = {0};
    for (int b = 1; b < nblk; ++b) r0[b] = r0[b - 1] + rows[b - 1];
    auto dA_blk = [&](int b) { return dA + (size_t)planes * r0[b] * K * esz; };
    auto pA_blk = [&](int b) { return pA + pa_elem * r0[b] * K; };
    auto copy_rows = [&](char *dst, int64_t first, int64_t nrows) -> cudaError_t {
        for (uint32_t i = 0; i < planes; ++i) {
            const cudaError_t e = cudaMemcpyAsync(
                dst + (size_t)i * nrows * K * esz,
                (const char *)A_host + ((size_t)i * m + first) * K * esz, (size_t)nrows * K * esz,
                cudaMemcpyHostToDevice, side);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const int opA = path == QADIC_PATH_FP64_QADIC ? QADIC_FMT_QADIC_F64 : QADIC_FMT_OPERAND_A;
    const int opB = path == QADIC_PATH_FP64_QADIC ? QADIC_FMT_QADIC_F64 : QADIC_FMT_OPERAND_B;
    // copies (side stream starts after everything already queued on `stream`)
    if (cudaEventRecord(ev_start, s) || cudaStreamWaitEvent(side, ev_start, 0) ||
        cudaMemcpyAsync(dB, B_host, eb * K * n, cudaMemcpyHostToDevice, side) ||
        cudaEventRecord(ev_b, side))
        return cuda_fail("H2D copy");
    for (int b = 0; b < nblk; ++b)
        if (copy_rows(dA_blk(b), r0[b], rows[b]) || cudaEventRecord(ev_copied[b], side))
            return cuda_fail("H2D copy");
    int st;
    // packs of the later blocks on the second side stream
    for (int b = 1; b < nblk; ++b) {
        if (cudaStreamWaitEvent(side2, ev_copied[b], 0)) return cuda_fail("wait");
        if ((st = qadic_pack(field, in_fmt, dA_blk(b), rows[b], K, K, opA, pA_blk(b), K, side2)))
            return cleanup(st);
        if (cudaEventRecord(ev_packed[b], side2)) return cuda_fail("event");
    }
    if (cudaStreamWaitEvent(s, ev_b, 0)) return cuda_fail("wait");
    if ((st = qadic_pack(field, in_fmt, dB, K, n, n, opB, pB, path == QADIC_PATH_FP64_QADIC ? n : K,
                         stream)))
        return cleanup(st);
    if (cudaStreamWaitEvent(s, ev_copied[0], 0)) return cuda_fail("wait");
    if ((st = qadic_pack(field, in_fmt, dA_blk(0), rows[0], K, K, opA, pA_blk(0), K, stream)))
        return cleanup(st);
    if (path == QADIC_PATH_FP64_QADIC) {
        if ((st = qadic_gemm(field, path, m, n, K, pA, K, pB, n, dC, n, nullptr, 0, stream)))
            return cleanup(st);
    } else {
        for (int b = 0; b < nblk; ++b) {
            if (b > 0 && cudaStreamWaitEvent(s, ev_packed[b], 0)) return cuda_fail("wait");
            if ((st = launch_gemm_planes_tc_strided(f, rows[b], n, K, pA_blk(b), K,
                                                    (int64_t)rows[b] * K, pB, K, (int64_t)n * K,
                                                    dC + r0[b] * n, n, (int64_t)c_plane, s)))
                return cleanup(st);
            if (b + 1 < nblk) {   // this block's C goes back while the next one is computed
                if (cudaEventRecord(ev_gemm[b], s) || cudaStreamWaitEvent(d2h, ev_gemm[b], 0))
                    return cuda_fail("event");
                for (uint32_t i = 0; i < f.k; ++i)
                    if (cudaMemcpyAsync(C_host + i * c_plane + r0[b] * n, dC + i * c_plane + r0[b] * n,
                                        (size_t)rows[b] * n, cudaMemcpyDeviceToHost, d2h))
                        return cuda_fail("D2H copy");
            }
        }
    }
    if (nblk > 1) {   // last block of every plane
        const int b = nblk - 1;
        for (uint32_t i = 0; i < f.k; ++i)
            if (cudaMemcpyAsync(C_host + i * c_plane + r0[b] * n, dC + i * c_plane + r0[b] * n,
                                (size_t)rows[b] * n, cudaMemcpyDeviceToHost, s))
                return cuda_fail("D2H copy");
    } else if (cudaMemcpyAsync(C_host, dC, (size_t)f.k * m * n, cudaMemcpyDeviceToHost, s)) {
        return cuda_fail("D2H copy");
    }
    // join: `stream` also waits for the side streams' copies
    if (cudaEventRecord(ev_join, side) || cudaStreamWaitEvent(s, ev_join, 0) ||
        cudaEventRecord(ev_d2h, d2h) || cudaStreamWaitEvent(s, ev_d2h, 0))
        return cuda_fail("join");
    return cleanup(QADIC_OK);
}

int qadic_redq(uint32_t p, uint32_t log2_q, uint32_t ndigits, const double *in, double *out,
               int64_t count, uint32_t table_mode, void *stream) {
    if (!is_prime(p) || p > 251) return set_error(QADIC_E_INVALID, "p must be a prime <= 251");
    if (log2_q < 1 || ndigits < 1 || ndigits > 51)
        return set_error(QADIC_E_INVALID, "bad log2_q or ndigits");
    if ((uint64_t)ndigits * log2_q > 51)
        return set_error(QADIC_E_OVERFLOW,
                         "ndigits*log2_q=%u exceeds 51 bits (Lemma 1 limit for binary64)",
                         ndigits * log2_q);
    if ((1ull << log2_q) <= p) return set_error(QADIC_E_INVALID, "q must exceed p");
    if (count < 0) return set_error(QADIC_E_INVALID, "negative count");
    if (count == 0) return QADIC_OK;
    if (!in || !out) return set_error(QADIC_E_INVALID, "NULL pointer");
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15))
        return set_error(QADIC_E_INVALID, "in/out must be 16-byte aligned");
    const uint32_t mode = table_mode & 0xff;
    if (mode > 3) return set_error(QADIC_E_INVALID, "table_mode %u", mode);
    return launch_redq(p, log2_q, ndigits, in, out, count, mode,
                       (table_mode & QADIC_REDQ_INT_FLOOR) != 0, (cudaStream_t)stream);
}

int qadic_redq_pq(uint32_t p, uint64_t q, uint32_t ndigits, const double *in, double *out,
                  int64_t count, uint32_t flags, void *stream) {
    if (!is_prime(p) || p > 251) return set_error(QADIC_E_INVALID, "p must be a prime <= 251");
    if (q < p || q % p != 0) return set_error(QADIC_E_INVALID, "q must be a multiple of p");
    if (ndigits < 1 || ndigits > 51) return set_error(QADIC_E_INVALID, "bad ndigits");
    unsigned __int128 qd = 1;
    for (uint32_t j = 0; j < ndigits && qd <= ((unsigned __int128)1 << 51); ++j) qd *= q;
    if (qd > ((unsigned __int128)1 << 51))
        return set_error(QADIC_E_OVERFLOW,
                         "q^ndigits exceeds 2^51 (Lemma 1 limit for binary64)");
    if ((flags & ~(QADIC_REDQ_INT_FLOOR | QADIC_REDQ_F32_DIGITS)) ||
        flags == (QADIC_REDQ_INT_FLOOR | QADIC_REDQ_F32_DIGITS))
        return set_error(QADIC_E_INVALID, "flags 0x%x", flags);
    if ((flags & QADIC_REDQ_F32_DIGITS) && (q > 1448 || ndigits > 8))   // 1448^2 < 2^21 < 1449^2
        return set_error(QADIC_E_UNSUPPORTED, "FP32 digits need q^2 < 2^21 and at most 8 digits");
    if (count < 0) return set_error(QADIC_E_INVALID, "negative count");
    if (count == 0) return QADIC_OK;
    if (!in || !out) return set_error(QADIC_E_INVALID, "NULL pointer");
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15))
        return set_error(QADIC_E_INVALID, "in/out must be 16-byte aligned");
    return launch_redq_pq(p, q, ndigits, in, out, count, (flags & QADIC_REDQ_INT_FLOOR) != 0,
                          (flags & QADIC_REDQ_F32_DIGITS) != 0, (cudaStream_t)stream);
}

int qadic_polymul_fqt_info(uint32_t p, uint32_t N, uint32_t d, uint32_t flags,
                           qadic_fqt_info *out) {
    if (!out) return set_error(QADIC_E_INVALID, "NULL info");
    if (flags & ~QADIC_FQT_INT_WORDS) return set_error(QADIC_E_INVALID, "flags 0x%x", flags);
    return fqt_parameters(p, N, d, (flags & QADIC_FQT_INT_WORDS) != 0, out);
}

int qadic_polymul_fqt(uint32_t p, uint32_t N, uint32_t d, const uint8_t *a, const uint8_t *b,
                      uint8_t *out, int64_t count, uint32_t flags, void *stream) {
    if (flags & ~QADIC_FQT_INT_WORDS) return set_error(QADIC_E_INVALID, "flags 0x%x", flags);
    qadic_fqt_info info;
    const int st = fqt_parameters(p, N, d, (flags & QADIC_FQT_INT_WORDS) != 0, &info);
    if (st != QADIC_OK) return st;
    if (count < 0) return set_error(QADIC_E_INVALID, "negative count");
    if (count == 0) return QADIC_OK;
    if (!a || !b || !out) return set_error(QADIC_E_INVALID, "NULL pointer");
    return launch_polymul_fqt(p, N, d, (flags & QADIC_FQT_INT_WORDS) != 0, a, b, out, count,
                              (cudaStream_t)stream);
}

int qadic_polymul_batched(uint32_t p, uint32_t k, const uint8_t *a, const uint8_t *b, uint8_t *out,
                          int64_t count, uint32_t flags, void *stream) {
    if (!is_prime(p) || p > 251) return set_error(QADIC_E_INVALID, "p must be a prime <= 251");
    if (k < 1 || k > kMaxK) return set_error(QADIC_E_INVALID, "k outside [1, 8]");
    if (count < 0) return set_error(QADIC_E_INVALID, "negative count");
    if (count == 0) return QADIC_OK;
    if (!a || !b || !out) return set_error(QADIC_E_INVALID, "NULL pointer");
    // q: the smallest power of two above k (p-1)^2 (Thm. 1 with n_q = 1).
    const uint64_t bound = (uint64_t)k * (p - 1) * (p - 1);
    uint32_t s = 1;
    while ((1ull << s) <= bound) ++s;
    if (flags & ~(QADIC_POLYMUL_PLAIN_F64 | QADIC_POLYMUL_INT_WORDS))
        return set_error(QADIC_E_INVALID, "flags 0x%x", flags);
    const bool plain = (flags & QADIC_POLYMUL_PLAIN_F64) != 0;
    const bool ints = (flags & QADIC_POLYMUL_INT_WORDS) != 0;
    if (plain && ints) return set_error(QADIC_E_INVALID, "PLAIN_F64 and INT_WORDS exclude each other");
    if (plain && (2 * k - 1) * s >= 53)
        return set_error(QADIC_E_OVERFLOW,
                         "(2k-1) log2 q = %u >= 53: Eq. 2 fails for a single-rounded FP64 product",
                         (2 * k - 1) * s);
    if (!plain && (2 * k - 1) * s > 63)
        return set_error(QADIC_E_OVERFLOW, "(2k-1) log2 q = %u > 63", (2 * k - 1) * s);
    if (!ints && k * s > 53)
        return set_error(QADIC_E_OVERFLOW, "k log2 q = %u > 53: a packed operand is not an exact double",
                         k * s);
    return launch_polymul(p, k, s, ints ? 2 : plain ? 1 : 0, a, b, out, count,
                          (cudaStream_t)stream);
}

int qadic_sync_status(void *stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    int *word = device_status_word();
    if (!word) return set_error(QADIC_E_CUDA, "status word unavailable");
    int v = 0;
    if (cudaMemcpy(&v, word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(QADIC_E_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    if (v != 0) {
        int zero = 0;
        cudaMemcpy(word, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return set_error(QADIC_E_DEVICE_TIMEOUT, "a bounded device wait ran out (site %d)", v);
    }
    return QADIC_OK;
}

const char *qadic_status_string(int status) {
    switch (status) {
        case QADIC_OK: return "ok";
        case QADIC_E_INVALID: return "invalid argument";
        case QADIC_E_NOT_PRIME: return "p is not prime";
        case QADIC_E_REDUCIBLE: return "defining polynomial is reducible";
        case QADIC_E_OVERFLOW: return "exactness bound violated";
        case QADIC_E_UNSUPPORTED: return "unsupported by this build";
        case QADIC_E_CUDA: return "CUDA error";
        case QADIC_E_DEVICE_TIMEOUT: return "device wait timed out";
        case QADIC_E_NOMEM: return "out of memory or workspace too small";
        default: return "unknown status";
    }
}

const char *qadic_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"

extern "C" {

size_t qadic_batched_workspace_size(const qadic_gemm_desc *descs, int64_t count) {
    return batched_workspace_size(descs, count);
}

size_t qadic_batched_workspace_size_fields(const qadic_field *const *fields, int32_t nfields,
                                           const qadic_gemm_desc *descs, int64_t count) {
    if (!fields || nfields < 1 || nfields > 64) return 0;
    const Field *fs[64];
    for (int32_t i = 0; i < nfields; ++i) {
        if (!fields[i]) return 0;
        fs[i] = &fields[i]->f;
    }
    return batched_workspace_size_fields(fs, nfields, descs, count);
}

int qadic_batched_gemm(const qadic_field *const *fields, int32_t nfields,
                       const qadic_gemm_desc *descs, int64_t count, void *workspace,
                       size_t ws_bytes, uint32_t flags, void *stream) {
    if (count < 0) return set_error(QADIC_E_INVALID, "negative count");
    if (count == 0) return QADIC_OK;
    if (!fields || !descs) return set_error(QADIC_E_INVALID, "NULL fields or descs");
    if (flags & ~QADIC_BATCHED_GRAPH) return set_error(QADIC_E_INVALID, "unknown flags");
    if (nfields < 1 || nfields > 64) return set_error(QADIC_E_INVALID, "nfields outside [1, 64]");
    const Field *fs[64];
    for (int32_t i = 0; i < nfields; ++i) {
        if (!fields[i]) return set_error(QADIC_E_INVALID, "field %d is NULL", i);
        fs[i] = &fields[i]->f;
    }
    return launch_batched(fs, nfields, descs, count, workspace, ws_bytes,
                          (flags & QADIC_BATCHED_GRAPH) != 0, (cudaStream_t)stream);
}

}  // extern "C"
