// Internal declarations shared by the host code and the kernel launchers of
// libqadic.  Nothing here is part of the public ABI (include/qadic.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "qadic.h"

namespace qadic {

constexpr uint32_t kMaxK = 8;

// Host + device copy of everything a field needs (Sec. 7: conversion tables
// between the log, polynomial and q-adic representations).
struct Field {
    uint32_t p = 0, k = 0, order = 0;       // order = p^k
    uint32_t poly[17] = {0};
    uint32_t gen[16] = {0};
    uint32_t log2_q = 0, n_q = 0;           // FP64 q-adic radix and block (Eq. 2)
    uint32_t h = 0;                         // centred bound (p-1)/2, 1 for p = 2
    int64_t k_max_int32 = 0;                // Eq. 3, 32-bit signed accumulator
    int64_t k_chunk_f32 = 0;                // exact FP32 accumulation chunk
    int device = 0;
    uint64_t uid = 0;                       // process-unique, never reused (keys of cached graphs)

    // Host tables.
    std::vector<uint8_t> antilog;           // order x k coefficients; row order-1 = zero
    std::vector<double> log_f64;            // log code -> sum c_i q^i
    std::vector<int8_t> log_centred;        // order x k centred coefficients
    std::vector<uint32_t> tab_L, tab_H;     // Thm. 3 tables (order entries, k bytes packed)
    std::vector<uint8_t> fold;              // (k-1) x k: X^(k+t) mod P, t = 0..k-2

    // Device copies (owned), from the allocator installed at init.
    qadic_free_fn table_free = nullptr;
    void *table_ctx = nullptr;
    uint8_t *d_antilog = nullptr;
    double *d_log_f64 = nullptr;
    int8_t *d_log_centred = nullptr;
    uint32_t *d_tab_L = nullptr, *d_tab_H = nullptr;
    uint8_t *d_fold = nullptr;
};

// The library-side field behind an opaque handle (capi.cu).
const Field *field_of(const qadic_field *handle);

// Field construction (field.cpp).
bool is_prime(uint32_t p);
bool poly_irreducible(uint32_t p, uint32_t k, const uint32_t *P);
int build_field(Field &f, uint32_t p, uint32_t k, const uint32_t *poly);  // qadic_status

// Error reporting (capi.cu).
int set_error(int status, const char *fmt, ...);
int *device_status_word();   // per-device bounded-wait status word (device address)

// Bound used by every wait loop in the kernels: after this many polls the
// kernel records QADIC_E_DEVICE_TIMEOUT in the status word and bails out.
constexpr uint32_t kSpinLimit = 1u << 26;

// ------------------------------------------------------------ launchers --
// Each returns a qadic_status after enqueueing on `stream`.

// mode 0: exact FP64 product (hi + lo), 1: single-rounded FP64 product,
// 2: 64-bit integer words.
int launch_polymul(uint32_t p, uint32_t k, uint32_t log2_q, int mode, const uint8_t *a,
                   const uint8_t *b, uint8_t *out, int64_t count, cudaStream_t stream);

int launch_redq(uint32_t p, uint32_t log2_q, uint32_t ndigits, const double *in, double *out,
                int64_t count, uint32_t table_mode, bool int_floor, cudaStream_t stream);

// 1/d rounded toward +infinity (d < 2^52), checked exactly (k_redq.cu).
double inv_up(uint64_t d);

// d-FQT long polynomial products (k_polyfqt.cu).
int fqt_parameters(uint32_t p, uint32_t N, uint32_t d, bool int_words, qadic_fqt_info *info);
int launch_polymul_fqt(uint32_t p, uint32_t N, uint32_t d, bool int_words, const uint8_t *a,
                       const uint8_t *b, uint8_t *out, int64_t count, cudaStream_t stream);

// REDQ with q a multiple of p (q^ndigits <= 2^51): no correction step.
int launch_redq_pq(uint32_t p, uint64_t q, uint32_t ndigits, const double *in, double *out,
                   int64_t count, bool int_floor, bool f32_digits, cudaStream_t stream);

int launch_pack(const Field &f, int in_fmt, const void *in, int64_t rows, int64_t cols,
                int64_t ld_in, int out_fmt, void *out, int64_t ld_out, cudaStream_t stream);

int launch_pack_pair(const Field &f, int in_fmt, const void *A, int64_t m, int64_t K,
                     int64_t lda_in, void *outA, int64_t lda_out, const void *B, int64_t n,
                     int64_t ldb_in, void *outB, int64_t ldb_out, cudaStream_t stream,
                     bool e4m3 = false);

int launch_gemm_f64(const Field &f, int64_t m, int64_t n, int64_t K, const double *A, int64_t lda,
                    const double *B, int64_t ldb, uint8_t *C, int64_t ldc, cudaStream_t stream);

int launch_gemm_planes_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                          int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                          cudaStream_t stream, bool fp8 = false);

// Same, with explicit element strides between the k planes of A, B and C
// (row ranges of k-plane matrices).
int launch_gemm_planes_tc_strided(const Field &f, int64_t m, int64_t n, int64_t K,
                                  const void *A, int64_t lda, int64_t a_plane, const void *B,
                                  int64_t ldb, int64_t b_plane, uint8_t *C, int64_t ldc,
                                  int64_t c_plane, cudaStream_t stream, bool fp8 = false);

bool gemm_planes_tc_supported(const Field &f);

// Fold-before form: rows of one output block in an OPERAND_B_FOLD plane.
inline int64_t fold_n_pad(int64_t n) { return (n + 255) / 256 * 256; }

int launch_gemm_karatsuba_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                             int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                             cudaStream_t stream);

int launch_gemm_fold_tc(const Field &f, int64_t m, int64_t n, int64_t K, const void *A,
                        int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                        cudaStream_t stream);

size_t batched_workspace_size(const qadic_gemm_desc *descs, int64_t count);
size_t batched_workspace_size_fields(const Field *const *fields, int32_t nfields,
                                     const qadic_gemm_desc *descs, int64_t count);

int launch_batched(const Field *const *fields, int32_t nfields, const qadic_gemm_desc *descs,
                   int64_t count, void *workspace, size_t ws_bytes, bool use_graph,
                   cudaStream_t stream);

int batched_tile_configs(uint32_t k, qadic_tile_config *out, int32_t capacity, int32_t *n);
int batched_select_tiles(uint32_t k, int32_t index);
int batched_selected_tiles(uint32_t k, int32_t *index);
int autotune_batched(const Field *const *fields, int32_t nfields, const qadic_gemm_desc *descs,
                     int64_t count, void *workspace, size_t ws_bytes, int32_t reps,
                     int32_t *chosen, cudaStream_t stream);

}  // namespace qadic
