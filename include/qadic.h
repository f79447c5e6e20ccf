/*
 * qadic.h -- C ABI of the GB300 (sm_103a) library for matrix multiplication
 * over small extension fields GF(p^k) through the q-adic transform
 * ("Q-adic Transform Revisited", J.-G. Dumas).
 *
 * Conventions shared by every call
 * --------------------------------
 * Field.   GF(p^k) = Z_p[X]/(P), P monic irreducible of degree k; an element is
 *          the coefficient vector (c_0..c_{k-1}), c_i in [0, p-1]  (Sec. 7).
 *          Discrete-log codes: code e in [0, p^k-2] is g^e for the field's
 *          generator g; code p^k-1 is zero (Sec. 7, Alg. 4's input requirement).
 * Planes.  A "k-plane" matrix of rows x cols stores coefficient i of every
 *          element in plane i: element (r, c) of plane i is at
 *          base + (i * rows + r) * ld + c, i.e. planes are contiguous blocks
 *          of rows * ld elements.
 * Memory.  Every data pointer is a DEVICE pointer (cudaMalloc, or a torch
 *          CUDA tensor) unless the name ends in _host.  The caller owns all
 *          data buffers and workspaces; the library owns only the field
 *          handle and the device tables it uploads at qadic_field_init and
 *          frees at qadic_field_destroy.  Those tables are the only device
 *          memory the library allocates; qadic_set_device_allocator lets the
 *          caller supply that memory.
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *          stream).  Calls that take a stream only enqueue work and return.
 * Errors.  Every call returns a qadic_status.  Argument, size, alignment and
 *          exactness-bound violations are detected on the host before
 *          anything is enqueued; outputs are then left untouched ("overflow
 *          rejected rather than miscomputed").  A CUDA launch error returns
 *          QADIC_E_CUDA.  Device-side conditions (a bounded wait that ran
 *          out) set a per-device status word read by qadic_sync_status.
 *          qadic_last_error() gives a one-line description of the last
 *          failure on the calling thread.
 * Threads. Field handles are immutable after init and may be shared by
 *          threads and streams.
 */
#ifndef QADIC_H
#define QADIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QADIC_OK = 0,
    QADIC_E_INVALID = 1,        /* bad argument, size, stride or alignment */
    QADIC_E_NOT_PRIME = 2,      /* p is not prime */
    QADIC_E_REDUCIBLE = 3,      /* the given P is not irreducible mod p */
    QADIC_E_OVERFLOW = 4,       /* an exactness bound (Eq. 2, Lemma 1, Eq. 3) fails */
    QADIC_E_UNSUPPORTED = 5,    /* valid request this build has no kernel for */
    QADIC_E_CUDA = 6,           /* a CUDA runtime call failed */
    QADIC_E_DEVICE_TIMEOUT = 7, /* a bounded device wait ran out (qadic_sync_status) */
    QADIC_E_NOMEM = 8           /* host or device allocation failed, or workspace too small */
} qadic_status;

/* Element formats accepted / produced by qadic_pack. */
typedef enum {
    QADIC_FMT_LOG = 0,        /* one discrete-log code per element: uint8 when p^k <= 256, else uint16 */
    QADIC_FMT_COEFF_U8 = 1,   /* k planes of uint8 coefficients in [0, p-1] */
    QADIC_FMT_INT8_PLANES = 2,/* k planes of int8 coefficients, any representative mod p */
    QADIC_FMT_QADIC_F64 = 3,  /* one double per element: sum_i c_i q^i, c_i in [0, p-1] (Eq. 1) */
    QADIC_FMT_OPERAND_A = 4,  /* k planes of bf16 centred coefficients, rows x cols (K contiguous) */
    QADIC_FMT_OPERAND_B = 5,  /* k planes of bf16 centred coefficients, TRANSPOSED: cols x rows */
    QADIC_FMT_OPERAND_B_FOLD = 6,/* k planes i, each k blocks j of n_pad rows: plane j of B X^i mod P,
                                    TRANSPOSED (K contiguous); n_pad = cols rounded up to 256 */
    QADIC_FMT_OPERAND_A_KARA = 7,/* k = 2: 3 bf16 planes c_0, c_1, (c_0 + c_1) mod p, centred, rows x cols */
    QADIC_FMT_OPERAND_B_KARA = 8,/* k = 2: the same 3 planes, TRANSPOSED: cols x rows */
    QADIC_FMT_OPERAND_A_E4M3 = 9,/* p <= 31: k planes of fp8 e4m3 centred coefficients (one byte
                                    each; |c| <= 15 is exact), rows x cols (K contiguous) */
    QADIC_FMT_OPERAND_B_E4M3 = 10/* p <= 31: the same, TRANSPOSED: cols x rows */
} qadic_format;

/* Contraction forms of qadic_gemm. */
typedef enum {
    QADIC_PATH_FP64_QADIC = 0, /* FP64 q-adic GEMM, REDQ after every n_q-product K-block (Alg. 4) */
    QADIC_PATH_PLANES = 1,     /* k x k coefficient-plane tensor-core GEMMs + fused mod-p / mod-P epilogue */
    QADIC_PATH_FOLD = 2,       /* fold-before: B's multiplication matrices, one prime-field tensor-core GEMM */
    QADIC_PATH_KARATSUBA = 3,  /* k = 2: three plane products (Karatsuba) on the tensor cores */
    QADIC_PATH_PLANES_E4M3 = 4 /* p <= 31: the plane path on fp8 e4m3 operands (kind::f8f6f4) */
} qadic_path;

/* Field description returned by qadic_field_info. */
typedef struct {
    uint32_t p, k;
    uint32_t poly[17];        /* P, k+1 coefficients low -> high (poly[k] == 1) */
    uint32_t generator[16];   /* coefficients of g */
    uint32_t order;           /* p^k */
    uint32_t zero_code;       /* p^k - 1 */
    uint32_t log_bytes;       /* 1 or 2: width of a QADIC_FMT_LOG code */
    uint32_t log2_q;          /* FP64 q-adic radix q = 2^log2_q (Eq. 2 with m = 53) */
    uint32_t n_q;             /* products per K-block of the FP64 path (Eq. 2); 0 = path unavailable */
    uint32_t reserved;
    int64_t k_max_int32;      /* Eq. 3 with centred planes and a 32-bit signed accumulator */
    int64_t k_chunk_f32;      /* K per exact FP32 tensor-core accumulation chunk */
} qadic_info;

/* One product of qadic_batched_gemm: C = A * B over fields[field].
 * A: k-plane COEFF_U8 m x K (ld = lda), B: k-plane COEFF_U8 K x n (ld = ldb),
 * C: k-plane COEFF_U8 m x n (ld = ldc).  All device pointers.  Input bytes
 * at or above p are taken mod p; C holds coefficients in [0, p). */
typedef struct {
    int32_t field;            /* index into the fields array */
    int32_t m, n, K;
    const uint8_t *A;
    const uint8_t *B;
    uint8_t *C;
    int32_t lda, ldb, ldc;
    int32_t reserved;
} qadic_gemm_desc;

typedef struct qadic_field qadic_field;

/* ---------------------------------------------------------------- field --
 * qadic_field_init: build GF(p^k) on the current CUDA device.
 *   p     prime, 2 <= p <= 251 (coefficients fit a byte).
 *   k     1 <= k <= 8, p^k <= 65536.
 *   poly  k+1 coefficients low -> high, monic, or NULL for the default: the
 *         monic irreducible whose low coefficients have the smallest value
 *         sum_i a_i p^i.  (Sec. 7: the field as polynomials modulo p and
 *         modulo an irreducible P of degree k.)
 *   flags 0, or QADIC_FIELD_HOST_ONLY: build the field and its tables on the
 *         host only (no device upload, no CUDA call); such a handle serves
 *         qadic_field_info and is rejected by every call that launches work.
 * Host side: checks p prime (QADIC_E_NOT_PRIME) and P irreducible
 * (QADIC_E_REDUCIBLE), picks the generator (smallest primitive element),
 * derives q and n_q from Eq. 2, the Eq. 3 K bound, and builds the tables of
 * Sec. 5-6: log -> q-adic FP64 word, log -> centred planes, the Thm. 3 L/H
 * correction-and-fold tables and X^t mod P; then uploads them (owned by the
 * handle).  *out is set only on success. */
#define QADIC_FIELD_HOST_ONLY 0x1u
int qadic_field_init(qadic_field **out, uint32_t p, uint32_t k, const uint32_t *poly,
                     uint32_t flags);
/* Frees the handle and its device tables.  The caller must ensure no queued
 * work still uses the field.  NULL is accepted. */
int qadic_field_destroy(qadic_field *field);

/* ------------------------------------------------------ device allocator --
 * Not from the paper: a property of the library.  The device tables of a
 * field are the only device memory the library allocates itself.  A caller
 * whose own allocator owns the device memory (a framework's caching
 * allocator) installs it here; qadic_field_init then asks `alloc` for every
 * table, before any other CUDA call, and qadic_field_destroy (or a failed
 * init) hands each table back to the `free_fn` that was installed when the
 * field was built.
 *   alloc(&ptr, bytes, ctx) returns QADIC_OK with ptr set to at least
 *     `bytes` bytes of device memory on the current device (256-byte
 *     aligned), or QADIC_E_NOMEM / QADIC_E_CUDA; qadic_field_init then
 *     returns that status after giving back the tables it already got.
 *   free_fn(ptr, bytes, ctx) releases one table.
 *   alloc = free_fn = NULL restores cudaMalloc / cudaFree (the default).
 * Process-wide; fields built earlier keep the allocator they were built
 * with, so free_fn and ctx must stay valid until every such field has been
 * destroyed.  QADIC_E_INVALID when exactly one of alloc, free_fn is NULL. */
typedef int (*qadic_alloc_fn)(void **ptr, size_t bytes, void *ctx);
typedef void (*qadic_free_fn)(void *ptr, size_t bytes, void *ctx);
int qadic_set_device_allocator(qadic_alloc_fn alloc, qadic_free_fn free_fn, void *ctx);
/* Copies the field description into *out (host memory). */
int qadic_field_info(const qadic_field *field, qadic_info *out);

/* ----------------------------------------------------------------- pack --
 * DQT (Sec. 2, Alg. 1's packing; Alg. 4's pack step with the Sec. 7 improvement:
 * one table lookup instead of a Horner evaluation).  Converts a rows x cols
 * matrix from in_fmt to out_fmt.
 *   in, ld_in    input in in_fmt (element stride per row = ld_in elements)
 *   out, ld_out  output in out_fmt; for QADIC_FMT_OPERAND_B the output is the
 *                transpose (cols x rows, ld_out >= rows); for
 *                QADIC_FMT_OPERAND_B_FOLD (a K x n matrix B: rows = K,
 *                cols = n) it is k planes i of k * n_pad rows of ld_out
 *                elements, n_pad = (n + 255) / 256 * 256: row j * n_pad + c
 *                of plane i holds coefficient j of B[:, c] * X^i mod P,
 *                centred, with zero rows for c >= n (the matrix b -> b X^i
 *                mod P of Thm. 3's fold applied before the product)
 * QADIC_FMT_OPERAND_A_KARA / _B_KARA (k = 2) write three planes like
 * OPERAND_A / OPERAND_B: c_0, c_1 and (c_0 + c_1) mod p, centred.
 * Supported pairs: LOG -> QADIC_F64 | OPERAND_A | OPERAND_B | OPERAND_B_FOLD |
 * OPERAND_A_KARA | OPERAND_B_KARA | COEFF_U8; COEFF_U8 or INT8_PLANES ->
 * QADIC_F64 | OPERAND_A | OPERAND_B | OPERAND_B_FOLD | OPERAND_A_KARA |
 * OPERAND_B_KARA.
 * Errors: QADIC_E_INVALID (format pair, ld < cols, NULL), QADIC_E_OVERFLOW
 * (QADIC_F64 requested but Eq. 2 has no q with n_q >= 1).
 * OPERAND formats need ld_out a multiple of 8 (of 16 for the E4M3 ones) and
 * 16-byte aligned bases; the E4M3 ones need p <= 31 (QADIC_E_UNSUPPORTED). */
int qadic_pack(const qadic_field *field, int in_fmt, const void *in, int64_t rows, int64_t cols,
               int64_t ld_in, int out_fmt, void *out, int64_t ld_out, void *stream);

/* ----------------------------------------------------------------- gemm --
 * C = A * B over GF(p^k) (Alg. 4 applied to every row/column pair, the
 * numerical routine being a GEMM, Sec. 7).  m x K times K x n.
 * QADIC_PATH_FP64_QADIC: A is QADIC_F64 m x K (lda), B is QADIC_F64 K x n
 *   (ldb).  K is cut into blocks of n_q products (Eq. 2); after each block
 *   the packed sums go through REDQ (Alg. 2 with Lemma 1's floor) and the
 *   two Thm. 3 table lookups, and the block results are added mod p.
 * QADIC_PATH_PLANES: A is OPERAND_A (k planes, m x K, lda), B is OPERAND_B
 *   (k planes, n x K, ldb).  The 2k-1 plane sums C_t = sum_{i+j=t} A_i B_j
 *   (Eq. 1 coefficientwise) are accumulated exactly on the tensor cores in
 *   K-chunks of at most k_chunk_f32, reduced mod p, and folded mod P with
 *   X^t mod P in the epilogue.  lda, ldb multiples of 8.
 * QADIC_PATH_PLANES_E4M3 (p <= 31): the same contraction on A in
 *   OPERAND_A_E4M3 and B in OPERAND_B_E4M3 (one byte per coefficient;
 *   |c| <= 15 is exact in e4m3), through tcgen05 kind::f8f6f4 MMAs with FP32
 *   accumulators: half the operand bytes of the bf16 planes and twice the
 *   tensor rate.  lda, ldb multiples of 16; QADIC_E_UNSUPPORTED for p > 31.
 * QADIC_PATH_FOLD: A is OPERAND_A, B is OPERAND_B_FOLD (ldb >= K, multiple
 *   of 8).  out_j = sum_i A_i M_ij(B) with M_ij(B) plane j of B X^i mod P:
 *   the reduction mod P happens before the contraction (the same map Thm. 3
 *   tabulates after it), which is one prime-field GEMM over k K with the k
 *   output planes side by side; one exact FP32 accumulator per plane i,
 *   reduced mod p in the epilogue.  Any k from 1 to 8 (k = 1: GF(p)).
 * QADIC_PATH_KARATSUBA (k = 2): A is OPERAND_A_KARA (lda), B is
 *   OPERAND_B_KARA (ldb).  Karatsuba's identity on the coefficient planes:
 *   D_0 = A_0 B_0, D_2 = A_1 B_1, D_m = (A_0 + A_1)(B_0 + B_1), so
 *   C_1 = D_m - D_0 - D_2 -- three plane products instead of four; each in
 *   its own exact FP32 accumulator, combined and folded with X^2 mod P in
 *   the epilogue.
 * C: k planes of uint8 in [0, p-1], m x n (ldc).
 * workspace/ws_bytes: unused by these kernels (pass NULL, 0).
 * Errors: QADIC_E_INVALID, QADIC_E_OVERFLOW (FP64 path with n_q = 0),
 * QADIC_E_UNSUPPORTED (plane path for a k without a tensor-core kernel). */
int qadic_gemm(const qadic_field *field, int path, int64_t m, int64_t n, int64_t K,
               const void *A, int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
               void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------- pack_operands --
 * Both operands of the plane path at once: A (m x K) -> OPERAND_A (outA,
 * lda_out) and B (K x n) -> OPERAND_B (outB, ldb_out), as two qadic_pack
 * calls would.  Coefficient-plane inputs with K % 16 == 0, n % 64 == 0 and
 * 16-byte aligned rows are packed by ONE launch; other inputs by two.
 * lda_out, ldb_out >= K, multiples of 8; 16-byte aligned outputs. */
int qadic_pack_operands(const qadic_field *field, int in_fmt, const void *A, int64_t m, int64_t K,
                        int64_t lda_in, void *outA, int64_t lda_out, const void *B, int64_t n,
                        int64_t ldb_in, void *outB, int64_t ldb_out, void *stream);

/* The same for the e4m3 plane path (p <= 31, else QADIC_E_UNSUPPORTED):
 * A -> OPERAND_A_E4M3 and B -> OPERAND_B_E4M3, one launch under the same
 * conditions; lda_out, ldb_out >= K, multiples of 16; 16-byte aligned
 * outputs. */
int qadic_pack_operands_e4m3(const qadic_field *field, int in_fmt, const void *A, int64_t m,
                             int64_t K, int64_t lda_in, void *outA, int64_t lda_out, const void *B,
                             int64_t n, int64_t ldb_in, void *outB, int64_t ldb_out, void *stream);

/* ----------------------------------------------------------------- matmul --
 * The whole path on device operands in one call: A (m x K) and B (K x n) in
 * in_fmt (LOG, COEFF_U8 or INT8_PLANES; lda, ldb element strides per row,
 * planes of a plane format `rows * ld` elements apart), packed into
 * `workspace` (device, 256-byte aligned, at least
 * qadic_matmul_device_workspace_size bytes) and multiplied with `path`
 * (any of the five); C: k planes of uint8, m x n (ldc).  For the plane path
 * with plane inputs both operands are packed by one launch.  Errors as for
 * qadic_pack and qadic_gemm, QADIC_E_NOMEM for a short workspace. */
size_t qadic_matmul_device_workspace_size(const qadic_field *field, int path, int64_t m,
                                          int64_t n, int64_t K);
int qadic_matmul(const qadic_field *field, int path, int in_fmt, int64_t m, int64_t n, int64_t K,
                 const void *A, int64_t lda, const void *B, int64_t ldb, uint8_t *C, int64_t ldc,
                 void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------ matmul_host --
 * End-to-end convenience: A (m x K) and B (K x n) in in_fmt (LOG, COEFF_U8 or
 * INT8_PLANES) in HOST memory (pinned for asynchrony), C (k planes of uint8,
 * m x n) in HOST memory.  Copies the inputs into `workspace` (device, at
 * least qadic_matmul_workspace_size bytes), packs, multiplies with `path`,
 * and copies C back, all enqueued on `stream`.  Dense leading dimensions.
 * path: QADIC_PATH_FP64_QADIC or QADIC_PATH_PLANES (K % 8 == 0). */
size_t qadic_matmul_workspace_size(const qadic_field *field, int path, int in_fmt, int64_t m,
                                   int64_t n, int64_t K);
int qadic_matmul_host(const qadic_field *field, int path, int in_fmt, int64_t m, int64_t n,
                      int64_t K, const void *A_host, const void *B_host, uint8_t *C_host,
                      void *workspace, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------------- redq --
 * REDQ (Alg. 2) on `count` packed words in[i] = sum_{j<=d} mu~_j q^j with
 * q = 2^log2_q, d = ndigits-1, each an exact non-negative integer held in a
 * double.  Writes out[i] = rho = sum_j (mu~_j mod p) q^j (exact, as double).
 * rop = floor(r/p) by Lemma 1 (multiplication by 1/p rounded upward, then
 * floor) or, with QADIC_REDQ_INT_FLOOR, by an integer multiply-high; the
 * u_j by shifts; the corrections mu_j = (u_j - q u_{j+1}) mod p per
 * table_mode (Table 1): 0 arithmetic, 1 a p^2 table (d lookups), 2 a p^k'
 * table (ceil(d/(k'-1)) lookups, largest k' fitting shared memory), 3 the
 * full p^(d+1) table (one lookup) when it fits.
 * Requires ndigits * log2_q <= 51 (Lemma 1's limit 1/(2eps+eps^2) with
 * eps = 2^-52), else QADIC_E_OVERFLOW; in/out 16-byte aligned; may alias. */
#define QADIC_REDQ_INT_FLOOR 0x100u
int qadic_redq(uint32_t p, uint32_t log2_q, uint32_t ndigits, const double *in, double *out,
               int64_t count, uint32_t table_mode, void *stream);

/* -------------------------------------------------------------- redq_pq --
 * REDQ (Alg. 2) for q a multiple of p, the other choice of q that the
 * paper's conclusion leaves to compare (q = 10^4, p = 5 in Ex. 2).  Since
 * -q = 0 mod p the corrections of Alg. 2 vanish and mu_j = u_j (Thm. 2): no
 * table.  The divisions by q^j (no longer shifts) are taken as a chain
 * t_{j+1} = floor(t_j / q) (Lemma 2), each a Lemma 1 floor by 1/q rounded
 * upward, or with QADIC_REDQ_INT_FLOOR an integer multiply-high; then
 * u_j = t_j mod p = (t_j - q t_{j+1}) mod p since p | q.  Where q^s < 2^32
 * for the first s with q^(ndigits-s) <= 2^32, the chain starts with one such
 * floor by q^s, and the floors of r mod q^s and of t_s below 2^32 are 32-bit
 * integer ones (exact, so the flag then only picks the floor by q^s).
 * With QADIC_REDQ_F32_DIGITS (q^2 < 2^21, at most 8 digits, else
 * QADIC_E_UNSUPPORTED) the word is cut into chunks of two base-q digits by
 * integer floors by q^2, and the floors by q and by p inside a chunk
 * (below 2^21) are exact FP32 ones: the same rho, with no FP64 arithmetic.
 * in[i] = sum_{j<=d} mu~_j q^j with 0 <= mu~_j < q, d = ndigits-1, an exact
 * integer held in a double; out[i] = rho = sum_j (mu~_j mod p) q^j (exact).
 * Requires p prime <= 251, q >= p with p | q, q^ndigits <= 2^51 (else
 * QADIC_E_OVERFLOW: Lemma 1's limit), flags 0, QADIC_REDQ_INT_FLOOR or
 * QADIC_REDQ_F32_DIGITS (one of them), in/out 16-byte aligned device
 * pointers (may alias).  Words at or above q^ndigits give unspecified values
 * without faulting. */
#define QADIC_REDQ_F32_DIGITS 0x200u
int qadic_redq_pq(uint32_t p, uint64_t q, uint32_t ndigits, const double *in, double *out,
                  int64_t count, uint32_t flags, void *stream);

/* ---------------------------------------------------------- polymul_fqt --
 * Products of long polynomials in Z_p[X] by the d-FQT (Sec. 6, Table 2).
 * a, b: count polynomials of degree N, N+1 uint8 coefficients each (lowest
 * first; values are reduced mod p).  out: count x (2N+1) uint8 coefficients
 * in [0, p-1].  Device pointers, owned by the caller.
 * Each polynomial is cut into D_q+1 blocks of d+1 coefficients packed into
 * one word each (Y = X^(d+1), q = 2^log2_q); the word convolution is summed
 * exactly and reduced by REDQ_{2d+1} (Alg. 2) after at most n_q products,
 * the reduced word being fed back into the sum; overlapping block digits
 * are added mod p.  d = 0 is the classical algorithm with delayed
 * reduction.  Words (flags):
 *   0                    binary64, the paper's choice: (2d+1) log2_q <= 51
 *                        (Lemma 1's limit), floor(r/p) by Lemma 1;
 *   QADIC_FQT_INT_WORDS  64-bit integers with 32-bit operands (Sec. 2 allows
 *                        m = 64): (d+1) log2_q <= 32, (2d+1) log2_q <= 64,
 *                        floor(r/p) by an integer multiply-high.
 * n_q is the largest integer with q > n_q (d+1)(p-1)^2 + (p-1) (Eq. 2 with
 * k = d+1, plus room for the fed-back word).  Errors: QADIC_E_INVALID (p not
 * a prime <= 251, d > 24, bad flags, NULL with count > 0), QADIC_E_OVERFLOW
 * (n_q = 0 for this d), QADIC_E_UNSUPPORTED (N too large for one CTA's
 * shared memory: about 200 KB for the words and residue sums). */
#define QADIC_FQT_INT_WORDS 0x1u
typedef struct qadic_fqt_info {
    uint32_t log2_q;           /* q = 2^log2_q */
    uint32_t n_q;              /* products summed between reductions (capped at 2^32-1) */
    uint32_t D_q;              /* blocks per polynomial, minus one: ceil((N+1)/(d+1)) - 1 */
    uint32_t word_bits;        /* 53 (binary64) or 64 */
    uint64_t word_products;    /* (D_q+1)^2 word multiply-adds per polynomial product */
} qadic_fqt_info;
/* Host only: the parameters qadic_polymul_fqt would use (same errors). */
int qadic_polymul_fqt_info(uint32_t p, uint32_t N, uint32_t d, uint32_t flags,
                           qadic_fqt_info *out);
int qadic_polymul_fqt(uint32_t p, uint32_t N, uint32_t d, const uint8_t *a, const uint8_t *b,
                      uint8_t *out, int64_t count, uint32_t flags, void *stream);

/* ------------------------------------------------------ polymul_batched --
 * Alg. 1 on `count` independent pairs in Z_p[X] (no defining polynomial):
 * a, b: count x k uint8 coefficients in [0, p-1] (pair s at a + s*k);
 * out: count x (2k-1) uint8, the product's coefficients mod p.
 * q = the smallest power of two above k (p-1)^2 (one product, n_q = 1);
 * pack by shifts, product in FP64, REDQ in 64-bit words (Sec. 2 allows
 * 64-bit machine words).  With QADIC_POLYMUL_PLAIN_F64 the product is the
 * single-rounded FP64 product and Eq. 2 (m = 53) must hold, else
 * QADIC_E_OVERFLOW.  Otherwise the product is made exact with an FMA
 * error term (hi + lo), which needs (2k-1) log2 q <= 63 and k log2 q <= 53.
 * With QADIC_POLYMUL_INT_WORDS the packed words are multiplied as 64-bit
 * integers instead (exact while (2k-1) log2 q <= 63). */
#define QADIC_POLYMUL_PLAIN_F64 0x1u
#define QADIC_POLYMUL_INT_WORDS 0x2u
int qadic_polymul_batched(uint32_t p, uint32_t k, const uint8_t *a, const uint8_t *b, uint8_t *out,
                          int64_t count, uint32_t flags, void *stream);

/* -------------------------------------------------------- batched_gemm --
 * `count` independent products descs[i] over fields[descs[i].field] in ONE
 * persistent launch (tiles of all products on a device work list).
 * Requires 1 <= m, n, K <= 4096 per product, k <= 8.  `workspace` (device,
 * 256-byte aligned) must hold at least qadic_batched_workspace_size(descs,
 * count) bytes: the host packs the work list into it, and the operand bytes
 * are staged through registers tile by tile (warp-level bf16 MMAs).  With
 * at least qadic_batched_workspace_size_fields(fields, nfields, descs, count)
 * bytes the tensor-core path runs instead: one launch converts every operand
 * once to centred planes in the workspace -- fp8 e4m3 for p <= 31 (exact:
 * |c| <= 15), bf16 for larger p -- cut into the blocks the MMAs read (B
 * transposed), and a persistent tcgen05 kernel copies them into shared
 * memory and accumulates the plane sums in FP32 in tensor memory (128-row
 * tiles, 128 / k output columns per tile, rounded to the sizes in tc_bn of
 * the implementation), reducing them in place at every exact chunk.
 * Both paths give the same bytes.  The size query with fields returns 0 for
 * invalid arguments.  With QADIC_BATCHED_GRAPH the launch is captured in
 * a CUDA graph keyed by (descs, count, workspace) and replayed on later calls
 * with the same key (and the same tile configurations); a replay first
 * re-uploads its own work list if another call wrote a different one into
 * the same workspace.  Tiles of the register-staged path: for each field the
 * configuration selected for its k (qadic_batched_select_tiles /
 * qadic_batched_autotune below), or configuration 0.  Errors:
 * QADIC_E_INVALID (including a list of more tiles than the work queue
 * indexes), QADIC_E_NOMEM (workspace too small), QADIC_E_OVERFLOW (exact
 * FP32 chunk of a field below 32). */
#define QADIC_BATCHED_GRAPH 0x1u
size_t qadic_batched_workspace_size(const qadic_gemm_desc *descs, int64_t count);
size_t qadic_batched_workspace_size_fields(const qadic_field *const *fields, int32_t nfields,
                                           const qadic_gemm_desc *descs, int64_t count);
int qadic_batched_gemm(const qadic_field *const *fields, int32_t nfields,
                       const qadic_gemm_desc *descs, int64_t count, void *workspace,
                       size_t ws_bytes, uint32_t flags, void *stream);

/* ----------------------------------------------- batched tile autotuning --
 * The register-staged batched kernel (the path of work-list-only workspaces
 * and of qadic_batched_gemm_noalloc) can run each product with one of a few
 * tile configurations per field degree k (the shapes whose 2k-1 accumulator
 * sets fit in registers): output tile bm x bn, K-block bk, and the shared
 * memory it needs.  Configuration 0 is the default.  No counterpart in the
 * paper (it concerns the GPU schedule, not the arithmetic).  The autotuner
 * always times that kernel (it offers the batch the work-list part of the
 * workspace only).
 * qadic_batched_tile_configs: writes min(capacity, n) entries of the table
 *   for k and sets *count = n.
 * qadic_batched_select_tiles: process-wide choice for fields with k
 *   coefficients (index -1 restores the default).  A field whose exact FP32
 *   chunk is shorter than the chosen bk runs configuration 0.
 * qadic_batched_autotune: for each k present in `descs` (largest total work
 *   first), runs the whole batch with every configuration -- a graph
 *   capture as warm-up, then `reps` graph replays timed with CUDA events on
 *   `stream` -- selects the fastest and writes it to chosen[k] (chosen has
 *   9 entries; -1 for an absent k).  It synchronizes `stream`, and the
 *   outputs hold the products (every configuration computes them exactly).
 *   Arguments as for qadic_batched_gemm; reps in [1, 1000]. */
typedef struct qadic_tile_config {
    int32_t bm, bn, bk;
    int32_t smem_bytes;
} qadic_tile_config;
int qadic_batched_tile_configs(uint32_t k, qadic_tile_config *out, int32_t capacity,
                               int32_t *count);
int qadic_batched_select_tiles(uint32_t k, int32_t index);
int qadic_batched_selected_tiles(uint32_t k, int32_t *index);
int qadic_batched_autotune(const qadic_field *const *fields, int32_t nfields,
                           const qadic_gemm_desc *descs, int64_t count, void *workspace,
                           size_t ws_bytes, int32_t reps, int32_t *chosen, void *stream);

/* ------------------------------------------------ batched_gemm_noalloc --
 * The same products as qadic_batched_gemm (same descriptors, same results),
 * for callers that must not allocate memory during the call: code running
 * under a framework whose allocator owns all device memory, latency-bound
 * loops where cudaMalloc/cudaFree would synchronise the device, or plugins
 * that are handed only their input and output buffers and no workspace.
 * The paper has no counterpart; this is a property of the library only.
 *   The work list is kept in a fixed 8 MiB device array inside the library
 *   (built on the host in a fixed host array of the same size); no device or
 *   host memory is allocated and no allocating routine is called.  Every
 *   device that loads the library holds that array until the process exits.
 *   The first call on a device does the set-up: it looks up the array's
 *   device address and creates one event (no memory allocation).
 *   All calls share the one array and each call rewrites it from the start
 *   (the tile counter included), so calls whose kernels overlap on the GPU
 *   race: order them on one stream, or synchronise in between.  A call
 *   waits on the host until the previous call's upload of the work list
 *   has read the host array, then rewrites it.
 *   QADIC_E_INVALID when the work list would exceed the array (about
 *   8 MiB / 8 bytes per 32 x 16 output tile); use qadic_batched_gemm then. */
int qadic_batched_gemm_noalloc(const qadic_field *const *fields, int32_t nfields,
                               const qadic_gemm_desc *descs, int64_t count, void *stream);

/* ------------------------------------------------------------- selftest --
 * Diagnostic with no counterpart in the paper.  It exercises the failure
 * path of the bounded device waits that every kernel here uses: one warp
 * waits on a fresh mbarrier that nothing arrives on, gives up after `polls`
 * polls (1 <= polls <= 2^26), records QADIC_E_DEVICE_TIMEOUT in the status
 * word and returns.  The next qadic_sync_status(stream) reports it and
 * clears it; the context stays usable.  Nothing faults, traps or hangs. */
int qadic_selftest_bounded_wait(uint32_t polls, void *stream);

/* --------------------------------------------------------------- status --
 * Synchronises `stream` and returns QADIC_E_DEVICE_TIMEOUT if a kernel of
 * this library on the current device gave up a bounded wait since the last
 * call (the word is then cleared), QADIC_E_CUDA on a CUDA error, else OK. */
int qadic_sync_status(void *stream);
const char *qadic_status_string(int status);
const char *qadic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QADIC_H */
