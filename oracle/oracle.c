/*
 * Oracle for GF(p^k) arithmetic through the q-adic transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything here is the plain definition of what the q-adic method computes,
 * written as slow schoolbook integer arithmetic on coefficient vectors, with
 * no packing into machine words:
 *
 *   * GF(p^k) = Z_p[X]/(P) with P monic irreducible of degree k, elements as
 *     coefficient vectors c_0..c_{k-1} in [0, p-1]   (Sec. 7, canonical
 *     representation of a finite field extension).
 *   * A product a*b is the schoolbook product in Z[X] (Eq. 1 gives its
 *     coefficients sum_{i+j=t} alpha_i beta_j), each coefficient reduced
 *     mod p, then long division by P mod p.
 *   * A GEMM entry is sum_l A_il * B_lj evaluated as above, with the 2k-1
 *     unreduced coefficients accumulated in int64 before the reductions
 *     (reduction mod p and mod P are ring homomorphisms, so this is the same
 *     element as reducing every product).
 *   * REDQ (Alg. 2) has the plain specification rho = sum_i (mu~_i mod p) q^i
 *     for r~ = sum_i mu~_i q^i with 0 <= mu~_i < q; the plain oracle extracts
 *     the base-q digits by repeated integer division.  A second routine walks
 *     Alg. 2's own steps (rop, u_i, mu_i) in 128-bit integers so the worked
 *     Example 3 and Thm. 2's invariants can be checked.
 *
 * Conventions where the paper is silent (the readings taken):
 *   * The default defining polynomial is the monic irreducible of degree k
 *     with the smallest value sum_i a_i p^i over its non-leading coefficients.
 *   * The generator used for discrete-log codes is the primitive element with
 *     the smallest value sum_i c_i p^i; log code p^k - 1 stands for zero.
 *
 * Every routine has a pin in tests/ that does not go through this file:
 * worked examples of the paper, field invariants, brute force over tiny
 * fields and closed forms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <fenv.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXK 16

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the OpenMP loops that follow (timing runs only). */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Trial division. */
int or_is_prime(uint32_t p) {
    if (p < 2) return 0;
    for (uint64_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return 0;
    return 1;
}

static uint64_t ipow(uint64_t b, uint32_t e) {
    uint64_t r = 1;
    while (e--) r *= b;
    return r;
}

/* Remainder of f (degree df, coefficients low->high, in [0,p-1]) divided by
 * the monic g (degree dg), mod p.  Result left in f[0..dg-1]; returns 1 when
 * the remainder is zero. */
static int poly_rem_is_zero(uint32_t p, int64_t *f, int df, const int64_t *g, int dg) {
    for (int t = df; t >= dg; --t) {
        int64_t c = ((f[t] % (int64_t)p) + p) % p;
        if (c == 0) { f[t] = 0; continue; }
        for (int i = 0; i <= dg; ++i) {
            f[t - dg + i] -= c * g[i];
            f[t - dg + i] = ((f[t - dg + i] % (int64_t)p) + p) % p;
        }
    }
    for (int i = 0; i < dg; ++i)
        if (((f[i] % (int64_t)p) + p) % p != 0) return 0;
    return 1;
}

/* P has k+1 coefficients, low->high, P[k] == 1.  Irreducible over Z_p iff no
 * monic polynomial of degree 1..k/2 divides it: checked by trying them all. */
int or_irreducible(uint32_t p, uint32_t k, const uint32_t *P) {
    if (k == 0 || k > OR_MAXK || P[k] != 1) return 0;
    for (uint32_t i = 0; i <= k; ++i) if (P[i] >= p) return 0;
    if (k == 1) return 1;
    for (uint32_t d = 1; d <= k / 2; ++d) {
        uint64_t count = ipow(p, d);
        for (uint64_t v = 0; v < count; ++v) {
            int64_t g[OR_MAXK + 1], f[OR_MAXK + 1];
            uint64_t t = v;
            for (uint32_t i = 0; i < d; ++i) { g[i] = (int64_t)(t % p); t /= p; }
            g[d] = 1;
            for (uint32_t i = 0; i <= k; ++i) f[i] = P[i];
            if (poly_rem_is_zero(p, f, (int)k, g, (int)d)) return 0;
        }
    }
    return 1;
}

/* The monic irreducible of degree k whose low coefficients have the smallest
 * value sum_i a_i p^i.  Returns 0 on success. */
int or_smallest_irreducible(uint32_t p, uint32_t k, uint32_t *P) {
    if (!or_is_prime(p) || k == 0 || k > OR_MAXK) return -1;
    uint64_t count = ipow(p, k);
    for (uint64_t v = 0; v < count; ++v) {
        uint64_t t = v;
        for (uint32_t i = 0; i < k; ++i) { P[i] = (uint32_t)(t % p); t /= p; }
        P[k] = 1;
        if (or_irreducible(p, k, P)) return 0;
    }
    return -1;
}

/* c = a * b in Z_p[X]/(P): schoolbook product, coefficients mod p, long
 * division by P.  a, b, c hold k coefficients in [0, p-1]. */
void or_field_mul(uint32_t p, uint32_t k, const uint32_t *P,
                  const uint32_t *a, const uint32_t *b, uint32_t *c) {
    int64_t acc[2 * OR_MAXK];
    memset(acc, 0, sizeof(acc));
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = 0; j < k; ++j)
            acc[i + j] += (int64_t)a[i] * (int64_t)b[j];
    int64_t g[OR_MAXK + 1];
    for (uint32_t i = 0; i <= k; ++i) g[i] = P[i];
    for (uint32_t t = 0; t < 2 * k - 1; ++t) acc[t] = ((acc[t] % (int64_t)p) + p) % p;
    if (k > 1) poly_rem_is_zero(p, acc, (int)(2 * k - 2), g, (int)k);
    for (uint32_t i = 0; i < k; ++i) c[i] = (uint32_t)(((acc[i] % (int64_t)p) + p) % p);
}

static void digits_of(uint64_t v, uint32_t p, uint32_t k, uint32_t *c) {
    for (uint32_t i = 0; i < k; ++i) { c[i] = (uint32_t)(v % p); v /= p; }
}

static int is_one(const uint32_t *c, uint32_t k) {
    if (c[0] != 1) return 0;
    for (uint32_t i = 1; i < k; ++i) if (c[i] != 0) return 0;
    return 1;
}

/* Multiplicative order of a non-zero element, by repeated multiplication. */
uint64_t or_order(uint32_t p, uint32_t k, const uint32_t *P, const uint32_t *a) {
    uint32_t x[OR_MAXK], y[OR_MAXK];
    memcpy(x, a, k * sizeof(uint32_t));
    uint64_t n = 1, limit = ipow(p, k);
    while (!is_one(x, k)) {
        or_field_mul(p, k, P, x, a, y);
        memcpy(x, y, k * sizeof(uint32_t));
        if (++n > limit) return 0;   /* a was zero */
    }
    return n;
}

/* The primitive element with the smallest value sum_i c_i p^i. */
int or_generator(uint32_t p, uint32_t k, const uint32_t *P, uint32_t *g) {
    uint64_t q = ipow(p, k);
    for (uint64_t v = 1; v < q; ++v) {
        digits_of(v, p, k, g);
        if (or_order(p, k, P, g) == q - 1) return 0;
    }
    return -1;
}

/* table[e*k + i] = coefficient i of g^e for e = 0..p^k-2; entry p^k-1 is
 * the zero element (the log code of zero). */
void or_antilog(uint32_t p, uint32_t k, const uint32_t *P, const uint32_t *g, uint32_t *table) {
    uint64_t q = ipow(p, k);
    uint32_t x[OR_MAXK], y[OR_MAXK];
    memset(x, 0, sizeof(x));
    x[0] = 1;
    for (uint64_t e = 0; e + 1 < q; ++e) {
        memcpy(table + e * k, x, k * sizeof(uint32_t));
        or_field_mul(p, k, P, x, g, y);
        memcpy(x, y, k * sizeof(uint32_t));
    }
    memset(table + (q - 1) * k, 0, k * sizeof(uint32_t));
}

/* Dot product sum_l a_l * b_l over GF(p^k).  a_l is at a + l*sa (k int32
 * coefficients, any integer values, taken mod p), b_l at b + l*sb. */
static void dot_entry(uint32_t p, uint32_t k, const uint32_t *P, int64_t K,
                      const int32_t *a, int64_t sa, const int32_t *b, int64_t sb,
                      uint32_t *out) {
    int64_t acc[2 * OR_MAXK];
    memset(acc, 0, sizeof(acc));
    for (int64_t l = 0; l < K; ++l) {
        const int32_t *al = a + l * sa, *bl = b + l * sb;
        for (uint32_t i = 0; i < k; ++i)
            for (uint32_t j = 0; j < k; ++j)
                acc[i + j] += (int64_t)al[i] * (int64_t)bl[j];
    }
    int64_t g[OR_MAXK + 1];
    for (uint32_t i = 0; i <= k; ++i) g[i] = P[i];
    for (uint32_t t = 0; t < 2 * k - 1; ++t) acc[t] = ((acc[t] % (int64_t)p) + p) % p;
    if (k > 1) poly_rem_is_zero(p, acc, (int)(2 * k - 2), g, (int)k);
    for (uint32_t i = 0; i < k; ++i) out[i] = (uint32_t)(((acc[i] % (int64_t)p) + p) % p);
}

/* C = A * B over GF(p^k).  Element-major layouts: A[(i*K + l)*k + c] (m x K),
 * B[(l*n + j)*k + c] (K x n), C[(i*n + j)*k + c] (m x n), C in [0, p-1]. */
void or_gemm(uint32_t p, uint32_t k, const uint32_t *P, int64_t m, int64_t n, int64_t K,
             const int32_t *A, const int32_t *B, uint32_t *C) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            dot_entry(p, k, P, K, A + i * K * k, (int64_t)k, B + j * k, n * (int64_t)k,
                      C + (i * n + j) * k);
}

/* `count` independent entries: entry s is the dot product of the row
 * rows + s*K*k (K elements, element-major) with the column cols + s*K*k. */
void or_dot_batch(uint32_t p, uint32_t k, const uint32_t *P, int64_t K, int64_t count,
                  const int32_t *rows, const int32_t *cols, uint32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < count; ++s)
        dot_entry(p, k, P, K, rows + s * K * k, (int64_t)k, cols + s * K * k, (int64_t)k,
                  out + s * k);
}

/* Products of polynomials with k coefficients in Z_p[X] (no reduction by a
 * defining polynomial): out[s*(2k-1) + t] = (sum_{i+j=t} a_i b_j) mod p. */
void or_polymul(uint32_t p, uint32_t k, int64_t count, const int32_t *a, const int32_t *b,
                uint32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < count; ++s) {
        int64_t acc[2 * OR_MAXK];
        memset(acc, 0, sizeof(acc));
        for (uint32_t i = 0; i < k; ++i)
            for (uint32_t j = 0; j < k; ++j)
                acc[i + j] += (int64_t)a[s * k + i] * (int64_t)b[s * k + j];
        for (uint32_t t = 0; t < 2 * k - 1; ++t)
            out[s * (2 * k - 1) + t] = (uint32_t)(((acc[t] % (int64_t)p) + p) % p);
    }
}

/* Long polynomial products in Z_p[X] (Sec. 6's workload, the plain
 * definition behind both the classical method and the d-FQT): a and b are
 * count polynomials of degree N (N+1 coefficients each, lowest first);
 * out[s*(2N+1) + t] = (sum_{i+j=t} a_i b_j) mod p, accumulated in int64. */
void or_polymul_long(uint32_t p, int64_t N, int64_t count, const int32_t *a, const int32_t *b,
                     uint32_t *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < count; ++s) {
        const int32_t *x = a + s * (N + 1), *y = b + s * (N + 1);
        for (int64_t t = 0; t <= 2 * N; ++t) {
            int64_t acc = 0;
            const int64_t lo = t > N ? t - N : 0, hi = t < N ? t : N;
            for (int64_t i = lo; i <= hi; ++i) acc += (int64_t)x[i] * (int64_t)y[t - i];
            out[s * (2 * N + 1) + t] = (uint32_t)(((acc % (int64_t)p) + p) % p);
        }
    }
}

/* Plain REDQ specification (Alg. 2 ENSURE): for each word r = sum_{i<=d}
 * mu~_i q^i (an exact non-negative integer held in a double, < 2^53), write
 * rho = sum_i (mu~_i mod p) q^i.  Digits by repeated integer division. */
void or_redq(uint32_t p, uint64_t q, uint32_t d, int64_t count, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < count; ++s) {
        uint64_t r = (uint64_t)in[s];
        uint64_t rho = 0, scale = 1;
        for (uint32_t i = 0; i <= d; ++i) {
            uint64_t digit = (i == d) ? r : r % q;
            r = (i == d) ? 0 : r / q;
            rho += (digit % p) * scale;
            scale *= q;
        }
        out[s] = (double)rho;
    }
}

typedef unsigned __int128 u128;

/* Plain specification in 128-bit integers: mu[i] = (digit i of r in base q)
 * mod p for i = 0..d, the top digit d taking all remaining high part. */
void or_redq_digits_u128(uint32_t p, uint64_t q, uint32_t d, uint64_t r_lo, uint64_t r_hi,
                         uint32_t *mu) {
    u128 r = ((u128)r_hi << 64) | r_lo;
    for (uint32_t i = 0; i <= d; ++i) {
        u128 digit = (i == d) ? r : r % q;
        r = (i == d) ? 0 : r / q;
        mu[i] = (uint32_t)(digit % p);
    }
}

/* Alg. 2 step by step in 128-bit integers.  rop = floor(r/p);
 * u_i = floor(r/q^i) - p*floor(rop/q^i); mu_d = u_d;
 * mu_i = (u_i - q*u_{i+1}) mod p for i < d.
 * rop_out[0] = low 64 bits, rop_out[1] = high 64 bits. */
void or_redq_alg2_u128(uint32_t p, uint64_t q, uint32_t d, uint64_t r_lo, uint64_t r_hi,
                       uint64_t *rop_out, int64_t *u, uint32_t *mu) {
    u128 r = ((u128)r_hi << 64) | r_lo;
    u128 rop = r / p;
    rop_out[0] = (uint64_t)rop;
    rop_out[1] = (uint64_t)(rop >> 64);
    u128 qi = 1;
    for (uint32_t i = 0; i <= d; ++i) {
        u[i] = (int64_t)((r / qi) - (u128)p * (rop / qi));
        qi *= q;
    }
    mu[d] = (uint32_t)u[d];
    int64_t qmod = (int64_t)(q % p);
    for (uint32_t i = 0; i < d; ++i) {
        int64_t v = (u[i] - qmod * u[i + 1]) % (int64_t)p;
        mu[i] = (uint32_t)(v < 0 ? v + p : v);
    }
}

/* Lemma 1 evaluated literally: with rounding toward +infinity, compute
 * inv = 1/p, t = r*inv and return floor(t).  Used by the tests to check the
 * lemma's bound against integer division. */
double or_lemma1_floor(double r, double p) {
    int old = fegetround();
    fesetround(FE_UPWARD);
    volatile double inv = 1.0 / p;
    volatile double t = r * inv;
    fesetround(old);
    return floor(t);
}
