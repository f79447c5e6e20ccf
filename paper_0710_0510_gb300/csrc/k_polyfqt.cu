// Long polynomial products over Z_p by the d-FQT (Sec. 6, Table 2).
//
// A polynomial of degree N is cut into D_q + 1 blocks of d + 1 coefficients
// (P = sum_i P_i Y^i with Y = X^(d+1)), and each block is packed into one
// machine word by the q-adic substitution, P_i(q) = sum_j a_{i(d+1)+j} q^j
// (q = 2^s, so packing is shifts).  The product's blocks are the word
// convolution W_t = sum_i P_i Q_{t-i}; a word product holds the 2d + 1
// coefficients of a degree-2d block product, and up to n_q of them are
// summed exactly before a simultaneous reduction REDQ_{2d+1} (Alg. 2) turns
// the word back into residues.  Block t's digits d+1..2d overlap block t+1's
// digits 0..d-1 (Y^(t+1) = X^((t+1)(d+1))), so each output coefficient is
// the sum of at most two residues mod p.
//
// d = 0 is the classical algorithm with delayed reduction (one coefficient
// per word, a plain mod p every n_q products), the other row of Table 2.
//
// Two machine words:
//   binary64 (the paper's choice): exact FMAs on integers < 2^51, floor(r/p)
//       by Lemma 1 (multiply by 1/p rounded up); (2d+1) s <= 51;
//   64-bit integers (allowed by Sec. 2: m = 64): 32-bit operands multiplied
//       into 64-bit accumulators (IMAD.WIDE), floor(r/p) by a multiply-high;
//       (d+1) s <= 32 and (2d+1) s <= 64.  On GB300 the integer pipe issues
//       tens of times more multiply-adds per clock than the FP64 pipe.
// In both, q > n_q (d+1) (p-1)^2 + (p-1) (Eq. 2 with k = d+1, plus room for
// the fed-back reduced word, see below).
//
// One CTA per polynomial pair (grid-stride over pairs).  Work items are
// (block of kTB consecutive output words t, piece of the i range); a thread
// keeps the kTB accumulators in registers and slides a window over Q, so
// each step loads one P_i and one Q_j for kTB multiply-adds.  After every
// `chunk` <= n_q products each accumulator is reduced by REDQ and the
// reduced word rho (digits < p) is fed back as the start of the next chunk
// -- the reduction "delayed as long as the bounds hold" of Sec. 6.  The
// item's final words are unpacked into per-coefficient residue sums in
// shared memory (atomics: pieces of the same t run on different threads),
// and a last pass adds the overlapping digits mod p and stores bytes.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace qadic {

namespace {

constexpr int kFqtThreads = 128;
constexpr int kTB = 4;     // output words per work item
constexpr int kPad = kTB;  // zero words on each side of Q

struct FqtParams {
    uint32_t p, N, d, s;    // prime, degree, FQT degree, log2 q
    uint32_t Dq;            // words per input, minus one
    uint32_t chunk;         // products per accumulator between reductions
    uint32_t piece;         // i-range length of one work item (multiple of chunk)
    uint32_t npc;           // pieces of the i range [0, Dq], cut at multiples of piece
    uint32_t span;          // work items per piece (t-blocks that may meet it)
    uint32_t nblocks;       // blocks of kTB output words
    uint32_t qneg, m32;
    double inv_p_up;
    Div64 divp;
};

// q = 2^s is fixed by d and the word: the largest s with (2d+1) s within
// the word (64 bits, or 51 for Lemma 1 on binary64) and, for integer words,
// (d+1) s <= 32 (32-bit operands).  The host derives it the same way.
__host__ __device__ constexpr uint32_t fqt_log2_q(uint32_t d, bool int_words) {
    return int_words ? (64 / (2 * d + 1) < 32 / (d + 1) ? 64 / (2 * d + 1) : 32 / (d + 1))
                     : 51 / (2 * d + 1);
}

// DT >= 0: the kernel is specialised for d = DT (every digit shift a
// constant, every loop over digits unrolled); DT = -1 reads d from P.
template <int DT>
__device__ __forceinline__ uint32_t fqt_d(const FqtParams &P) { return DT >= 0 ? (uint32_t)DT : P.d; }

template <bool INT, int DT>
__device__ __forceinline__ uint32_t fqt_s(const FqtParams &P) {
    return DT >= 0 ? fqt_log2_q((uint32_t)DT, INT) : P.s;
}

// REDQ_{2d+1} of an accumulator (Alg. 2): rop = floor(r/p), u_j from the
// shifted words, mu_j = (u_j - q u_{j+1}) mod p; returns rho = sum_j mu_j q^j.
template <bool INT, int DT>
__device__ __forceinline__ uint64_t redq_rho(uint64_t r, double rd, const FqtParams &P) {
    uint64_t rop;
    if constexpr (INT) rop = div64(r, P.divp);
    else rop = f64_to_u64_exact(__dmul_ru(rd, P.inv_p_up));
    const uint32_t p = P.p, s = fqt_s<INT, DT>(P), top = 2 * fqt_d<DT>(P);
    uint64_t rho = 0;
    uint32_t u_next = 0;
#pragma unroll
    for (int j = (int)top; j >= 0; --j) {
        const uint32_t sh = s * (uint32_t)j;
        const uint32_t u = (uint32_t)(r >> sh) - p * (uint32_t)(rop >> sh);
        const uint32_t mu = (j == (int)top) ? u : mod_small(u + P.qneg * u_next, p, P.m32);
        rho |= (uint64_t)mu << sh;
        u_next = u;
    }
    return rho;
}

template <bool INT, int DT>
__global__ void __launch_bounds__(kFqtThreads)
polymul_fqt_kernel(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b,
                   uint8_t *__restrict__ out, int64_t count, const FqtParams P) {
    using Word = typename std::conditional<INT, uint32_t, double>::type;
    using Acc = typename std::conditional<INT, uint64_t, double>::type;
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t dd = fqt_d<DT>(P);
    const uint32_t p = P.p, N = P.N, Dq = P.Dq, nw = Dq + 1, d1 = dd + 1, D = 2 * dd + 1;
    const uint32_t s_bits = fqt_s<INT, DT>(P);
    Word *Pw = reinterpret_cast<Word *>(smem);                 // nw words
    Word *Qw = Pw + nw;                                        // Q_j at Qw[kPad + j]
    uint32_t *R = reinterpret_cast<uint32_t *>(Qw + nw + 2 * kPad);   // (2 Dq + 1) x D
    const uint32_t nR = (2 * Dq + 1) * D;
    const uint64_t dmask = (s_bits >= 64) ? ~0ull : ((1ull << s_bits) - 1);

    for (int64_t pr = blockIdx.x; pr < count; pr += gridDim.x) {
        const uint8_t *x = a + pr * (int64_t)(N + 1);
        const uint8_t *y = b + pr * (int64_t)(N + 1);
        // DQT pack by shifts (q = 2^s), inputs reduced mod p.
        for (uint32_t i = threadIdx.x; i < nw; i += blockDim.x) {
            uint64_t wa = 0, wb = 0;
#pragma unroll
            for (uint32_t j = 0; j < d1; ++j) {
                const uint32_t c = i * d1 + j;
                if (c <= N) {
                    wa |= (uint64_t)mod_small(x[c], p, P.m32) << (s_bits * j);
                    wb |= (uint64_t)mod_small(y[c], p, P.m32) << (s_bits * j);
                }
            }
            Pw[i] = (Word)wa;
            Qw[kPad + i] = (Word)wb;
        }
        if (threadIdx.x < kPad) {
            Qw[threadIdx.x] = (Word)0;
            Qw[kPad + nw + threadIdx.x] = (Word)0;
        }
        for (uint32_t i = threadIdx.x; i < nR; i += blockDim.x) R[i] = 0;
        __syncthreads();

        // Work items: (piece pc of the i range, cut at multiples of `piece`,
        // block of kTB output words meeting it).  Consecutive threads take
        // consecutive word blocks of one piece, so most lanes of a warp run
        // exactly `piece` steps; only the blocks at the two edges of a
        // piece's range (the sides of the triangle i <= t, t - i <= Dq) do
        // less.
        const uint32_t slots = P.npc * P.span;
        for (uint32_t it = threadIdx.x; it < slots; it += blockDim.x) {
            const int pc = (int)(it / P.span);
            const int tb = max(0, pc * (int)P.piece / kTB - 1) + (int)(it % P.span);
            if (tb >= (int)P.nblocks) continue;
            const int t0 = tb * kTB;
            const int ilo = max(max(0, t0 - (int)Dq), pc * (int)P.piece);
            const int iend = min(min(t0 + kTB - 1, (int)Dq), (pc + 1) * (int)P.piece - 1);
            if (ilo > iend) continue;
            // window: qv[tt] = Q_{t0+tt-i}, zero outside [0, Dq]
            Word qv[kTB];
#pragma unroll
            for (int tt = 0; tt < kTB; ++tt) qv[tt] = Qw[kPad + t0 + tt - ilo];
            Acc acc[kTB];
#pragma unroll
            for (int tt = 0; tt < kTB; ++tt) acc[tt] = (Acc)0;
            for (int c0 = ilo; c0 <= iend; c0 += (int)P.chunk) {
                const int c1 = min(iend, c0 + (int)P.chunk - 1);
                for (int i = c0; i <= c1; ++i) {
                    const Word pv = Pw[i];
#pragma unroll
                    for (int tt = 0; tt < kTB; ++tt) {
                        if constexpr (INT) acc[tt] += (uint64_t)pv * (uint64_t)qv[tt];
                        else acc[tt] = fma(pv, qv[tt], acc[tt]);
                    }
#pragma unroll
                    for (int tt = kTB - 1; tt > 0; --tt) qv[tt] = qv[tt - 1];
                    qv[0] = Qw[kPad + t0 - i - 1];   // index >= 0: i <= t0 + kTB - 1
                }
                // reduce and feed the reduced word back (digits < p)
#pragma unroll
                for (int tt = 0; tt < kTB; ++tt) {
                    if constexpr (INT) acc[tt] = redq_rho<true, DT>(acc[tt], 0.0, P);
                    else acc[tt] = u64_to_f64_exact(redq_rho<false, DT>(f64_to_u64_exact(acc[tt]), acc[tt], P));
                }
            }
#pragma unroll
            for (int tt = 0; tt < kTB; ++tt) {
                const uint32_t t = (uint32_t)(t0 + tt);
                if (t >= 2 * Dq + 1) break;
                uint64_t rho;
                if constexpr (INT) rho = acc[tt];
                else rho = f64_to_u64_exact(acc[tt]);
#pragma unroll
                for (uint32_t j = 0; j < D; ++j) {
                    const uint32_t mu = (uint32_t)((rho >> (s_bits * j)) & dmask);
                    if (mu) atomicAdd(&R[t * D + j], mu);
                }
            }
        }
        __syncthreads();

        // overlap-add: coefficient c = t (d+1) + j gets digit j of word t
        // and digit j + d + 1 of word t - 1
        uint8_t *o = out + pr * (int64_t)(2 * N + 1);
        for (uint32_t c = threadIdx.x; c <= 2 * N; c += blockDim.x) {
            const uint32_t t = c / d1, j = c - t * d1;
            uint32_t v = t <= 2 * Dq ? R[t * D + j] : 0;
            if (t >= 1 && j < dd) v += R[(t - 1) * D + j + d1];
            o[c] = (uint8_t)(v % p);
        }
        __syncthreads();
    }
}

}  // namespace

int fqt_parameters(uint32_t p, uint32_t N, uint32_t d, bool int_words, qadic_fqt_info *info) {
    if (!is_prime(p) || p > 251) return set_error(QADIC_E_INVALID, "p must be a prime <= 251");
    if (d > 24) return set_error(QADIC_E_INVALID, "d outside [0, 24]");
    const uint32_t D = 2 * d + 1;
    uint32_t s = fqt_log2_q(d, int_words);
    (void)D;
    if (s < 1) return set_error(QADIC_E_OVERFLOW, "no q = 2^s fits %u digits", D);
    const uint64_t q = 1ull << s;
    const uint64_t unit = (uint64_t)(d + 1) * (p - 1) * (p - 1);
    // q > n_q (d+1)(p-1)^2 + (p-1): n_q products added to a reduced word
    // keep every digit below q
    const uint64_t n_q = q > p ? (q - p) / (unit ? unit : 1) : 0;
    if (n_q < 1)
        return set_error(QADIC_E_OVERFLOW,
                         "q = 2^%u admits no product block for d = %u (Eq. 2 with k = d+1)", s, d);
    info->log2_q = s;
    info->n_q = (uint32_t)std::min<uint64_t>(n_q, 0xffffffffull);
    info->D_q = (N + 1 + d) / (d + 1) - 1;
    info->word_bits = int_words ? 64 : 53;
    info->word_products = (uint64_t)(info->D_q + 1) * (info->D_q + 1);
    return QADIC_OK;
}

size_t fqt_smem_bytes(const qadic_fqt_info &I, uint32_t d, bool int_words) {
    const size_t nw = I.D_q + 1;
    const size_t word = int_words ? 4 : 8;
    size_t bytes = (2 * nw + 2 * kPad) * word;
    bytes = (bytes + 15) & ~size_t(15);
    return bytes + (size_t)(2 * I.D_q + 1) * (2 * d + 1) * 4;
}

int launch_polymul_fqt(uint32_t p, uint32_t N, uint32_t d, bool int_words, const uint8_t *a,
                       const uint8_t *b, uint8_t *out, int64_t count, cudaStream_t stream) {
    qadic_fqt_info I;
    int st = fqt_parameters(p, N, d, int_words, &I);
    if (st != QADIC_OK) return st;
    const size_t smem = fqt_smem_bytes(I, d, int_words);
    if (smem > 200 * 1024)
        return set_error(QADIC_E_UNSUPPORTED, "degree %u with d = %u needs %zu bytes of shared memory",
                         N, d, smem);
    FqtParams P;
    P.p = p;
    P.N = N;
    P.d = d;
    P.s = I.log2_q;
    P.Dq = I.D_q;
    // A short chunk keeps work items small enough to balance the CTA; the
    // reduction it adds is cheap next to the multiply-adds.
    P.chunk = std::min<uint32_t>(I.n_q, 32);
    P.piece = P.chunk * std::max<uint32_t>(1, 32 / P.chunk);
    P.nblocks = (2 * I.D_q + 1 + kTB - 1) / kTB;
    P.npc = (I.D_q + P.piece) / P.piece;   // ceil((D_q + 1) / piece)
    // blocks meeting piece pc: t0 in [pc piece - (kTB - 1), (pc + 1) piece - 1 + D_q]
    P.span = (P.piece + I.D_q) / kTB + 3;
    P.qneg = (uint32_t)((p - (uint32_t)((1ull << I.log2_q) % p)) % p);
    P.m32 = make_mod_small(p);
    P.divp = make_div64(p);
    P.inv_p_up = inv_up(p);

    using Kern = void (*)(const uint8_t *, const uint8_t *, uint8_t *, int64_t, const FqtParams);
    Kern kern;
    switch (d) {   // the degrees of the bench's sweep and around it; others read d at run time
#define QADIC_FQT_CASE(D_) \
    case D_: kern = int_words ? polymul_fqt_kernel<true, D_> : polymul_fqt_kernel<false, D_>; break;
        QADIC_FQT_CASE(0) QADIC_FQT_CASE(1) QADIC_FQT_CASE(2) QADIC_FQT_CASE(3)
        QADIC_FQT_CASE(4) QADIC_FQT_CASE(5) QADIC_FQT_CASE(6)
#undef QADIC_FQT_CASE
        default: kern = int_words ? polymul_fqt_kernel<true, -1> : polymul_fqt_kernel<false, -1>; break;
    }
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return set_error(QADIC_E_CUDA, "polymul_fqt smem attribute: %s",
                         cudaGetErrorString(cudaGetLastError()));
    const int64_t blocks = std::min<int64_t>(count, resident_blocks(kern, kFqtThreads, smem) * 8);
    kern<<<(unsigned)blocks, kFqtThreads, smem, stream>>>(a, b, out, count, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(QADIC_E_CUDA, "polymul_fqt launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace qadic
