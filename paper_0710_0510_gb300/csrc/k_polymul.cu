// Batched polynomial products in Z_p[X] by the DQT (Alg. 1) followed by
// REDQ (Alg. 2): one thread per pair.
//
//   pack:    a~ = sum_i a_i q^i, q = 2^s, by shifts (Sec. 2, power-of-two q)
//   product: r = a~ b~ in FP64; exact as hi + lo with lo = fma(a~, b~, -hi)
//            (or the single-rounded product when Eq. 2 holds for m = 53)
//   REDQ:    rop = floor(r/p) (one multiply-high), u_i = (r >> s i) -
//            p (rop >> s i), mu_{2k-2} = u_{2k-2}, mu_i = (u_i - q u_{i+1})
//            mod p through a p^2 table (Table 2, "p^2 extra memory, d
//            accesses").
#include "common.cuh"

namespace qadic {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
polymul_kernel(const uint8_t *__restrict__ a, const uint8_t *__restrict__ b,
               uint8_t *__restrict__ out, int64_t count, uint32_t p, uint32_t k, uint32_t s,
               uint32_t qneg_mod_p, Div64 divp, int plain) {
    extern __shared__ uint8_t smem[];
    const uint32_t D = 2 * k - 1;
    uint8_t *corr = smem;                         // p*p entries
    uint8_t *stage = smem + ((p * p + 15) & ~15u);  // kThreads * D bytes

    const uint32_t m32 = (uint32_t)((((uint64_t)1 << 32) + p - 1) / p);
    for (uint32_t i = threadIdx.x; i < p * p; i += blockDim.x) {
        const uint32_t x = i / p, y = i % p;      // table index x*p + y -> (x + (-q) y) mod p
        corr[i] = (uint8_t)mod_small(x + qneg_mod_p * y, p, m32);
    }
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * kThreads;
    const int64_t idx = base + threadIdx.x;
    if (idx < count) {
        uint64_t aw = 0, bw = 0;
        for (uint32_t i = 0; i < k; ++i) {   // coefficients taken mod p
            aw |= (uint64_t)mod_small(__ldg(a + idx * k + i), p, m32) << (s * i);
            bw |= (uint64_t)mod_small(__ldg(b + idx * k + i), p, m32) << (s * i);
        }
        const double ad = (double)aw, bd = (double)bw;   // exact: < 2^53
        uint64_t r;
        const double hi = ad * bd;
        if (plain) {
            r = (uint64_t)hi;
        } else {
            const double lo = fma(ad, bd, -hi);              // exact error term
            r = (uint64_t)((int64_t)hi + (int64_t)lo);
        }
        const uint64_t rop = div64(r, divp);
        uint32_t u_next = 0;
        uint8_t *dst = stage + threadIdx.x * D;
        for (int i = (int)D - 1; i >= 0; --i) {
            const uint32_t ui = (uint32_t)((r >> (s * i)) - (uint64_t)p * (rop >> (s * i)));
            dst[i] = (i == (int)D - 1) ? (uint8_t)ui : corr[ui * p + u_next];
            u_next = ui;
        }
    }
    __syncthreads();
    // Coalesced write-out of the block's contiguous output range.
    const int64_t nvalid = (count - base) < kThreads ? (count - base) : kThreads;
    uint8_t *gout = out + base * D;
    for (int64_t i = threadIdx.x; i < nvalid * D; i += blockDim.x) gout[i] = stage[i];
}

}  // namespace

int launch_polymul(uint32_t p, uint32_t k, uint32_t log2_q, bool plain_f64, const uint8_t *a,
                   const uint8_t *b, uint8_t *out, int64_t count, cudaStream_t stream) {
    const uint64_t q = 1ull << log2_q;
    const uint32_t qneg = (uint32_t)((p - q % p) % p);
    const size_t smem = ((p * p + 15) & ~15u) + (size_t)kThreads * (2 * k - 1);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(polymul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return set_error(QADIC_E_CUDA, "smem attribute: %s",
                             cudaGetErrorString(cudaGetLastError()));
    }
    const int64_t blocks = (count + kThreads - 1) / kThreads;
    if (blocks > 0x7fffffff) return set_error(QADIC_E_INVALID, "count too large");
    polymul_kernel<<<(unsigned)blocks, kThreads, smem, stream>>>(
        a, b, out, count, p, k, log2_q, qneg, make_div64(p), plain_f64 ? 1 : 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "polymul launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace qadic
