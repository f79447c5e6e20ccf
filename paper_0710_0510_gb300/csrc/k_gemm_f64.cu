// FP64 q-adic GEMM with fused REDQ (Alg. 4 for every output entry).
//
// A, B hold q-adic words a~ = sum_i c_i q^i (Eq. 1) as doubles.  The K loop
// runs in blocks of n_q products (Eq. 2: q > n_q k (p-1)^2 and
// (2k-1) log2 q < 53, so every block sum r is an exact integer whose base-q
// digits are the unreduced product coefficients).  After each block:
//   rop = floor(r/p)             Lemma 1: r * RU(1/p) rounded up, truncated
//   u_t = (r >> s t) - p (rop >> s t),  t = 0..2k-2          (Alg. 4, 3-7)
//   L = T_L[u_0..u_{k-1}],  H = T_H[u_{k-1}..u_{2k-2}]       (Alg. 4, 8-9)
//   block value = L + H, coefficientwise mod p                (Alg. 4, 10)
// and the block values are summed across K (reduction mod p at the end).
//
// FP64 runs at ~1 TFLOP/s on GB300, so this path is bound by the FP64 pipe,
// not by memory: a plain shared-memory tiled DFMA kernel (64 x 64 tile,
// 4 x 4 outputs per thread) with the Thm. 3 tables in shared memory.
#include "common.cuh"

namespace qadic {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int kThreads = (BM / TM) * (BN / TN);   // 256
constexpr uint32_t kSmemTableMax = 96 * 1024;

struct GemmF64Params {
    int64_t m, n, K, lda, ldb, ldc;
    uint32_t p, k, s, n_q, order;
    double inv_p_up;
    const uint32_t *tab_L, *tab_H;
    int tables_in_smem;
};

template <int KK>
__global__ void __launch_bounds__(kThreads)
gemm_f64_kernel(const double *__restrict__ A, const double *__restrict__ B, uint8_t *__restrict__ C,
                GemmF64Params P) {
    __shared__ double As[2][BK][BM];
    __shared__ double Bs[2][BK][BN];
    extern __shared__ __align__(16) uint32_t tabs[];

    const uint32_t *tL = P.tab_L, *tH = P.tab_H;
    if (P.tables_in_smem) {
        for (uint32_t i = threadIdx.x; i < P.order; i += blockDim.x) {
            tabs[i] = P.tab_L[i];
            tabs[P.order + i] = P.tab_H[i];
        }
        tL = tabs;
        tH = tabs + P.order;
    }

    const int tx = threadIdx.x % (BN / TN), ty = threadIdx.x / (BN / TN);
    const int64_t row0 = (int64_t)blockIdx.y * BM, col0 = (int64_t)blockIdx.x * BN;
    const uint32_t p = P.p, s = P.s;

    double acc[TM][TN];
    int32_t sum[TM][TN][KK];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            acc[i][j] = 0.0;
#pragma unroll
            for (int c = 0; c < KK; ++c) sum[i][j][c] = 0;
        }

    // tile loaders: A tile BM x BK (row-major in global), B tile BK x BN
    auto load_tiles = [&](int buf, int64_t k0) {
        for (int e = threadIdx.x; e < BM * BK; e += kThreads) {
            const int r = e / BK, kk = e % BK;
            const int64_t gr = row0 + r, gk = k0 + kk;
            As[buf][kk][r] = (gr < P.m && gk < P.K) ? __ldg(A + gr * P.lda + gk) : 0.0;
        }
        for (int e = threadIdx.x; e < BK * BN; e += kThreads) {
            const int kk = e / BN, c = e % BN;
            const int64_t gk = k0 + kk, gc = col0 + c;
            Bs[buf][kk][c] = (gk < P.K && gc < P.n) ? __ldg(B + gk * P.ldb + gc) : 0.0;
        }
    };

    auto redq_block = [&]() {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const double x = acc[i][j];
                const uint64_t r = f64_to_u64_exact(x);
                const uint64_t rop = f64_to_u64_exact(__dmul_ru(x, P.inv_p_up));
                uint32_t idxL = 0, idxH = 0, pw = 1;
#pragma unroll
                for (int t = 0; t < KK; ++t) {
                    const uint32_t u = (uint32_t)((r >> (s * t)) - (uint64_t)p * (rop >> (s * t)));
                    idxL += u * pw;
                    pw *= p;
                }
                pw = 1;
#pragma unroll
                for (int t = KK - 1; t < 2 * KK - 1; ++t) {
                    const uint32_t u = (uint32_t)((r >> (s * t)) - (uint64_t)p * (rop >> (s * t)));
                    idxH += u * pw;
                    pw *= p;
                }
                // in range for every input that respects Eq. 2 (Thm. 2: 0 <= u < p);
                // clamped so that malformed words cannot read past the tables
                const uint32_t L = tL[min(idxL, P.order - 1)], H = tH[min(idxH, P.order - 1)];
#pragma unroll
                for (int c = 0; c < KK; ++c)
                    sum[i][j][c] += (int32_t)((L >> (8 * c)) & 0xff) + (int32_t)((H >> (8 * c)) & 0xff);
                acc[i][j] = 0.0;
            }
    };

    load_tiles(0, 0);
    __syncthreads();
    uint32_t cnt = 0;
    const int64_t nk = (P.K + BK - 1) / BK;
    for (int64_t t = 0; t < nk; ++t) {
        const int buf = (int)(t & 1);
        if (t + 1 < nk) load_tiles(buf ^ 1, (t + 1) * BK);
        const int64_t krem = P.K - t * BK;
        const int kmax = krem < BK ? (int)krem : BK;
        for (int kk = 0; kk < kmax; ++kk) {
            double a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + i * (BM / TM)];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + j * (BN / TN)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            if (++cnt == P.n_q) {
                redq_block();
                cnt = 0;
            }
        }
        __syncthreads();
    }
    if (cnt != 0) redq_block();

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gr = row0 + ty + i * (BM / TM);
        if (gr >= P.m) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gc = col0 + tx + j * (BN / TN);
            if (gc >= P.n) continue;
#pragma unroll
            for (int c = 0; c < KK; ++c)
                C[((int64_t)c * P.m + gr) * P.ldc + gc] = (uint8_t)(sum[i][j][c] % (int32_t)p);
        }
    }
}

template <int KK>
int launch_k(const double *A, const double *B, uint8_t *C, const GemmF64Params &P, size_t smem,
             cudaStream_t stream) {
    auto kern = gemm_f64_kernel<KK>;
    if (smem > 32 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return set_error(QADIC_E_CUDA, "gemm_f64 smem attribute: %s",
                         cudaGetErrorString(cudaGetLastError()));
    const dim3 grid((unsigned)((P.n + BN - 1) / BN), (unsigned)((P.m + BM - 1) / BM));
    if (grid.y > 65535) return set_error(QADIC_E_INVALID, "m too large for the FP64 path");
    kern<<<grid, kThreads, smem, stream>>>(A, B, C, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(QADIC_E_CUDA, "gemm_f64 launch: %s", cudaGetErrorString(e));
    return QADIC_OK;
}

}  // namespace

int launch_gemm_f64(const Field &f, int64_t m, int64_t n, int64_t K, const double *A, int64_t lda,
                    const double *B, int64_t ldb, uint8_t *C, int64_t ldc, cudaStream_t stream) {
    GemmF64Params P;
    P.m = m;
    P.n = n;
    P.K = K;
    P.lda = lda;
    P.ldb = ldb;
    P.ldc = ldc;
    P.p = f.p;
    P.k = f.k;
    P.s = f.log2_q;
    P.n_q = f.n_q;
    P.order = f.order;
    P.tab_L = f.d_tab_L;
    P.tab_H = f.d_tab_H;
    {   // 1/p rounded toward +infinity, checked exactly
        double inv = 1.0 / (double)f.p;
        int e;
        const double mfrac = frexp(inv, &e);
        const uint64_t M = (uint64_t)ldexp(mfrac, 53);
        if ((unsigned __int128)M * f.p < ((unsigned __int128)1 << (53 - e))) inv = nextafter(inv, 2.0);
        P.inv_p_up = inv;
    }
    const size_t tab_bytes = (size_t)2 * f.order * sizeof(uint32_t);
    P.tables_in_smem = tab_bytes <= kSmemTableMax;
    const size_t smem = P.tables_in_smem ? tab_bytes : 0;
    switch (f.k) {
        case 1: return launch_k<1>(A, B, C, P, smem, stream);
        case 2: return launch_k<2>(A, B, C, P, smem, stream);
        case 3: return launch_k<3>(A, B, C, P, smem, stream);
        case 4: return launch_k<4>(A, B, C, P, smem, stream);
        default: return set_error(QADIC_E_UNSUPPORTED, "FP64 path supports k <= 4");
    }
}

}  // namespace qadic
