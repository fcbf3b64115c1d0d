// k_gemm.cu -- C := op(A) op(B) in multicomponent arithmetic (Section 3.1,
// Eq. 1; the block algorithm's GPU form).
//
// Compiled once per precision (MPGPU_GEMM_PREC selects it) so the translation
// units build in parallel.
//
// Design.  Every output c_ij is the sequential fold over l = 0..k-1 of
// c = add(c, mul(a_il, b_lj)) from c = 0, the operation order of the naive
// triple loop, so results are bit-identical to the CPU oracle; k is never split.
// A block owns a BM x BN tile of C, in grouped order: consecutive blocks walk
// down GEMM_GROUP tile rows before moving one tile column right, so the blocks
// resident at any moment cover a near-square patch of C and the op(A) and op(B)
// slabs they read fit in L2 together.  Each thread owns a TM x TN register
// micro-tile (TM*TN independent multiply-add chains for instruction-level
// parallelism).  K-component tiles of op(A) and op(B), BK deep, are staged in
// shared memory component-plane by component-plane, loaded so that consecutive
// threads read consecutive addresses of whichever index is contiguous in the
// operand's storage (transposed operands included).
//
// Roofline.  One QD multiply-add is 209 FP64 instructions (Algorithm 14:
// 106, Algorithm 13: 103) on 64 bytes of operands that each block reuses
// BM or BN times from shared memory, so the binary64 precisions are bound by
// the FP64 pipe, never by HBM or shared memory; the binary32 precisions run on
// the 64x wider FP32 pipe and use larger micro-tiles.
#include <cuda_runtime.h>

#include "mp_arith.cuh"
#include "mp_common.cuh"

namespace mp {

template <class P, int BM, int BN, int BK, int TM, int TN>
struct GemmCfg {
    static constexpr int NTX = BN / TN;  // threads along the columns
    static constexpr int NTY = BM / TM;  // threads along the rows
    static constexpr int NT = NTX * NTY;
    static_assert(BM % TM == 0 && BN % TN == 0, "tile");
    static_assert(NT % 32 == 0 && NT <= 1024, "threads");
};

constexpr int64_t GEMM_GROUP = 16;  // tile rows per group of the block order

template <class P, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(GemmCfg<P, BM, BN, BK, TM, TN>::NT)
    k_gemm(int opA, int opB, int64_t m, int64_t n, int64_t k, const typename P::T *__restrict__ A,
           int64_t lda, int64_t pA, const typename P::T *__restrict__ B, int64_t ldb, int64_t pB,
           typename P::T *__restrict__ C, int64_t ldc, int64_t pC)
{
    using T = typename P::T;
    using V = typename P::V;
    using G = GemmCfg<P, BM, BN, BK, TM, TN>;
    constexpr int K = P::K;
    __shared__ T As[K][BK][BM];
    __shared__ T Bs[K][BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    // grouped block order (1-D grid of tm * tn blocks)
    const int64_t tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
    const int64_t per_group = GEMM_GROUP * tn;
    const int64_t L = blockIdx.x, g = L / per_group, first = g * GEMM_GROUP;
    const int64_t rows = tm - first < GEMM_GROUP ? tm - first : GEMM_GROUP;
    const int64_t r_in = L - g * per_group;
    const int64_t i0 = (first + r_in % rows) * BM, j0 = (r_in / rows) * BN;

    V acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
        for (int s = 0; s < TN; s++) acc[r][s] = vzero<P>();

    for (int64_t k0 = 0; k0 < k; k0 += BK) {
        const int kc = (int)((k - k0) < BK ? (k - k0) : BK);
        // stage op(A)[i0 : i0+BM, k0 : k0+BK] and op(B)[k0 : k0+BK, j0 : j0+BN]
        for (int l = tid; l < BM * BK; l += G::NT) {
            int ii, kk;
            if (opA == 0) { kk = l % BK; ii = l / BK; } else { ii = l % BM; kk = l / BM; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            const bool in = gi < m && kk < kc;
            const int64_t off = opA == 0 ? gi * lda + gk : gk * lda + gi;
#pragma unroll
            for (int c = 0; c < K; c++) As[c][kk][ii] = in ? A[c * pA + off] : T(0);
        }
        for (int l = tid; l < BK * BN; l += G::NT) {
            int jj, kk;
            if (opB == 0) { jj = l % BN; kk = l / BN; } else { kk = l % BK; jj = l / BK; }
            const int64_t gj = j0 + jj, gk = k0 + kk;
            const bool in = gj < n && kk < kc;
            const int64_t off = opB == 0 ? gk * ldb + gj : gj * ldb + gk;
#pragma unroll
            for (int c = 0; c < K; c++) Bs[c][kk][jj] = in ? B[c * pB + off] : T(0);
        }
        __syncthreads();
#pragma unroll 1
        for (int kk = 0; kk < kc; kk++) {
            V a[TM], b[TN];
#pragma unroll
            for (int r = 0; r < TM; r++)
#pragma unroll
                for (int c = 0; c < K; c++) a[r].c[c] = As[c][kk][ty + r * G::NTY];
#pragma unroll
            for (int s = 0; s < TN; s++)
#pragma unroll
                for (int c = 0; c < K; c++) b[s].c[c] = Bs[c][kk][tx + s * G::NTX];
#pragma unroll
            for (int r = 0; r < TM; r++)
#pragma unroll
                for (int s = 0; s < TN; s++) acc[r][s] = P::add(acc[r][s], P::mul(a[r], b[s]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; r++) {
        const int64_t gi = i0 + ty + r * G::NTY;
        if (gi >= m) continue;
#pragma unroll
        for (int s = 0; s < TN; s++) {
            const int64_t gj = j0 + tx + s * G::NTX;
            if (gj < n) vstore<P>(C, pC, gi * ldc + gj, acc[r][s]);
        }
    }
}

template <class P, int BM, int BN, int BK, int TM, int TN>
static mp_status gemm_run(int opA, int opB, int64_t m, int64_t n, int64_t k, const typename P::T *A,
                          int64_t lda, int64_t pA, const typename P::T *B, int64_t ldb, int64_t pB,
                          typename P::T *C, int64_t ldc, int64_t pC, cudaStream_t s)
{
    using G = GemmCfg<P, BM, BN, BK, TM, TN>;
    const int64_t gx = (n + BN - 1) / BN, gy = (m + BM - 1) / BM;
    if (gx * gy > 0x7fffffff) return MP_EINVAL;
    dim3 grid((unsigned)(gx * gy));
    k_gemm<P, BM, BN, BK, TM, TN><<<grid, G::NT, 0, s>>>(opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C,
                                                          ldc, pC);
    return launch_status();
}

// Tile configurations.  Binary64 precisions are FP64-pipe bound, so a few
// independent chains per thread suffice; binary32 ones need more in flight.
template <class P, bool F64 = P::fp64> struct GemmTable;

template <class P> struct GemmTable<P, true> {
    static constexpr int count = 4;
    static const char *name(int c)
    {
        switch (c) {
        case 0: return "BM32 BN32 BK16 TM2 TN2 (256 thr)";
        case 1: return "BM16 BN16 BK16 TM1 TN1 (256 thr)";
        case 2: return "BM32 BN64 BK8 TM2 TN4 (256 thr)";
        case 3: return "BM16 BN32 BK16 TM1 TN2 (256 thr)";
        }
        return nullptr;
    }
    template <typename... Args> static mp_status run(int c, Args... a)
    {
        switch (c) {
        case 1: return gemm_run<P, 16, 16, 16, 1, 1>(a...);
        case 2: return gemm_run<P, 32, 64, 8, 2, 4>(a...);
        case 3: return gemm_run<P, 16, 32, 16, 1, 2>(a...);
        default: return gemm_run<P, 32, 32, 16, 2, 2>(a...);
        }
    }
};

template <class P> struct GemmTable<P, false> {
    static constexpr int count = 4;
    static const char *name(int c)
    {
        switch (c) {
        case 0: return "BM64 BN64 BK16 TM4 TN4 (256 thr)";
        case 1: return "BM32 BN32 BK16 TM2 TN2 (256 thr)";
        case 2: return "BM64 BN32 BK16 TM4 TN2 (256 thr)";
        case 3: return "BM128 BN64 BK8 TM8 TN4 (256 thr)";
        }
        return nullptr;
    }
    template <typename... Args> static mp_status run(int c, Args... a)
    {
        switch (c) {
        case 1: return gemm_run<P, 32, 32, 16, 2, 2>(a...);
        case 2: return gemm_run<P, 64, 32, 16, 4, 2>(a...);
        case 3: return gemm_run<P, 128, 64, 8, 8, 4>(a...);
        default: return gemm_run<P, 64, 64, 16, 4, 4>(a...);
        }
    }
};

template <class P>
static mp_status gemm_launch(int opA, int opB, int64_t m, int64_t n, int64_t k, const typename P::T *A,
                             int64_t lda, int64_t pA, const typename P::T *B, int64_t ldb, int64_t pB,
                             typename P::T *C, int64_t ldc, int64_t pC, int config, mp_stream s)
{
    if ((opA != 0 && opA != 1) || (opB != 0 && opB != 1) || m < 0 || n < 0 || k < 0) return MP_EINVAL;
    if (config < -1 || config >= GemmTable<P>::count) return MP_EINVAL;
    if (m == 0 || n == 0) return MP_OK;
    if (C == nullptr || ldc < n || pC < (m - 1) * ldc + n) return MP_EINVAL;
    if (k > 0) {
        const int64_t ar = opA ? k : m, ac = opA ? m : k;  // storage rows x cols
        const int64_t br = opB ? n : k, bc = opB ? k : n;
        if (A == nullptr || lda < ac || pA < (ar - 1) * lda + ac) return MP_EINVAL;
        if (B == nullptr || ldb < bc || pB < (br - 1) * ldb + bc) return MP_EINVAL;
    }
    return GemmTable<P>::run(config < 0 ? 0 : config, opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C, ldc,
                             pC, as_stream(s));
}

}  // namespace mp

using namespace mp;

#define MP_EXPORT_GEMM(S, PT)                                                                      \
    extern "C" mp_status mp_gemm_ex_##S(int opA, int opB, int64_t m, int64_t n, int64_t k,         \
                                        const PT::T *A, int64_t lda, int64_t pA, const PT::T *B,  \
                                        int64_t ldb, int64_t pB, PT::T *C, int64_t ldc,           \
                                        int64_t pC, int config, mp_stream s)                      \
    {                                                                                              \
        return gemm_launch<PT>(opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, config, s); \
    }                                                                                              \
    extern "C" mp_status mp_gemm_##S(int opA, int opB, int64_t m, int64_t n, int64_t k,            \
                                     const PT::T *A, int64_t lda, int64_t pA, const PT::T *B,     \
                                     int64_t ldb, int64_t pB, PT::T *C, int64_t ldc, int64_t pC,  \
                                     mp_stream s)                                                 \
    {                                                                                              \
        return gemm_launch<PT>(opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, -1, s);     \
    }                                                                                              \
    extern "C" int mp_gemm_num_configs_##S(void) { return GemmTable<PT>::count; }                 \
    extern "C" const char *mp_gemm_config_name_##S(int c) { return GemmTable<PT>::name(c); }

#ifndef MPGPU_GEMM_PREC
#error "compile k_gemm.cu with -DMPGPU_GEMM_PREC=<dd|ddc|td|qd|ds|tf|qf>"
#endif
#define MP_CAT2(a, b) a##b
#define MP_CAT(a, b) MP_CAT2(a, b)
#define MP_EXPORT_GEMM_EXPANDED(S, PT) MP_EXPORT_GEMM(S, PT)
MP_EXPORT_GEMM_EXPANDED(MPGPU_GEMM_PREC, MP_CAT(P_, MPGPU_GEMM_PREC))
