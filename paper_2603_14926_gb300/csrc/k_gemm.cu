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
#include <cuda.h>
#include <cudaTypedefs.h>
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

// The hybrid engine's rare way out: a thread whose integer path left its domain
// (failed()) recomputes its own outputs with the FP64 pipe, reading op(A) and
// op(B) from global memory in the same fold order, so its bits are the FP64
// sequence's.  Never taken on data whose components stay far from the binary64
// range limits.
static __device__ unsigned int mp_hybrid_fallbacks;

template <class P, int TM, int TN, int NTX, int NTY>
__device__ __noinline__ void gemm_fixup(int opA, int opB, int64_t k, const typename P::T *__restrict__ A, int64_t lda,
                                        int64_t pA, const typename P::T *__restrict__ B, int64_t ldb, int64_t pB,
                                        int64_t i0, int64_t j0, int ty, int tx, int64_t m, int64_t n,
                                        typename P::T *__restrict__ C, int64_t ldc, int64_t pC)
{
    using T = typename P::T;
    using V = typename P::V;
    NativeEngine<T> nat;
    atomicAdd(&mp_hybrid_fallbacks, 1u);
    for (int r = 0; r < TM; r++) {
        const int64_t gi = i0 + ty + r * NTY;
        if (gi >= m) continue;
        for (int q = 0; q < TN; q++) {
            const int64_t gj = j0 + tx + q * NTX;
            if (gj >= n) continue;
            V acc = vzero<P>();
            for (int64_t l = 0; l < k; l++) {
                const V a = vload<P>(A, pA, opA == 0 ? gi * lda + l : l * lda + gi);
                const V b = vload<P>(B, pB, opB == 0 ? l * ldb + gj : gj * ldb + l);
                acc = P::add(acc, P::mul(a, b, nat), nat);
            }
            vstore<P>(C, pC, gi * ldc + gj, acc);
        }
    }
}

template <class P, class E, int MINB, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(GemmCfg<P, BM, BN, BK, TM, TN>::NT, MINB)
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
    E eng;
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
                for (int s = 0; s < TN; s++) acc[r][s] = P::add(acc[r][s], P::mul(a[r], b[s], eng), eng);
        }
        __syncthreads();
    }
    if (eng.failed()) {
        gemm_fixup<P, TM, TN, G::NTX, G::NTY>(opA, opB, k, A, lda, pA, B, ldb, pB, i0, j0, ty, tx, m, n, C, ldc, pC);
        return;
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

template <class P, class E, int MINB, int BM, int BN, int BK, int TM, int TN>
static mp_status gemm_run(int opA, int opB, int64_t m, int64_t n, int64_t k, const typename P::T *A,
                          int64_t lda, int64_t pA, const typename P::T *B, int64_t ldb, int64_t pB,
                          typename P::T *C, int64_t ldc, int64_t pC, cudaStream_t s)
{
    using G = GemmCfg<P, BM, BN, BK, TM, TN>;
    const int64_t gx = (n + BN - 1) / BN, gy = (m + BM - 1) / BM;
    if (gx * gy > 0x7fffffff) return MP_EINVAL;
    dim3 grid((unsigned)(gx * gy));
    k_gemm<P, E, MINB, BM, BN, BK, TM, TN><<<grid, G::NT, 0, s>>>(opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C,
                                                                   ldc, pC);
    return launch_status();
}

// ---------------------------------------------------------------------------
// TMA-staged variant: the op(A) and op(B) tiles of every k-step arrive in
// shared memory by cp.async.bulk.tensor (3-D tensor maps over contiguous
// dimension x rows x component planes, zero-filled past the matrix edges),
// double-buffered: while the block computes on one stage, the copy of the
// k-tile after next lands in the other.  One thread issues the copies; every
// thread waits on the stage's mbarrier with an iteration limit.  If a wait ever
// runs out, the block agrees on it (__syncthreads_or), counts it in
// mp_tma_timeouts, waits (bounded) for its copies still in flight and returns,
// so a fault in the copy path can never hang the GPU.  Same fold, same bits as
// the plain kernel.
// ---------------------------------------------------------------------------

static __device__ unsigned int mp_tma_timeouts;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// true when the phase with this parity completed within the iteration limit
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 24); i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <class P, class E, int MINB, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(GemmCfg<P, BM, BN, BK, TM, TN>::NT, MINB)
    k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int opA, int opB,
               int64_t m, int64_t n, int64_t k, const typename P::T *__restrict__ A, int64_t lda, int64_t pA,
               const typename P::T *__restrict__ B, int64_t ldb, int64_t pB, typename P::T *__restrict__ C,
               int64_t ldc, int64_t pC)
{
    using T = typename P::T;
    using V = typename P::V;
    using G = GemmCfg<P, BM, BN, BK, TM, TN>;
    constexpr int K = P::K;
    constexpr int AE = K * BM * BK, BE = K * BK * BN;  // elements per stage
    static_assert((AE * sizeof(T)) % 128 == 0 && (BE * sizeof(T)) % 128 == 0, "stage alignment");
    extern __shared__ __align__(1024) unsigned char tma_smem[];
    T *const base = reinterpret_cast<T *>(tma_smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + 2 * (AE + BE));

    const int tid = threadIdx.x;
    const int tx = tid % G::NTX, ty = tid / G::NTX;
    const int64_t tm = (m + BM - 1) / BM, tn = (n + BN - 1) / BN;
    const int64_t per_group = GEMM_GROUP * tn;
    const int64_t L = blockIdx.x, g = L / per_group, first = g * GEMM_GROUP;
    const int64_t rows = tm - first < GEMM_GROUP ? tm - first : GEMM_GROUP;
    const int64_t r_in = L - g * per_group;
    const int64_t i0 = (first + r_in % rows) * BM, j0 = (r_in / rows) * BN;
    const int64_t ktiles = (k + BK - 1) / BK;
    const uint32_t bytes = (uint32_t)((AE + BE) * sizeof(T));

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t t, int s) {
        T *sa = base + s * (AE + BE), *sb = sa + AE;
        const int k0 = (int)(t * BK);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bars[s], bytes);
        if (opA == 0) tma_load_3d(sa, &tmA, &bars[s], k0, (int)i0, 0);
        else tma_load_3d(sa, &tmA, &bars[s], (int)i0, k0, 0);
        if (opB == 0) tma_load_3d(sb, &tmB, &bars[s], (int)j0, k0, 0);
        else tma_load_3d(sb, &tmB, &bars[s], k0, (int)j0, 0);
    };
    if (tid == 0) {
        if (ktiles > 0) issue(0, 0);
        if (ktiles > 1) issue(1, 1);
    }

    V acc[TM][TN];
    E eng;
#pragma unroll
    for (int r = 0; r < TM; r++)
#pragma unroll
        for (int s = 0; s < TN; s++) acc[r][s] = vzero<P>();

    for (int64_t t = 0; t < ktiles; t++) {
        const int s = (int)(t & 1);
        const uint32_t par = (uint32_t)((t >> 1) & 1);
        const bool ok = mbar_wait_bounded(&bars[s], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicAdd(&mp_tma_timeouts, 1u);
                if (t + 1 < ktiles) mbar_wait_bounded(&bars[s ^ 1], (uint32_t)(((t + 1) >> 1) & 1));
            }
            return;
        }
        const T *sa = base + s * (AE + BE), *sb = sa + AE;
        const int kc = (int)((k - t * BK) < BK ? (k - t * BK) : BK);
#pragma unroll 1
        for (int kk = 0; kk < kc; kk++) {
            V a[TM], b[TN];
#pragma unroll
            for (int r = 0; r < TM; r++) {
                const int i = ty + r * G::NTY;
#pragma unroll
                for (int c = 0; c < K; c++)
                    a[r].c[c] = opA == 0 ? sa[(c * BM + i) * BK + kk] : sa[(c * BK + kk) * BM + i];
            }
#pragma unroll
            for (int q = 0; q < TN; q++) {
                const int j = tx + q * G::NTX;
#pragma unroll
                for (int c = 0; c < K; c++)
                    b[q].c[c] = opB == 0 ? sb[(c * BK + kk) * BN + j] : sb[(c * BN + j) * BK + kk];
            }
#pragma unroll
            for (int r = 0; r < TM; r++)
#pragma unroll
                for (int q = 0; q < TN; q++) acc[r][q] = P::add(acc[r][q], P::mul(a[r], b[q], eng), eng);
        }
        __syncthreads();  // every read of stage s is done before it is refilled
        if (tid == 0 && t + 2 < ktiles) issue(t + 2, s);
    }
    if (eng.failed()) {
        gemm_fixup<P, TM, TN, G::NTX, G::NTY>(opA, opB, k, A, lda, pA, B, ldb, pB, i0, j0, ty, tx, m, n, C, ldc, pC);
        return;
    }
#pragma unroll
    for (int r = 0; r < TM; r++) {
        const int64_t gi = i0 + ty + r * G::NTY;
        if (gi >= m) continue;
#pragma unroll
        for (int q = 0; q < TN; q++) {
            const int64_t gj = j0 + tx + q * G::NTX;
            if (gj < n) vstore<P>(C, pC, gi * ldc + gj, acc[r][q]);
        }
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D map of a K-plane matrix: dims (inner, outer, K), box (bi, bo, K).  False when
// TMA's rules are not met (16-byte aligned base, 16-byte multiple strides), so the
// caller can use the plain kernel instead.
template <class P>
static bool make_tensor_map(CUtensorMap *map, const typename P::T *ptr, int64_t inner, int64_t outer, int64_t ld,
                            int64_t ps, int bi, int bo)
{
    using T = typename P::T;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc == nullptr || ptr == nullptr || inner <= 0 || outer <= 0) return false;
    if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return false;
    if ((ld * (int64_t)sizeof(T)) % 16 != 0 || (ps * (int64_t)sizeof(T)) % 16 != 0) return false;
    if (ld * (int64_t)sizeof(T) >= (1LL << 40) || ps * (int64_t)sizeof(T) >= (1LL << 40)) return false;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)P::K};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * sizeof(T)), (cuuint64_t)(ps * sizeof(T))};
    cuuint32_t box[3] = {(cuuint32_t)bi, (cuuint32_t)bo, (cuuint32_t)P::K};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return enc(map, dt, 3, const_cast<T *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class P, class E, int MINB, int BM, int BN, int BK, int TM, int TN>
static mp_status gemm_run_tma(int opA, int opB, int64_t m, int64_t n, int64_t k, const typename P::T *A, int64_t lda,
                              int64_t pA, const typename P::T *B, int64_t ldb, int64_t pB, typename P::T *C, int64_t ldc,
                              int64_t pC, cudaStream_t s)
{
    using T = typename P::T;
    using G = GemmCfg<P, BM, BN, BK, TM, TN>;
    CUtensorMap ma, mb;
    const bool ok = k > 0 && (opA == 0 ? make_tensor_map<P>(&ma, A, k, m, lda, pA, BK, BM)
                                       : make_tensor_map<P>(&ma, A, m, k, lda, pA, BM, BK)) &&
                    (opB == 0 ? make_tensor_map<P>(&mb, B, n, k, ldb, pB, BN, BK)
                              : make_tensor_map<P>(&mb, B, k, n, ldb, pB, BK, BN));
    if (!ok)  // layout outside TMA's rules: the plain kernel computes the same bits
        return gemm_run<P, E, MINB, BM, BN, BK, TM, TN>(opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, s);
    const int64_t gx = (n + BN - 1) / BN, gy = (m + BM - 1) / BM;
    if (gx * gy > 0x7fffffff) return MP_EINVAL;
    const size_t smem = 2 * (size_t)P::K * (BM * BK + BK * BN) * sizeof(T) + 2 * sizeof(uint64_t);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tma<P, E, MINB, BM, BN, BK, TM, TN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    k_gemm_tma<P, E, MINB, BM, BN, BK, TM, TN><<<(unsigned)(gx * gy), G::NT, smem, s>>>(
        ma, mb, opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC);
    return launch_status();
}

// Tile configurations.  Binary64 precisions are FP64-pipe bound, so one chain
// per thread suffices: the built-in choice is the TMA-staged 16x16 tile with one
// output per thread on the hybrid engine (configuration 10).  At QD n = 2048 it
// issues FP64 work at the rate DFMA chains reach (1594 ms against 1692 ms for
// 32x32 tiles with 2x2 micro-tiles, whose four chains per thread spill at the
// two-blocks-per-SM register budget; n = 1024: 199.5 against 224.3 ms, where
// its 16384 tiles also fill the last wave).  Same bits in every configuration.
// For binary32 the 32x32 tile with 2x2 micro-tiles measured fastest (QF
// n = 2048: 34.1 T FP32 instructions/s against 29.5 T for 64x64).
template <class P, bool F64 = P::fp64> struct GemmTable;

template <class P> struct GemmTable<P, true> {
    using N = NativeEngine<double>;
    using H = HybridEngine<false>;
    using HQ = HybridEngine<true>;
    using HP = HybridEngine<false, true>;
    static constexpr int count = 11;
    static const char *name(int c)
    {
        switch (c) {
        case 0: return "BM32 BN32 BK16 TM2 TN2 (256 thr)";
        case 1: return "BM16 BN16 BK16 TM1 TN1 (256 thr)";
        case 2: return "BM32 BN64 BK8 TM2 TN4 (256 thr)";
        case 3: return "BM16 BN32 BK16 TM1 TN2 (256 thr)";
        case 4: return "BM32 BN32 BK16 TM2 TN2 (256 thr), TMA-staged double buffer";
        case 5: return "BM32 BN32 BK16 TM2 TN2 (256 thr), TMA, hybrid TwoSum (integer error term)";
        case 6: return "BM32 BN32 BK16 TM2 TN2 (256 thr), TMA, hybrid TwoSum + QuickTwoSum";
        case 7: return "BM32 BN32 BK16 TM2 TN2 (256 thr), hybrid TwoSum";
        case 8: return "BM32 BN32 BK16 TM2 TN2 (256 thr), TMA, hybrid TwoSum, 1 block/SM register budget";
        case 9: return "BM32 BN32 BK16 TM2 TN2 (256 thr), TMA, hybrid TwoSum + TwoProd";
        case 10: return "BM16 BN16 BK16 TM1 TN1 (256 thr), TMA, hybrid TwoSum (integer error term)";
        }
        return nullptr;
    }
    static constexpr int fallback = 10;  // configuration used for config = -1
    template <typename... Args> static mp_status run(int c, Args... a)
    {
        switch (c) {
        case 1: return gemm_run<P, N, 2, 16, 16, 16, 1, 1>(a...);
        case 2: return gemm_run<P, N, 1, 32, 64, 8, 2, 4>(a...);
        case 3: return gemm_run<P, N, 2, 16, 32, 16, 1, 2>(a...);
        case 4: return gemm_run_tma<P, N, 2, 32, 32, 16, 2, 2>(a...);
        case 5: return gemm_run_tma<P, H, 2, 32, 32, 16, 2, 2>(a...);
        case 6: return gemm_run_tma<P, HQ, 2, 32, 32, 16, 2, 2>(a...);
        case 7: return gemm_run<P, H, 2, 32, 32, 16, 2, 2>(a...);
        case 8: return gemm_run_tma<P, H, 1, 32, 32, 16, 2, 2>(a...);
        case 9: return gemm_run_tma<P, HP, 2, 32, 32, 16, 2, 2>(a...);
        case 10: return gemm_run_tma<P, H, 2, 16, 16, 16, 1, 1>(a...);
        default: return gemm_run<P, N, 2, 32, 32, 16, 2, 2>(a...);
        }
    }
};

template <class P> struct GemmTable<P, false> {
    using N = NativeEngine<float>;
    static constexpr int count = 5;
    static const char *name(int c)
    {
        switch (c) {
        case 0: return "BM32 BN32 BK16 TM2 TN2 (256 thr)";
        case 1: return "BM64 BN64 BK16 TM4 TN4 (256 thr)";
        case 2: return "BM64 BN32 BK16 TM4 TN2 (256 thr)";
        case 3: return "BM128 BN64 BK8 TM8 TN4 (256 thr)";
        case 4: return "BM32 BN32 BK16 TM2 TN2 (256 thr), TMA-staged double buffer";
        }
        return nullptr;
    }
    static constexpr int fallback = 0;  // configuration used for config = -1
    template <typename... Args> static mp_status run(int c, Args... a)
    {
        switch (c) {
        case 1: return gemm_run<P, N, 1, 64, 64, 16, 4, 4>(a...);
        case 2: return gemm_run<P, N, 1, 64, 32, 16, 4, 2>(a...);
        case 3: return gemm_run<P, N, 1, 128, 64, 8, 8, 4>(a...);
        case 4: return gemm_run_tma<P, N, 1, 32, 32, 16, 2, 2>(a...);
        default: return gemm_run<P, N, 1, 32, 32, 16, 2, 2>(a...);
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
    return GemmTable<P>::run(config < 0 ? GemmTable<P>::fallback : config, opA, opB, m, n, k, A, lda, pA, B, ldb,
                             pB, C, ldc, pC, as_stream(s));
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
    extern "C" mp_status mp_gemm_tma_timeouts_##S(unsigned int *count)                             \
    {                                                                                              \
        if (count == nullptr) return MP_EINVAL;                                                    \
        return cuda_status(cudaMemcpyFromSymbol(count, mp_tma_timeouts, sizeof(unsigned int)));    \
    }                                                                                              \
    extern "C" mp_status mp_gemm_hybrid_fallbacks_##S(unsigned int *count)                         \
    {                                                                                              \
        if (count == nullptr) return MP_EINVAL;                                                    \
        return cuda_status(cudaMemcpyFromSymbol(count, mp_hybrid_fallbacks, sizeof(unsigned int))); \
    }                                                                                              \
    extern "C" const char *mp_gemm_config_name_##S(int c) { return GemmTable<PT>::name(c); }

#ifndef MPGPU_GEMM_PREC
#error "compile k_gemm.cu with -DMPGPU_GEMM_PREC=<dd|ddc|td|qd|tdc|qdc|ds|tf|qf>"
#endif
#define MP_CAT2(a, b) a##b
#define MP_CAT(a, b) MP_CAT2(a, b)
#define MP_EXPORT_GEMM_EXPANDED(S, PT) MP_EXPORT_GEMM(S, PT)
MP_EXPORT_GEMM_EXPANDED(MPGPU_GEMM_PREC, MP_CAT(P_, MPGPU_GEMM_PREC))
