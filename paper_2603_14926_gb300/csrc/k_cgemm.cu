// k_cgemm.cu -- complex C := op(A) op(B) by the 3M method (Section 3.2, Eq. 3):
//   C1 = Re A Re B,  C2 = Im A Im B,  Re C = C1 - C2,
//   Im C = (Re A + Im A)(Re B + Im B) - C1 - C2   (subtracted left to right).
// Three real multicomponent GEMMs (mp_gemm_ex_P, sequential k, bit-identical to
// the oracle), the operand sums in the operands' own storage layout, and one
// fused epilogue.  C1 is accumulated directly in Re C and C3 in Im C; the
// workspace holds Re A + Im A, Re B + Im B and C2.
#include <cuda_runtime.h>

#include "mp_arith.cuh"
#include "mp_common.cuh"

namespace mp {

template <class P> struct RealGemm;
#define MP_REAL_GEMM(PT, FN)                                                                  \
    template <> struct RealGemm<PT> {                                                          \
        template <typename... A> static mp_status run(A... a) { return FN(a...); }            \
    };
MP_REAL_GEMM(P_dd, mp_gemm_ex_dd)
MP_REAL_GEMM(P_ddc, mp_gemm_ex_ddc)
MP_REAL_GEMM(P_td, mp_gemm_ex_td)
MP_REAL_GEMM(P_qd, mp_gemm_ex_qd)
MP_REAL_GEMM(P_ds, mp_gemm_ex_ds)
MP_REAL_GEMM(P_tf, mp_gemm_ex_tf)
MP_REAL_GEMM(P_qf, mp_gemm_ex_qf)
#undef MP_REAL_GEMM

// out[r*ld + c] = a[..] + b[..] for every component plane (plane stride ps).
template <class P>
__global__ void __launch_bounds__(256) k_add2d(int64_t rows, int64_t cols, int64_t ld, int64_t ps,
                                               const typename P::T *__restrict__ a,
                                               const typename P::T *__restrict__ b,
                                               typename P::T *__restrict__ out)
{
    const int64_t total = rows * cols;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t idx = (t / cols) * ld + t % cols;
        vstore<P>(out, ps, idx, P::add(vload<P>(a, ps, idx), vload<P>(b, ps, idx)));
    }
}

// Re C = C1 - C2 (C1 in Cr), Im C = (C3 - C1) - C2 (C3 in Ci); C2 packed m x n.
template <class P>
__global__ void __launch_bounds__(256) k_cgemm_finish(int64_t m, int64_t n, typename P::T *__restrict__ Cr,
                                                      typename P::T *__restrict__ Ci, int64_t ldc, int64_t pC,
                                                      const typename P::T *__restrict__ C2)
{
    const int64_t total = m * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t idx = (t / n) * ldc + t % n;
        const typename P::V c1 = vload<P>(Cr, pC, idx), c3 = vload<P>(Ci, pC, idx), c2 = vload<P>(C2, total, t);
        vstore<P>(Ci, pC, idx, vsub<P>(vsub<P>(c3, c1), c2));
        vstore<P>(Cr, pC, idx, vsub<P>(c1, c2));
    }
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <class P> static size_t cgemm_ws(int64_t m, int64_t n, int64_t pA, int64_t pB)
{
    const size_t e = P::K * sizeof(typename P::T);
    if (m < 0 || n < 0 || pA < 0 || pB < 0) return 0;
    return align256(e * (size_t)pA) + align256(e * (size_t)pB) + align256(e * (size_t)(m * n));
}

template <class P>
static mp_status cgemm_launch(int opA, int opB, int64_t m, int64_t n, int64_t k, const typename P::T *Ar,
                              const typename P::T *Ai, int64_t lda, int64_t pA, const typename P::T *Br,
                              const typename P::T *Bi, int64_t ldb, int64_t pB, typename P::T *Cr,
                              typename P::T *Ci, int64_t ldc, int64_t pC, void *ws, size_t ws_bytes, mp_stream s)
{
    using T = typename P::T;
    if ((opA != 0 && opA != 1) || (opB != 0 && opB != 1) || m < 0 || n < 0 || k < 0) return MP_EINVAL;
    if (m == 0 || n == 0) return MP_OK;
    if (Cr == nullptr || Ci == nullptr || ldc < n || pC < (m - 1) * ldc + n) return MP_EINVAL;
    const int64_t ar = opA ? k : m, ac = opA ? m : k, br = opB ? n : k, bc = opB ? k : n;
    if (k > 0) {
        if (Ar == nullptr || Ai == nullptr || lda < ac || pA < (ar - 1) * lda + ac) return MP_EINVAL;
        if (Br == nullptr || Bi == nullptr || ldb < bc || pB < (br - 1) * ldb + bc) return MP_EINVAL;
    }
    if (ws == nullptr || ws_bytes < cgemm_ws<P>(m, n, k > 0 ? pA : 0, k > 0 ? pB : 0)) return MP_ENOMEM;
    const size_t e = P::K * sizeof(T);
    char *w = static_cast<char *>(ws);
    T *SA = reinterpret_cast<T *>(w);
    T *SB = reinterpret_cast<T *>(w + align256(e * (size_t)(k > 0 ? pA : 0)));
    T *C2 = reinterpret_cast<T *>(w + align256(e * (size_t)(k > 0 ? pA : 0)) + align256(e * (size_t)(k > 0 ? pB : 0)));
    cudaStream_t st = as_stream(s);
    if (k > 0) {
        k_add2d<P><<<grid_for(ar * ac, 256, 8), 256, 0, st>>>(ar, ac, lda, pA, Ar, Ai, SA);
        mp_status r = launch_status();
        if (r != MP_OK) return r;
        k_add2d<P><<<grid_for(br * bc, 256, 8), 256, 0, st>>>(br, bc, ldb, pB, Br, Bi, SB);
        if ((r = launch_status()) != MP_OK) return r;
    }
    mp_status r = RealGemm<P>::run(opA, opB, m, n, k, Ar, lda, pA, Br, ldb, pB, Cr, ldc, pC, -1, s);
    if (r != MP_OK) return r;
    if ((r = RealGemm<P>::run(opA, opB, m, n, k, Ai, lda, pA, Bi, ldb, pB, C2, n, m * n, -1, s)) != MP_OK)
        return r;
    if ((r = RealGemm<P>::run(opA, opB, m, n, k, SA, lda, pA, SB, ldb, pB, Ci, ldc, pC, -1, s)) != MP_OK)
        return r;
    k_cgemm_finish<P><<<grid_for(m * n, 256, 8), 256, 0, st>>>(m, n, Cr, Ci, ldc, pC, C2);
    return launch_status();
}

}  // namespace mp

using namespace mp;

extern "C" {

#define MP_EXPORT_CGEMM(S, PT)                                                                        \
    size_t mp_cgemm_workspace_##S(int64_t m, int64_t n, int64_t pA, int64_t pB)                       \
    {                                                                                                 \
        return cgemm_ws<PT>(m, n, pA, pB);                                                            \
    }                                                                                                 \
    mp_status mp_cgemm_##S(int opA, int opB, int64_t m, int64_t n, int64_t k, const PT::T *Ar,         \
                           const PT::T *Ai, int64_t lda, int64_t pA, const PT::T *Br, const PT::T *Bi, \
                           int64_t ldb, int64_t pB, PT::T *Cr, PT::T *Ci, int64_t ldc, int64_t pC,     \
                           void *ws, size_t ws_bytes, mp_stream s)                                    \
    {                                                                                                 \
        return cgemm_launch<PT>(opA, opB, m, n, k, Ar, Ai, lda, pA, Br, Bi, ldb, pB, Cr, Ci, ldc, pC, \
                                ws, ws_bytes, s);                                                     \
    }

MP_EXPORT_CGEMM(dd, P_dd)
MP_EXPORT_CGEMM(ddc, P_ddc)
MP_EXPORT_CGEMM(td, P_td)
MP_EXPORT_CGEMM(qd, P_qd)
MP_EXPORT_CGEMM(ds, P_ds)
MP_EXPORT_CGEMM(tf, P_tf)
MP_EXPORT_CGEMM(qf, P_qf)

}  // extern "C"
