// k_strassen.cu -- real C := A B by Strassen's recursion, the matrix
// multiplication scheme of Section 3.1 (recursion ending below a cutoff; the
// paper's is 32), with Strassen's seven products:
//   M1 = (A11 + A22)(B11 + B22)   M2 = (A21 + A22) B11   M3 = A11 (B12 - B22)
//   M4 = A22 (B21 - B11)          M5 = (A11 + A12) B22   M6 = (A21 - A11)(B11 + B12)
//   M7 = (A12 - A22)(B21 + B22)
//   C11 = ((M1 + M4) - M5) + M7   C12 = M3 + M5   C21 = M2 + M4
//   C22 = ((M1 - M2) + M3) + M6.
// A node of sizes (m, n, k) with min(m, n, k) < cutoff is one classical
// multicomponent GEMM (mp_gemm_ex_P, sequential k).  Otherwise its quadrants are
// ceil(m/2) x ceil(k/2) and ceil(k/2) x ceil(n/2) blocks, zero-padded where a
// dimension is odd; sums and differences are elementwise multicomponent adds (a
// difference adds the negated operand), a padded entry taking part as +0.
//
// GPU form: the recursion runs depth first on the host, on one stream.  Each
// level owns three buffers in the caller's workspace -- the left operand S,
// the right operand T and the product M -- reused by its seven products; the
// quadrants of C are accumulated in place in the order of the formulas above
// (C11 = M1, then + M4, - M5, + M7; ...), so no level keeps more than one
// product.  The leaves are the library's GEMM kernels; operands that are plain
// quadrants of A or B (A11, B11, and A22, B22 when unpadded) are passed as views.
#include <cuda_runtime.h>

#include "mp_arith.cuh"
#include "mp_common.cuh"

namespace mp {

template <class P> struct StrassenLeaf;
#define MP_STRASSEN_LEAF(PT, FN)                                                              \
    template <> struct StrassenLeaf<PT> {                                                      \
        template <typename... A> static mp_status run(A... a) { return FN(a...); }            \
    };
MP_STRASSEN_LEAF(P_dd, mp_gemm_ex_dd)
MP_STRASSEN_LEAF(P_ddc, mp_gemm_ex_ddc)
MP_STRASSEN_LEAF(P_td, mp_gemm_ex_td)
MP_STRASSEN_LEAF(P_qd, mp_gemm_ex_qd)
MP_STRASSEN_LEAF(P_tdc, mp_gemm_ex_tdc)
MP_STRASSEN_LEAF(P_qdc, mp_gemm_ex_qdc)
MP_STRASSEN_LEAF(P_ds, mp_gemm_ex_ds)
MP_STRASSEN_LEAF(P_tf, mp_gemm_ex_tf)
MP_STRASSEN_LEAF(P_qf, mp_gemm_ex_qf)
#undef MP_STRASSEN_LEAF

// out (r x c, packed, plane stride r*c) = X' + Y' or X' - Y' (sub), where X' is the
// block of the view X (xr x xc valid entries, leading dimension ldx, plane stride
// px) zero-padded to r x c, and likewise Y'.  Y == nullptr: out = X' (a copy).
template <class P>
__global__ void __launch_bounds__(256) k_pad_sum(int64_t r, int64_t c, const typename P::T *__restrict__ X,
                                                 int64_t ldx, int64_t px, int64_t xr, int64_t xc,
                                                 const typename P::T *__restrict__ Y, int64_t ldy, int64_t py,
                                                 int64_t yr, int64_t yc, int sub, typename P::T *__restrict__ out)
{
    const int64_t total = r * c;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t i = t / c, j = t % c;
        const typename P::V x = (i < xr && j < xc) ? vload<P>(X, px, i * ldx + j) : vzero<P>();
        if (Y == nullptr) {
            vstore<P>(out, total, t, x);
            continue;
        }
        const typename P::V y = (i < yr && j < yc) ? vload<P>(Y, py, i * ldy + j) : vzero<P>();
        vstore<P>(out, total, t, sub ? vsub<P>(x, y) : P::add(x, y));
    }
}

// C (r x c view, leading dimension ldc, plane stride pC) = M (mode 0), C + M
// (mode 1) or C - M (mode 2); M has leading dimension ldm and plane stride pm.
template <class P>
__global__ void __launch_bounds__(256) k_acc2d(int64_t r, int64_t c, typename P::T *__restrict__ C, int64_t ldc,
                                               int64_t pC, const typename P::T *__restrict__ M, int64_t ldm,
                                               int64_t pm, int mode)
{
    const int64_t total = r * c;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t i = t / c, j = t % c;
        const typename P::V mv = vload<P>(M, pm, i * ldm + j);
        typename P::V out = mv;
        if (mode != 0) {
            const typename P::V cv = vload<P>(C, pC, i * ldc + j);
            out = mode == 1 ? P::add(cv, mv) : vsub<P>(cv, mv);
        }
        vstore<P>(C, pC, i * ldc + j, out);
    }
}

static size_t align256s(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace bytes of the recursion below a node of sizes (m, n, k).
template <class P> static size_t strassen_ws(int64_t m, int64_t n, int64_t k, int64_t cutoff)
{
    const size_t e = P::K * sizeof(typename P::T);
    size_t total = 0;
    while (cutoff >= 2 && m >= cutoff && n >= cutoff && k >= cutoff) {
        const int64_t hm = (m + 1) / 2, hk = (k + 1) / 2, hn = (n + 1) / 2;
        total += align256s(e * (size_t)(hm * hk)) + align256s(e * (size_t)(hk * hn)) + align256s(e * (size_t)(hm * hn));
        m = hm;
        n = hn;
        k = hk;
    }
    return total;
}

template <class P> struct StrassenRun {
    using T = typename P::T;
    int64_t cutoff;
    mp_stream s;
    cudaStream_t st;

    mp_status pad_sum(int64_t r, int64_t c, const T *X, int64_t ldx, int64_t px, int64_t xr, int64_t xc,
                      const T *Y, int64_t ldy, int64_t py, int64_t yr, int64_t yc, int sub, T *out)
    {
        k_pad_sum<P><<<grid_for(r * c, 256, 8), 256, 0, st>>>(r, c, X, ldx, px, xr, xc, Y, ldy, py, yr, yc, sub,
                                                               out);
        return launch_status();
    }

    mp_status acc(int64_t r, int64_t c, T *C, int64_t ldc, int64_t pC, const T *M, int64_t ldm, int64_t pm,
                  int mode)
    {
        k_acc2d<P><<<grid_for(r * c, 256, 8), 256, 0, st>>>(r, c, C, ldc, pC, M, ldm, pm, mode);
        return launch_status();
    }

    mp_status node(int64_t m, int64_t n, int64_t k, const T *A, int64_t lda, int64_t pA, const T *B, int64_t ldb,
                   int64_t pB, T *C, int64_t ldc, int64_t pC, char *ws)
    {
        if (m < cutoff || n < cutoff || k < cutoff)
            return StrassenLeaf<P>::run(0, 0, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, -1, s);
        const int64_t hm = (m + 1) / 2, hk = (k + 1) / 2, hn = (n + 1) / 2;
        const int64_t m2 = m - hm, k2 = k - hk, n2 = n - hn;
        const int64_t na = hm * hk, nb = hk * hn, nc = hm * hn;
        const size_t e = P::K * sizeof(T);
        T *S = reinterpret_cast<T *>(ws);
        T *Tb = reinterpret_cast<T *>(ws + align256s(e * (size_t)na));
        T *M = reinterpret_cast<T *>(ws + align256s(e * (size_t)na) + align256s(e * (size_t)nb));
        char *child = ws + align256s(e * (size_t)na) + align256s(e * (size_t)nb) + align256s(e * (size_t)nc);
        // quadrant views (plane strides stay those of A, B, C)
        const T *A11 = A, *A12 = A + hk, *A21 = A + hm * lda, *A22 = A + hm * lda + hk;
        const T *B11 = B, *B12 = B + hn, *B21 = B + hk * ldb, *B22 = B + hk * ldb + hn;
        T *C11 = C, *C12 = C + hn, *C21 = C + hm * ldc, *C22 = C + hm * ldc + hn;
        mp_status r;
#define MP_TRY(x)                          \
    if ((r = (x)) != MP_OK) return r;
        // M1 = (A11 + A22)(B11 + B22): C11 = M1, C22 = M1
        MP_TRY(pad_sum(hm, hk, A11, lda, pA, hm, hk, A22, lda, pA, m2, k2, 0, S));
        MP_TRY(pad_sum(hk, hn, B11, ldb, pB, hk, hn, B22, ldb, pB, k2, n2, 0, Tb));
        MP_TRY(node(hm, hn, hk, S, hk, na, Tb, hn, nb, M, hn, nc, child));
        MP_TRY(acc(hm, hn, C11, ldc, pC, M, hn, nc, 0));
        MP_TRY(acc(m2, n2, C22, ldc, pC, M, hn, nc, 0));
        // M2 = (A21 + A22) B11: C21 = M2, C22 -= M2
        MP_TRY(pad_sum(hm, hk, A21, lda, pA, m2, hk, A22, lda, pA, m2, k2, 0, S));
        MP_TRY(node(hm, hn, hk, S, hk, na, B11, ldb, pB, M, hn, nc, child));
        MP_TRY(acc(m2, hn, C21, ldc, pC, M, hn, nc, 0));
        MP_TRY(acc(m2, n2, C22, ldc, pC, M, hn, nc, 2));
        // M3 = A11 (B12 - B22): C12 = M3, C22 += M3
        MP_TRY(pad_sum(hk, hn, B12, ldb, pB, hk, n2, B22, ldb, pB, k2, n2, 1, Tb));
        MP_TRY(node(hm, hn, hk, A11, lda, pA, Tb, hn, nb, M, hn, nc, child));
        MP_TRY(acc(hm, n2, C12, ldc, pC, M, hn, nc, 0));
        MP_TRY(acc(m2, n2, C22, ldc, pC, M, hn, nc, 1));
        // M4 = A22 (B21 - B11): C11 += M4, C21 += M4
        MP_TRY(pad_sum(hk, hn, B21, ldb, pB, k2, hn, B11, ldb, pB, hk, hn, 1, Tb));
        if (m2 == hm && k2 == hk) {
            MP_TRY(node(hm, hn, hk, A22, lda, pA, Tb, hn, nb, M, hn, nc, child));
        } else {
            MP_TRY(pad_sum(hm, hk, A22, lda, pA, m2, k2, nullptr, 0, 0, 0, 0, 0, S));
            MP_TRY(node(hm, hn, hk, S, hk, na, Tb, hn, nb, M, hn, nc, child));
        }
        MP_TRY(acc(hm, hn, C11, ldc, pC, M, hn, nc, 1));
        MP_TRY(acc(m2, hn, C21, ldc, pC, M, hn, nc, 1));
        // M5 = (A11 + A12) B22: C11 -= M5, C12 += M5
        MP_TRY(pad_sum(hm, hk, A11, lda, pA, hm, hk, A12, lda, pA, hm, k2, 0, S));
        if (k2 == hk && n2 == hn) {
            MP_TRY(node(hm, hn, hk, S, hk, na, B22, ldb, pB, M, hn, nc, child));
        } else {
            MP_TRY(pad_sum(hk, hn, B22, ldb, pB, k2, n2, nullptr, 0, 0, 0, 0, 0, Tb));
            MP_TRY(node(hm, hn, hk, S, hk, na, Tb, hn, nb, M, hn, nc, child));
        }
        MP_TRY(acc(hm, hn, C11, ldc, pC, M, hn, nc, 2));
        MP_TRY(acc(hm, n2, C12, ldc, pC, M, hn, nc, 1));
        // M6 = (A21 - A11)(B11 + B12): C22 += M6
        MP_TRY(pad_sum(hm, hk, A21, lda, pA, m2, hk, A11, lda, pA, hm, hk, 1, S));
        MP_TRY(pad_sum(hk, hn, B11, ldb, pB, hk, hn, B12, ldb, pB, hk, n2, 0, Tb));
        MP_TRY(node(hm, hn, hk, S, hk, na, Tb, hn, nb, M, hn, nc, child));
        MP_TRY(acc(m2, n2, C22, ldc, pC, M, hn, nc, 1));
        // M7 = (A12 - A22)(B21 + B22): C11 += M7
        MP_TRY(pad_sum(hm, hk, A12, lda, pA, hm, k2, A22, lda, pA, m2, k2, 1, S));
        MP_TRY(pad_sum(hk, hn, B21, ldb, pB, k2, hn, B22, ldb, pB, k2, n2, 0, Tb));
        MP_TRY(node(hm, hn, hk, S, hk, na, Tb, hn, nb, M, hn, nc, child));
        MP_TRY(acc(hm, hn, C11, ldc, pC, M, hn, nc, 1));
#undef MP_TRY
        return MP_OK;
    }
};

template <class P>
static mp_status strassen_launch(int64_t m, int64_t n, int64_t k, const typename P::T *A, int64_t lda, int64_t pA,
                                 const typename P::T *B, int64_t ldb, int64_t pB, typename P::T *C, int64_t ldc,
                                 int64_t pC, int64_t cutoff, void *ws, size_t ws_bytes, mp_stream s)
{
    if (m < 0 || n < 0 || k < 0 || cutoff < 2) return MP_EINVAL;
    if (m == 0 || n == 0) return MP_OK;
    if (C == nullptr || ldc < n || pC < (m - 1) * ldc + n) return MP_EINVAL;
    if (k > 0) {
        if (A == nullptr || lda < k || pA < (m - 1) * lda + k) return MP_EINVAL;
        if (B == nullptr || ldb < n || pB < (k - 1) * ldb + n) return MP_EINVAL;
    }
    const size_t need = strassen_ws<P>(m, n, k, cutoff);
    if (need > 0 && (ws == nullptr || ws_bytes < need)) return MP_ENOMEM;
    StrassenRun<P> run{cutoff, s, as_stream(s)};
    return run.node(m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, static_cast<char *>(ws));
}

}  // namespace mp

using namespace mp;

extern "C" {

#define MP_EXPORT_STRASSEN(S, PT)                                                                      \
    size_t mp_gemm_strassen_workspace_##S(int64_t m, int64_t n, int64_t k, int64_t cutoff)            \
    {                                                                                                  \
        if (m < 0 || n < 0 || k < 0) return 0;                                                         \
        return strassen_ws<PT>(m, n, k, cutoff);                                                       \
    }                                                                                                  \
    mp_status mp_gemm_strassen_##S(int64_t m, int64_t n, int64_t k, const PT::T *A, int64_t lda,       \
                                   int64_t pA, const PT::T *B, int64_t ldb, int64_t pB, PT::T *C,      \
                                   int64_t ldc, int64_t pC, int64_t cutoff, void *ws, size_t ws_bytes, \
                                   mp_stream s)                                                        \
    {                                                                                                  \
        return strassen_launch<PT>(m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, cutoff, ws, ws_bytes, s); \
    }

MP_EXPORT_STRASSEN(dd, P_dd)
MP_EXPORT_STRASSEN(ddc, P_ddc)
MP_EXPORT_STRASSEN(td, P_td)
MP_EXPORT_STRASSEN(qd, P_qd)
MP_EXPORT_STRASSEN(tdc, P_tdc)
MP_EXPORT_STRASSEN(qdc, P_qdc)
MP_EXPORT_STRASSEN(ds, P_ds)
MP_EXPORT_STRASSEN(tf, P_tf)
MP_EXPORT_STRASSEN(qf, P_qf)

}  // extern "C"
