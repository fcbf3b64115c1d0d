/*
 * mpref.c -- CPU oracle for branch-free multicomponent arithmetic
 * (Kouya, arXiv 2603.14926: Algorithms 1-14, Section 3 GEMM (classical fold,
 * Strassen's recursion, 3M complex), Section 4
 * polynomial evaluation and the Durand-Kerner solver).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, scalar restatement of the
 * method used to check the CUDA library (paper_2603_14926_gb300).  Only the
 * tests, the package's smoke check and the benchmark's CPU-baseline leg load
 * it.  It shares no code with the CUDA library.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared mpref.c -lm
 *        (add -DMPREF_COUNT for the operation-counting build).
 * -ffp-contract=off is required: GCC on AArch64 otherwise fuses a*b+c.
 *
 * Precisions (suffix: components x component type, add, multiply):
 *   dd  : 2 x binary64, Algorithm 6 (DWBFAdd),   Algorithm 8 (DWBFMul)
 *   ddc : 2 x binary64, Algorithm 4 (DWAdd),     Algorithm 7 (DWMul)  -- the
 *         conventional double-double the paper benchmarks as "DD"
 *   td  : 3 x binary64, Algorithm 11 (TWBFAdd),  Algorithm 12 (TWBFMul)
 *   tdc : 3 x binary64, Algorithm 9 (TWAdd),     Algorithm 10 (TWMul), each
 *         ending in TWRenormalize -- the conventional triple-word arithmetic
 *   qd  : 4 x binary64, Algorithm 13 (QWBFAdd),  Algorithm 14 (QDBFMul)
 *   qdc : 4 x binary64, the QD library's quad-word add and multiply, each
 *         ending in QWRenormalize -- the conventional quad-word arithmetic
 *   ds  : 2 x binary32, Algorithms 6 / 8
 *   tf  : 3 x binary32, Algorithms 11 / 12
 *   qf  : 4 x binary32, Algorithms 13 / 14
 * Array layout everywhere: a K-array of n numbers is K planes; component c of
 * element i is at ptr[c*plane_stride + i]; component 0 is the leading one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__FAST_MATH__)
#error "the oracle must not be built with fast-math"
#endif

#define MPREF_CAT2(a, b) a##b
#define MPREF_CAT(a, b) MPREF_CAT2(a, b)

/* operation counters: [0]=add [1]=sub [2]=mul [3]=fma */
static int64_t mpref_cnt[4];

#ifdef MPREF_COUNT
#define ADD(x, y) (mpref_cnt[0]++, (REAL)((x) + (y)))
#define SUB(x, y) (mpref_cnt[1]++, (REAL)((x) - (y)))
#define MUL(x, y) (mpref_cnt[2]++, (REAL)((x) * (y)))
#define FMA(x, y, z) (mpref_cnt[3]++, (REAL)FMA_FN((x), (y), (z)))
#else
#define ADD(x, y) ((REAL)((x) + (y)))
#define SUB(x, y) ((REAL)((x) - (y)))
#define MUL(x, y) ((REAL)((x) * (y)))
#define FMA(x, y, z) ((REAL)FMA_FN((x), (y), (z)))
#endif

/* ---- binary64 components ---- */
#define REAL double
#define SFX _d
#define FMA_FN fma
#include "mpref_core.inc"
#include "mpref_dk.inc"
#undef REAL
#undef SFX
#undef FMA_FN

/* ---- binary32 components ---- */
#define REAL float
#define SFX _f
#define FMA_FN fmaf
#include "mpref_core.inc"
#undef REAL
#undef SFX
#undef FMA_FN

/* Newton steps for the reciprocal: y_0 has the component type's precision p0 and
 * each step roughly doubles the correct bits; K=2 and K=3 take 2 steps, K=4 takes 3. */
static const prec_d P_dd = {2, dw_add_bf_d, dw_mul_bf_d, 2};
static const prec_d P_ddc = {2, dw_add_sloppy_d, dw_mul_d, 2};
static const prec_d P_td = {3, tw_add_bf_d, tw_mul_bf_d, 2};
static const prec_d P_qd = {4, qw_add_bf_d, qw_mul_bf_d, 3};
static const prec_d P_tdc = {3, tw_add_d, tw_mul_d, 2};
static const prec_d P_qdc = {4, qw_add_d, qw_mul_d, 3};
static const prec_f P_ds = {2, dw_add_bf_f, dw_mul_bf_f, 2};
static const prec_f P_tf = {3, tw_add_bf_f, tw_mul_bf_f, 2};
static const prec_f P_qf = {4, qw_add_bf_f, qw_mul_bf_f, 3};

/* ------------------------------------------------------------------------- */
/* Exports                                                                    */
/* ------------------------------------------------------------------------- */

void mpref_count_reset(void) { memset(mpref_cnt, 0, sizeof mpref_cnt); }
void mpref_count_get(int64_t out[4]) { memcpy(out, mpref_cnt, sizeof mpref_cnt); }
int mpref_is_counting(void)
{
#ifdef MPREF_COUNT
    return 1;
#else
    return 0;
#endif
}

/* scalar EFT primitives (Algorithms 1-3) */
void mpref_two_sum_d(double a, double b, double *s, double *e) { two_sum_d(a, b, s, e); }
void mpref_quick_two_sum_d(double a, double b, double *s, double *e) { quick_two_sum_d(a, b, s, e); }
void mpref_two_prod_d(double a, double b, double *p, double *e) { two_prod_d(a, b, p, e); }
void mpref_two_sum_f(float a, float b, float *s, float *e) { two_sum_f(a, b, s, e); }
void mpref_quick_two_sum_f(float a, float b, float *s, float *e) { quick_two_sum_f(a, b, s, e); }
void mpref_two_prod_f(float a, float b, float *p, float *e) { two_prod_f(a, b, p, e); }

/* elementary functions used for the Aberth starting values (exported for tests) */
void mpref_dk_cos_sin(double th, double *c, double *s) { dk_cos_sin(th, c, s); }
double mpref_dk_nthroot(double v, int64_t m) { return dk_nthroot(v, m); }

#define MPREF_EXPORT_COMMON(S, T, PV)                                                        \
    void mpref_add_##S(int64_t n, const T *a, int64_t pa, const T *b, int64_t pb, T *c,     \
                       int64_t pc)                                                          \
    {                                                                                       \
        MPREF_CAT(ew_add, SFXV)(&PV, n, a, pa, b, pb, c, pc);                                \
    }                                                                                       \
    void mpref_mul_##S(int64_t n, const T *a, int64_t pa, const T *b, int64_t pb, T *c,     \
                       int64_t pc)                                                          \
    {                                                                                       \
        MPREF_CAT(ew_mul, SFXV)(&PV, n, a, pa, b, pb, c, pc);                                \
    }                                                                                       \
    void mpref_recip_##S(int64_t n, const T *a, int64_t pa, T *c, int64_t pc)               \
    {                                                                                       \
        MPREF_CAT(ew_recip, SFXV)(&PV, n, a, pa, c, pc);                                     \
    }                                                                                       \
    void mpref_axpy_##S(int64_t n, const T *alpha, const T *x, int64_t px, T *y, int64_t py) \
    {                                                                                       \
        MPREF_CAT(axpy, SFXV)(&PV, n, alpha, x, px, y, py);                                  \
    }                                                                                       \
    void mpref_dot_##S(int64_t n, const T *x, int64_t px, const T *y, int64_t py, T *s)     \
    {                                                                                       \
        MPREF_CAT(dot, SFXV)(&PV, n, x, px, y, py, s);                                       \
    }                                                                                       \
    void mpref_gemv_##S(int64_t m, int64_t n, const T *A, int64_t lda, int64_t pA,          \
                        const T *x, int64_t px, T *y, int64_t py)                           \
    {                                                                                       \
        MPREF_CAT(gemv, SFXV)(&PV, m, n, A, lda, pA, x, px, y, py);                          \
    }                                                                                       \
    void mpref_gemm_##S(int opA, int opB, int64_t m, int64_t n, int64_t k, const T *A,      \
                        int64_t lda, int64_t pA, const T *B, int64_t ldb, int64_t pB, T *C, \
                        int64_t ldc, int64_t pC)                                            \
    {                                                                                       \
        MPREF_CAT(gemm, SFXV)(&PV, opA, opB, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC);   \
    }                                                                                       \
    void mpref_cgemm_##S(int opA, int opB, int64_t m, int64_t n, int64_t k, const T *Ar,      \
                         const T *Ai, int64_t lda, int64_t pA, const T *Br, const T *Bi,     \
                         int64_t ldb, int64_t pB, T *Cr, T *Ci, int64_t ldc, int64_t pC)     \
    {                                                                                       \
        MPREF_CAT(cgemm3m, SFXV)(&PV, opA, opB, m, n, k, Ar, Ai, lda, pA, Br, Bi, ldb, pB,   \
                                 Cr, Ci, ldc, pC);                                          \
    }                                                                                       \
    void mpref_gemm_strassen_##S(int64_t m, int64_t n, int64_t k, const T *A, int64_t lda,     \
                                 int64_t pA, const T *B, int64_t ldb, int64_t pB, T *C,      \
                                 int64_t ldc, int64_t pC, int64_t cutoff)                    \
    {                                                                                       \
        MPREF_CAT(strassen, SFXV)(&PV, m, n, k, A, lda, pA, B, ldb, pB, C, ldc, pC, cutoff); \
    }                                                                                       \
    void mpref_polyeval_##S(int64_t npoly, const int64_t *coef_off, const T *coef,          \
                            int64_t pcoef, int64_t npts, const T *x_re, const T *x_im,      \
                            int64_t px, T *y_re, T *y_im, int64_t py)                       \
    {                                                                                       \
        MPREF_CAT(polyeval, SFXV)(&PV, npoly, coef_off, coef, pcoef, npts, x_re, x_im, px,   \
                                  y_re, y_im, py);                                          \
    }                                                                                       \
    void mpref_polyeval_estrin_##S(int64_t npoly, const int64_t *coef_off, const T *coef,   \
                                   int64_t pcoef, int64_t npts, const T *x_re, const T *x_im, \
                                   int64_t px, T *y_re, T *y_im, int64_t py)                \
    {                                                                                       \
        MPREF_CAT(polyeval_estrin, SFXV)(&PV, npoly, coef_off, coef, pcoef, npts, x_re, x_im, \
                                         px, y_re, y_im, py);                               \
    }                                                                                       \
    void mpref_polyeval_backward_##S(int64_t npoly, const int64_t *coef_off, const T *coef, \
                                     int64_t pcoef, int64_t npts, const T *x, int64_t px,   \
                                     const T *dy, int64_t pdy, T *dcoef, int64_t pdc,       \
                                     T *dx, int64_t pdx)                                    \
    {                                                                                       \
        MPREF_CAT(polyeval_backward, SFXV)(&PV, npoly, coef_off, coef, pcoef, npts, x, px,   \
                                           dy, pdy, dcoef, pdc, dx, pdx);                   \
    }

#define SFXV _d
MPREF_EXPORT_COMMON(dd, double, P_dd)
MPREF_EXPORT_COMMON(ddc, double, P_ddc)
MPREF_EXPORT_COMMON(td, double, P_td)
MPREF_EXPORT_COMMON(qd, double, P_qd)
MPREF_EXPORT_COMMON(tdc, double, P_tdc)
MPREF_EXPORT_COMMON(qdc, double, P_qdc)
#undef SFXV
#define SFXV _f
MPREF_EXPORT_COMMON(ds, float, P_ds)
MPREF_EXPORT_COMMON(tf, float, P_tf)
MPREF_EXPORT_COMMON(qf, float, P_qf)
#undef SFXV

/* Root solving and the polynomial builder: binary64-component precisions. */
#define MPREF_EXPORT_DK(S, PV)                                                                \
    void mpref_poly_from_roots_##S(int64_t npoly, const int64_t *coef_off,                   \
                                   const double *rootdata, const double *delta, double *coef, \
                                   int64_t pcoef)                                            \
    {                                                                                        \
        poly_from_roots_d(&PV, npoly, coef_off, rootdata, delta, coef, pcoef);               \
    }                                                                                        \
    void mpref_aberth_##S(int64_t n, const double *coef, int64_t pcoef, double *z,           \
                          int64_t pz, double radius)                                         \
    {                                                                                        \
        dk_aberth(&PV, n, coef, pcoef, z, pz, radius);                                       \
    }                                                                                        \
    void mpref_roots_##S(int64_t npoly, const int64_t *coef_off, const double *coef,         \
                         int64_t pcoef, const double *z0, int64_t pz0, double *roots,        \
                         int64_t proots, int32_t *iters, int32_t *status, double tol,        \
                         int32_t max_iter, int32_t stag_window, int32_t stag_min_iter,       \
                         double radius)                                                      \
    {                                                                                        \
        mpref_roots_opts o = {tol, max_iter, stag_window, stag_min_iter, radius};           \
        for (int64_t b = 0; b < npoly; b++) {                                                \
            int64_t n = coef_off[b + 1] - coef_off[b] - 1;                                   \
            int64_t ro = coef_off[b] - b;                                                    \
            dk_solve_one(&PV, n, coef + coef_off[b], pcoef, z0 ? z0 + ro : NULL, pz0,        \
                         roots + ro, proots, &o, iters + b, status + b);                     \
        }                                                                                    \
    }

MPREF_EXPORT_DK(dd, P_dd)
MPREF_EXPORT_DK(ddc, P_ddc)
MPREF_EXPORT_DK(td, P_td)
MPREF_EXPORT_DK(qd, P_qd)
