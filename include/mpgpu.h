/*
 * mpgpu.h -- C ABI of libmpgpu.so: branch-free multicomponent (double-,
 * triple- and quad-word) arithmetic and the linear-algebra, polynomial and
 * root-solving kernels built on it, for NVIDIA GB300 (sm_103a).
 *
 * Method: T. Kouya, "Acceleration of multicomponent multiple-precision
 * arithmetic with branch-free algorithms and SIMD vectorization",
 * arXiv 2603.14926.  Section 2 (Algorithms 1-14) defines the arithmetic,
 * Section 3 the matrix product C := AB (Eq. 1), Section 4.1 polynomial
 * evaluation, Section 4.2 the Durand-Kerner iteration (Eq. 4) and its Aberth
 * starting values (Eq. 5).
 *
 * PRECISIONS.  Every function family exists once per precision suffix P:
 *   dd  : 2 x binary64, add = Algorithm 6 (DWBFAdd),  mul = Algorithm 8 (DWBFMul)
 *   ddc : 2 x binary64, add = Algorithm 4 (DWAdd),    mul = Algorithm 7 (DWMul; its
 *         undefined "QuickTwoProd" read as QuickTwoSum, which makes it Algorithm 8)
 *         -- the conventional double-double the paper benchmarks as "DD"
 *   td  : 3 x binary64, Algorithms 11 (TWBFAdd) and 12 (TWBFMul)
 *   qd  : 4 x binary64, Algorithms 13 (QWBFAdd) and 14 (QDBFMul)
 *   tdc : 3 x binary64, Algorithms 9 (TWAdd) and 10 (TWMul), each ending in
 *         TWRenormalize -- the conventional triple word of Table 4's
 *         standard / BF ratio; Algorithm 10's last TwoSum, printed with q3,
 *         is read with the order-eps^3 sum t0
 *   qdc : 4 x binary64, the QD library's quad-word add (sloppy form) and
 *         multiply (accurate form), each ending in QWRenormalize -- the
 *         conventional quad word (Section 2.3 names these without printing
 *         them; they follow Hida, Li and Bailey, ARITH-15, 2001)
 *   ds  : 2 x binary32, Algorithms 6 and 8
 *   tf  : 3 x binary32, Algorithms 11 and 12
 *   qf  : 4 x binary32, Algorithms 13 and 14
 * T below is double for dd/ddc/td/qd/tdc/qdc and float for ds/tf/qf; K is the
 * number of components.  Root solving and polynomial construction exist for
 * dd/ddc/td/qd only.  tdc and qdc provide the elementwise, AXPY, dot, GEMV,
 * GEMM and Strassen families (their renormalisations branch on zero tests;
 * results are still bit-identical to the CPU oracle).
 *
 * LAYOUT.  A "K-array" of n numbers is K planes of n components each: component
 * c (0 = leading) of element i is at ptr[c * plane_stride + i].  Plane strides
 * are in elements.  A complex K-array has 2K planes: the K real components, then
 * the K imaginary components.  Matrices are row-major inside each plane:
 * element (i, j) of a matrix with leading dimension ld is at [c*ps + i*ld + j].
 *
 * OWNERSHIP AND STREAMS.  All array arguments are device pointers owned by the
 * caller, unless marked "host".  The library allocates no memory: where a kernel
 * needs scratch space the caller passes a device workspace of the size the
 * matching *_workspace_P() function returns.  Every call is asynchronous on the
 * given stream (a cudaStream_t; NULL = the legacy default stream) and returns
 * after enqueuing its kernels, except where a function says it synchronizes.
 *
 * ERRORS.  Invalid arguments (negative sizes, NULL required pointers, strides
 * too small for the sizes, workspace too small, unsupported options) return
 * MP_EINVAL before anything is enqueued.  A failed launch returns MP_ECUDA
 * (mp_last_cuda_error() gives the CUDA error code).  Values are IEEE: there is
 * no error for overflow or NaN inputs, whose results are unspecified but never
 * fault or hang.  n = 0 (or m, n or k = 0) is valid and does nothing except
 * where stated (a dot of length 0 writes 0; C := A B with k = 0 writes zeros).
 */
#ifndef MPGPU_H
#define MPGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MP_OK = 0,
    MP_EINVAL = 1,   /* invalid argument; nothing enqueued */
    MP_ECUDA = 2,    /* CUDA launch or runtime error */
    MP_ENOMEM = 3,   /* workspace too small */
    MP_ETIMEOUT = 4, /* reserved for host-visible watchdog expiry */
    MP_ENOTSUP = 5   /* option not supported for this precision */
} mp_status;

typedef void *mp_stream; /* cudaStream_t */

const char *mp_status_str(mp_status s);
int mp_last_cuda_error(void);
const char *mp_version(void);

/* ------------------------------------------------------------------------ */
/* Elementwise: c_i := a_i + b_i (mp_add_P), a_i * b_i (mp_mul_P),          */
/* 1 / a_i (mp_recip_P).  Section 2: Algorithms 4-14 per precision above;  */
/* the reciprocal is Newton's method (Section 2 names it without details):  */
/* y0 = 1/a[0] in T, then s times e = 1 - a*y, y = y + y*e, s = 2 for K <= 3 */
/* and 3 for K = 4.  Bit-identical to the CPU oracle.  c may alias a or b.   */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_EW(P, T)                                                                 \
    mp_status mp_add_##P(int64_t n, const T *a, int64_t pa, const T *b, int64_t pb, T *c,   \
                         int64_t pc, mp_stream stream);                                     \
    mp_status mp_mul_##P(int64_t n, const T *a, int64_t pa, const T *b, int64_t pb, T *c,   \
                         int64_t pc, mp_stream stream);                                     \
    mp_status mp_recip_##P(int64_t n, const T *a, int64_t pa, T *c, int64_t pc,             \
                           mp_stream stream);

/* ------------------------------------------------------------------------ */
/* AXPY  y_i := alpha * x_i + y_i, evaluated add(mul(alpha, x_i), y_i)      */
/* (basic linear computations, Section 1).  alpha: HOST array of K values.  */
/* Bit-identical to the CPU oracle.                                         */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_AXPY(P, T)                                                               \
    mp_status mp_axpy_##P(int64_t n, const T *alpha, const T *x, int64_t px, T *y,          \
                          int64_t py, mp_stream stream);

/* ------------------------------------------------------------------------ */
/* DOT  result := sum_i x_i * y_i (K values written at result[0..K-1]).     */
/* Each thread folds a strided subsequence with add(acc, mul(x_i, y_i)),    */
/* partial sums are combined by warp shuffles and a block tree using the    */
/* multicomponent add itself, then one block combines the block partials in */
/* a fixed order (one full wave of SMs x resident blocks): deterministic on */
/* a given GPU model, but not the oracle's sequential order --              */
/* it agrees with the exact sum within (4n+16) 2^-p sum |x_i y_i|, p = K*53 */
/* (binary64) or K*24 (binary32).  ws: device workspace of at least         */
/* mp_dot_workspace_P(n) bytes (MP_ENOMEM if smaller); it holds the block   */
/* partials and need not be initialised.                                    */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_DOT(P, T)                                                                \
    size_t mp_dot_workspace_##P(int64_t n);                                                 \
    mp_status mp_dot_##P(int64_t n, const T *x, int64_t px, const T *y, int64_t py,         \
                         T *result, void *ws, size_t ws_bytes, mp_stream stream);

/* ------------------------------------------------------------------------ */
/* GEMV  y := A x, A m x n row-major (leading dimension lda >= n, plane     */
/* stride pA).  Each row is folded by T threads (T in 32..256, chosen from  */
/* m, n and the SM count): thread t folds columns t, t+T, ..., a warp       */
/* shuffle tree and then the row's warps in order combine the partials     */
/* with the multicomponent add; deterministic on a given GPU model, within */
/* the dot bound above of the exact result.  y must not alias A or x.      */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_GEMV(P, T)                                                               \
    mp_status mp_gemv_##P(int64_t m, int64_t n, const T *A, int64_t lda, int64_t pA,        \
                          const T *x, int64_t px, T *y, int64_t py, mp_stream stream);

/* ------------------------------------------------------------------------ */
/* GEMM  C := op(A) op(B)  (Section 3.1, Eq. 1: C := AB), op(X) = X for op 0 */
/* and X^T for op 1 (op 1 serves the adjoint dA = dC B^T, dB = A^T dC).     */
/* op(A) is m x k, op(B) is k x n, C is m x n, all row-major in their own   */
/* storage: A is m x k (lda >= k) for opA = 0 and k x m (lda >= m) for      */
/* opA = 1, likewise B.  Every c_ij is the sequential fold over l = 0..k-1  */
/* of add(c, mul(a_il, b_lj)) starting at c = 0 (the naive triple loop), so */
/* the result is bit-identical to the CPU oracle.  C must not alias A or B. */
/* mp_gemm_ex_P selects a tile configuration (0 .. mp_gemm_num_configs_P()-1,*/
/* or -1 for the built-in choice); configurations differ only in speed.     */
/* Configurations 4, 5, 6, 8 and 9 stage the tiles with TMA (cp.async.bulk. */
/* tensor, double buffered on mbarriers) when the operands meet TMA's       */
/* alignment rules (16-byte aligned base, lda/ldb and plane strides         */
/* multiples of 16 bytes) and otherwise run the same tile with plain loads. */
/* For binary64 components configurations 5-9 use the hybrid engine: each   */
/* TwoSum (Algorithm 2) takes s from the FP64 pipe and its error term from  */
/* an exact integer computation (configuration 6 likewise QuickTwoSum where */
/* Algorithm 1 is exact, configuration 9 likewise TwoProd's error term,     */
/* Algorithm 3).  The bits are the FP64 sequence's; a thread                */
/* whose operands leave the integer path's domain (exponents near the       */
/* binary64 limits, subnormal error terms, an inexact QuickTwoSum)          */
/* recomputes its outputs with the FP64 pipe.  The built-in choice (-1) is  */
/* configuration 5 for binary64 components, 0 for binary32.                 */
/* mp_gemm_tma_timeouts_P SYNCHRONIZES and reports how many TMA waits ever  */
/* ran out (always 0 unless the copy path failed; the kernel then returns   */
/* early instead of hanging).  mp_gemm_hybrid_fallbacks_P SYNCHRONIZES and  */
/* reports how many threads have taken the FP64 recomputation since the    */
/* library was loaded (counted across all GEMM calls of precision P).       */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_GEMM(P, T)                                                               \
    mp_status mp_gemm_##P(int opA, int opB, int64_t m, int64_t n, int64_t k, const T *A,    \
                          int64_t lda, int64_t pA, const T *B, int64_t ldb, int64_t pB,     \
                          T *C, int64_t ldc, int64_t pC, mp_stream stream);                 \
    mp_status mp_gemm_ex_##P(int opA, int opB, int64_t m, int64_t n, int64_t k, const T *A, \
                             int64_t lda, int64_t pA, const T *B, int64_t ldb, int64_t pB,  \
                             T *C, int64_t ldc, int64_t pC, int config, mp_stream stream);  \
    int mp_gemm_num_configs_##P(void);                                                      \
    mp_status mp_gemm_tma_timeouts_##P(unsigned int *count);                                \
    mp_status mp_gemm_hybrid_fallbacks_##P(unsigned int *count);                            \
    const char *mp_gemm_config_name_##P(int config);

/* ------------------------------------------------------------------------ */
/* CGEMM  complex C := op(A) op(B) by the 3M method (Section 3.2, Eq. 3):     */
/*   C1 = Re A Re B, C2 = Im A Im B, Re C = C1 - C2,                          */
/*   Im C = (Re A + Im A)(Re B + Im B) - C1 - C2 (subtracted left to right), */
/* three mp_gemm_ex_P products plus elementwise sums and differences; the    */
/* operand sums are formed in the operands' own storage layout.  Real and    */
/* imaginary parts are separate K-arrays sharing lda/pA (A), ldb/pB (B),     */
/* ldc/pC (C); layouts and op as for GEMM.  Bit-identical to the CPU oracle. */
/* ws: DEVICE workspace of mp_cgemm_workspace_P(m, n, pA, pB) bytes (the two */
/* operand sums and C2; no initialisation needed).  Cr, Ci must not alias   */
/* the inputs.                                                              */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_CGEMM(P, T)                                                              \
    size_t mp_cgemm_workspace_##P(int64_t m, int64_t n, int64_t pA, int64_t pB);            \
    mp_status mp_cgemm_##P(int opA, int opB, int64_t m, int64_t n, int64_t k, const T *Ar,  \
                           const T *Ai, int64_t lda, int64_t pA, const T *Br, const T *Bi,  \
                           int64_t ldb, int64_t pB, T *Cr, T *Ci, int64_t ldc, int64_t pC,  \
                           void *ws, size_t ws_bytes, mp_stream stream);

/* ------------------------------------------------------------------------ */
/* GEMM_STRASSEN  real C := A B by Strassen's recursion, the matrix         */
/* multiplication scheme of Section 3.1 (the paper recurses until the       */
/* submatrices drop below 32 x 32), with Strassen's seven products:         */
/*   M1 = (A11+A22)(B11+B22)  M2 = (A21+A22)B11  M3 = A11(B12-B22)          */
/*   M4 = A22(B21-B11)  M5 = (A11+A12)B22  M6 = (A21-A11)(B11+B12)           */
/*   M7 = (A12-A22)(B21+B22)                                                */
/*   C11 = ((M1+M4)-M5)+M7  C12 = M3+M5  C21 = M2+M4  C22 = ((M1-M2)+M3)+M6 */
/* A node with min(m, n, k) < cutoff is one classical GEMM (mp_gemm_ex_P,   */
/* sequential k).  Otherwise quadrants are ceil(m/2) x ceil(k/2) (A) and     */
/* ceil(k/2) x ceil(n/2) (B) blocks, zero-padded where a dimension is odd;  */
/* sums and differences are elementwise multicomponent adds (a difference    */
/* adds the negated operand), a padded entry taking part as +0; C keeps the */
/* unpadded part.  Bit-identical to the CPU oracle for the same cutoff.     */
/* No transposes: A is m x k (lda, pA), B is k x n (ldb, pB), row-major     */
/* K-arrays as for GEMM.  cutoff >= 2 (else MP_EINVAL).                      */
/* ws: DEVICE workspace of mp_gemm_strassen_workspace_P(m, n, k, cutoff)     */
/* bytes (three buffers per recursion level; 0 when no level recurses; no   */
/* initialisation needed); MP_ENOMEM if smaller.  C must not overlap A, B.   */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_STRASSEN(P, T)                                                           \
    size_t mp_gemm_strassen_workspace_##P(int64_t m, int64_t n, int64_t k, int64_t cutoff); \
    mp_status mp_gemm_strassen_##P(int64_t m, int64_t n, int64_t k, const T *A, int64_t lda, \
                                   int64_t pA, const T *B, int64_t ldb, int64_t pB, T *C,   \
                                   int64_t ldc, int64_t pC, int64_t cutoff, void *ws,       \
                                   size_t ws_bytes, mp_stream stream);

/* ------------------------------------------------------------------------ */
/* POLYEVAL  (Section 4.1) batched Horner evaluation of real-coefficient    */
/* polynomials p_b(x) = sum_{i=0}^{n_b} a_{b,i} x^i.                        */
/*   coef_off : DEVICE int64[npoly+1]; polynomial b owns coefficients        */
/*              coef_off[b] .. coef_off[b+1]-1 (a_0 first), n_b = count - 1  */
/*   x_re/x_im: points b*npts .. b*npts+npts-1 belong to polynomial b;      */
/*              x_im == NULL selects real arguments (y_im is then unused)    */
/* Real: h = a_n; h = add(mul(h, x), a_i).  Complex (four real products):   */
/*   re' = add(add(mul(hr,xr), neg(mul(hi,xi))), a_i),                      */
/*   im' = add(mul(hr,xi), mul(hi,xr)).  Bit-identical to the CPU oracle.   */
/* mp_polyeval_estrin_P: the same evaluation by Estrin's scheme (Section    */
/* 4.1 compares it with Horner's; the standard pairwise tree): level 0 holds */
/* a_0..a_n; each level replaces adjacent pairs (lo, hi) by                   */
/* add(mul(hi, y_k), lo), y_0 = x, y_{k+1} = mul(y_k, y_k); an unpaired last */
/* value moves up unchanged.  Complex arguments: every value complex, the    */
/* products in Horner's 4M order, re = add(sub(mul(hr,yr), mul(hi,yi)), lo), */
/* im = add(add(mul(hr,yi), mul(hi,yr)), lo_im).  Same arguments as          */
/* mp_polyeval_P; bit-identical to the CPU oracle.  Degrees up to 2^25 - 1;   */
/* a polynomial above that evaluates to NaN.                                 */
/* ------------------------------------------------------------------------ */
#define MPGPU_DECL_POLY(P, T)                                                               \
    mp_status mp_polyeval_##P(int64_t npoly, const int64_t *coef_off, const T *coef,         \
                              int64_t pcoef, int64_t npts, const T *x_re, const T *x_im,     \
                              int64_t px, T *y_re, T *y_im, int64_t py, mp_stream stream);   \
    mp_status mp_polyeval_estrin_##P(int64_t npoly, const int64_t *coef_off, const T *coef,  \
                                     int64_t pcoef, int64_t npts, const T *x_re,             \
                                     const T *x_im, int64_t px, T *y_re, T *y_im, int64_t py,\
                                     mp_stream stream);                                      \
    size_t mp_polyeval_backward_workspace_##P(int64_t npoly, int64_t npts);                 \
    mp_status mp_polyeval_backward_##P(int64_t npoly, const int64_t *coef_off, const T *coef,\
                                       int64_t pcoef, int64_t npts, const T *x, int64_t px,  \
                                       const T *dy, int64_t pdy, T *dcoef, int64_t pdc,      \
                                       T *dx, int64_t pdx, void *ws, size_t ws_bytes,        \
                                       mp_stream stream);

/* POLYEVAL_BACKWARD: adjoint of the real-argument evaluation for a given dy:   */
/*   dx_{b,m}    = mul(dy_{b,m}, p_b'(x_{b,m})), p' by the simultaneous Horner   */
/*                 recurrence d = add(mul(d,x), h); h = add(mul(h,x), a_i);      */
/*   dcoef_{b,i} = sum over m ascending of w_{b,m,i} (fold from 0 with add),     */
/*                 w_0 = dy, w_{i+1} = mul(w_i, x): the reverse sweep of Horner's*/
/*                 recurrence h_i = h_{i+1} x + a_i.                             */
/* Both are bit-identical to the CPU oracle.  Either output may be NULL.        */
/* ws, ws_bytes: unused (may be NULL, 0); mp_polyeval_backward_workspace_P     */
/* answers 0.  The coefficient sweep keeps its partial sums in dcoef itself, so */
/* dcoef's contents are undefined while the call runs.                          */

/* ------------------------------------------------------------------------ */
/* POLY_FROM_ROOTS: coefficients of prod (x - r) (the root-solving workload): */
/* per polynomial, rootdata holds floor(n/2) complex roots as (re, im)      */
/* pairs (conjugates implied) then one real root if n is odd; delta holds n */
/* relative perturbations.  Real factor first: p'_i = add(p_{i-1},          */
/* neg(mul(r, p_i))); each pair: x^2 + B x + C, B = -2 re, C = add(mul(re,re),*/
/* mul(im,im)), p'_i = add(add(p_{i-2}, mul(B, p_{i-1})), mul(C, p_i));     */
/* finally a_i = mul(a_i, (1, delta_i)) for i < n.  rootdata/delta are      */
/* indexed from coef_off[b] - b.  max_degree: host bound on every degree   */
/* (polynomials above it are left unwritten).  Bit-identical to the oracle. */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* ROOTS  Durand-Kerner (Section 4.2, Eq. 4) on every polynomial, complex   */
/* K-component iterates, Jacobi sweeps, batched.  For each root i:           */
/*   w_i = q(z_i) / prod_{j != i} (z_i - z_j),  z_i' = z_i - w_i,            */
/* q = p / a_n (monic; skipped when a_n == 1 exactly), q(z) by complex      */
/* Horner, the product over j ascending from 1, the quotient by cdiv (a *   */
/* conj b * recip(|b|^2)).  q(z_i) and the product carry an explicit power- */
/* of-two exponent (rescaled by exact powers of two when a leading component*/
/* reaches 2^257 or, for the product, falls below 2^-256), which is bit-    */
/* identical to plain evaluation whenever that stays in binary64's range.   */
/* Start (Eq. 5): z_i = -c_{n-1}/n + r e^{i((2(i-1)pi)/n + 3/(2n))} with    */
/* r = max |n_nz c_i|^(1/(n-i)), in binary64, by fixed operation sequences  */
/* (no libm), or r = opts->radius when > 0, or z0 when non-NULL.            */
/* Stop: delta = max_i(|Re w_i|+|Im w_i|) on leading components, zmax =      */
/* max_i(|Re z_i'|+|Im z_i'|); status 1 (converged) when delta <= tol *     */
/* max(1,zmax); 2 (stagnated) when from iteration stag_min_iter on, delta   */
/* has not reached a new minimum for stag_window sweeps and that minimum is */
/* <= 2^-(26K) max(1,zmax); 4 (breakdown) on a non-finite delta or zmax; 0  */
/* when max_iter sweeps ran; 3 when the device watchdog (watchdog_cycles > 0,*/
/* a clock64 budget per polynomial) stopped it.  Results, iteration counts  */
/* and statuses are bit-identical to the CPU oracle and identical between   */
/* the persistent batched launch (mode 0), one launch per polynomial        */
/* (mode 1) and the cluster solve (mode 2: one thread-block cluster of      */
/* C <= 8 CTAs per polynomial, each CTA owning ceil(n/C) roots: up to       */
/* max_degree 128, C = max(2, ceil(max_degree/16)) and every complex step   */
/* split over a lane quad, above it C = ceil(max_degree/32) and a lane      */
/* pair; the new iterate exchanged through distributed shared memory once   */
/* per sweep; for                                                           */
/* the latency of few polynomials; max_degree <= 256 and sort = 0, else     */
/* MP_EINVAL), and between the engines: the hybrid engine (opts->engine 0 = */
/* automatic, or 1) runs each root's update with TwoSum error terms on the  */
/* integer pipes (see GEMM), the multicomponent add and multiply called out */
/* of line; a root whose integer path leaves its domain is recomputed on the*/
/* FP64 pipe.  opts->engine 2 keeps every step on the FP64 pipe.            */
/*   roots  : complex K-array, root j of polynomial b at index              */
/*            coef_off[b] - b + j, plane stride proots                       */
/*   z0     : NULL or starting values in the same layout (plane stride pz0)  */
/*   iters, status : DEVICE int32[npoly]                                     */
/*   ws     : DEVICE workspace of mp_roots_workspace_deg_P(npoly,            */
/*            opts->max_degree) bytes, 8-byte aligned (its first word is the */
/*            64-bit work-queue counter; no initialisation needed).  Up to   */
/*            mp_roots_max_degree_P() (the shared-memory bound: QD 2421, TD  */
/*            3228, DD 4843) this equals mp_roots_workspace_P(npoly); above  */
/*            it each block keeps its coefficients and iterate in a slot of  */
/*            the workspace (4 slots per SM, at most 3 K (max_degree + 1)    */
/*            doubles each; the persistent grid is then capped at 4 blocks  */
/*            per SM), same results, and modes 0 and 1 only.                 */
/*   opts->max_degree : host upper bound of the degrees (> 0 required; the   */
/*            kernel skips, with status 4, any polynomial above it); at most */
/*            2^20                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    double tol;              /* <= 0: 2^-(53K - 6) */
    int32_t max_iter;        /* <= 0: 1000 */
    int32_t stag_window;     /* <= 0: 5 */
    int32_t stag_min_iter;   /* <= 0: 10 */
    int32_t mode;            /* 0: persistent batched launch, 1: one launch per polynomial,
                                2: cluster solve (one thread-block cluster of 2-8 CTAs per
                                polynomial, for latency; max_degree <= 256, sort = 0) */
    double radius;           /* > 0: start circle radius instead of Eq. 5's */
    int64_t watchdog_cycles; /* > 0: per-polynomial clock64 budget, status 3 when spent */
    int32_t max_degree;      /* host bound on every degree, required */
    int32_t threads;         /* threads per block: 0 = automatic (hybrid: the smallest multiple of 64 that is
                                >= 2 * max_degree, at most 256; engine 2: 128); else a multiple of 32, <= 256 */
    int32_t blocks_per_sm;   /* persistent grid = SMs * blocks_per_sm, 0 = automatic */
    int32_t sort;            /* 1: process polynomials in descending degree (default 0 = off) */
    int32_t engine;          /* 0: automatic (hybrid), 1: hybrid, 2: FP64 pipe throughout; same bits */
} mp_roots_opts;

#define MPGPU_DECL_ROOTS(P)                                                                 \
    mp_status mp_poly_from_roots_##P(int64_t npoly, const int64_t *coef_off,                \
                                     const double *rootdata, const double *delta,            \
                                     int32_t max_degree, double *coef, int64_t pcoef,        \
                                     mp_stream stream);                                      \
    mp_status mp_roots_init_##P(int64_t npoly, const int64_t *coef_off, const double *coef,  \
                                int64_t pcoef, double radius, int32_t max_degree, double *z, \
                                int64_t pz, mp_stream stream);                               \
    size_t mp_roots_workspace_##P(int64_t npoly);                                           \
    size_t mp_roots_workspace_deg_##P(int64_t npoly, int32_t max_degree);                   \
    int32_t mp_roots_max_degree_##P(void);                                                  \
    mp_status mp_roots_##P(int64_t npoly, const int64_t *coef_off, const double *coef,       \
                           int64_t pcoef, const double *z0, int64_t pz0, double *roots,      \
                           int64_t proots, int32_t *iters, int32_t *status,                  \
                           const mp_roots_opts *opts, void *ws, size_t ws_bytes,             \
                           mp_stream stream);

/* mp_roots_hybrid_fallbacks: how many root updates, over all precisions and  */
/* calls since the library was loaded, left the hybrid engine's domain and    */
/* were recomputed on the FP64 pipe (same bits either way).  SYNCHRONIZES.   */
mp_status mp_roots_hybrid_fallbacks(unsigned long long *count);

/* mp_roots_init_P writes the Eq. 5 starting values (or radius-r circle) that */
/* mp_roots_P uses when z0 == NULL, as a complex K-array (lower components 0); */
/* max_degree <= mp_roots_max_degree_P() (its kernel works in shared memory),  */
/* else MP_EINVAL.                                                             */

#define MPGPU_DECL_ALL(P, T)                                                                \
    MPGPU_DECL_EW(P, T)                                                                     \
    MPGPU_DECL_AXPY(P, T)                                                                   \
    MPGPU_DECL_DOT(P, T)                                                                    \
    MPGPU_DECL_GEMV(P, T)                                                                   \
    MPGPU_DECL_GEMM(P, T)                                                                   \
    MPGPU_DECL_CGEMM(P, T)                                                                  \
    MPGPU_DECL_STRASSEN(P, T)                                                               \
    MPGPU_DECL_POLY(P, T)

MPGPU_DECL_ALL(dd, double)
MPGPU_DECL_ALL(ddc, double)
MPGPU_DECL_ALL(td, double)
MPGPU_DECL_ALL(qd, double)
#define MPGPU_DECL_CONVENTIONAL(P, T)                                                       \
    MPGPU_DECL_EW(P, T)                                                                     \
    MPGPU_DECL_AXPY(P, T)                                                                   \
    MPGPU_DECL_DOT(P, T)                                                                    \
    MPGPU_DECL_GEMV(P, T)                                                                   \
    MPGPU_DECL_GEMM(P, T)                                                                   \
    MPGPU_DECL_STRASSEN(P, T)
MPGPU_DECL_CONVENTIONAL(tdc, double)
MPGPU_DECL_CONVENTIONAL(qdc, double)
MPGPU_DECL_ALL(ds, float)
MPGPU_DECL_ALL(tf, float)
MPGPU_DECL_ALL(qf, float)
MPGPU_DECL_ROOTS(dd)
MPGPU_DECL_ROOTS(ddc)
MPGPU_DECL_ROOTS(td)
MPGPU_DECL_ROOTS(qd)

/* ------------------------------------------------------------------------ */
/* mp_roots_noalloc_qd: the QD batched root solver (mp_roots_qd) without a    */
/* caller workspace, for code that cannot allocate device memory (a fixed     */
/* memory pool that must not grow, a plugin whose allocator belongs to its    */
/* host, a real-time loop where an allocation could stall).  The paper has no */
/* counterpart; this is a library convenience.  Same arguments and same       */
/* results (bit for bit) as mp_roots_qd without ws/ws_bytes.  Its workspace   */
/* (queue counter and degree order) is a fixed 64.25 KiB device array inside  */
/* the library, held by every GPU that loads the library until the process    */
/* exits, so it takes npoly <= MP_NOALLOC_MAX_POLYS (16384) and              */
/* opts->max_degree <= mp_roots_max_degree_qd() (no per-block slots); larger  */
/* requests return MP_ENOMEM before anything is enqueued.  The first call on  */
/* a device looks the array up (cudaGetSymbolAddress) for that device, so     */
/* make it before any stream capture.  Concurrent calls from host threads are */
/* safe on the host side (the lookup is guarded), but calls share the array: */
/* calls whose kernels overlap on the GPU race on it.  The solve clears the   */
/* queue counter itself; nothing else needs initialisation.  After            */
/* cudaDeviceReset on a device, do not call it on that device again (the      */
/* looked-up address is kept).                                                */
/* ------------------------------------------------------------------------ */
#define MP_NOALLOC_MAX_POLYS (1 << 14)
mp_status mp_roots_noalloc_qd(int64_t npoly, const int64_t *coef_off, const double *coef, int64_t pcoef,
                              const double *z0, int64_t pz0, double *roots, int64_t proots, int32_t *iters,
                              int32_t *status, const mp_roots_opts *opts, mp_stream stream);

/* ------------------------------------------------------------------------ */
/* Pipe-peak microbenchmark (measurement support, not part of the method):   */
/* `blocks` x `threads` threads each run `iters` iterations of 8 independent */
/* dependency chains of one instruction kind: 0 = DFMA, 1 = DADD, 2 = DMUL,  */
/* 3 = FFMA, 4 = FADD, 5 = packed fma.rn.f32x2, 6 = packed add.rn.f32x2,     */
/* 7 = LOP3 (integer ALU pipe), 8 = IMAD (integer on the FMA pipe),          */
/* 9 = IADD3 and LOP3 alternating, 10 = FLO + IADD3 (count leading zeros),   */
/* 11 = DFMA with one active lane per warp.                                   */
/* SYNCHRONIZES the stream; *ms receives the elapsed time between CUDA      */
/* events recorded on it and *lane_ops the number of per-lane operations     */
/* executed (blocks * threads * iters * 8, doubled for kinds 5, 6 and 10;    */
/* for kind 11 one lane per warp).                                           */
/* ------------------------------------------------------------------------ */
mp_status mp_peak_run(int kind, int64_t iters, int blocks, int threads, float *ms,
                      double *lane_ops, mp_stream stream);
int mp_sm_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MPGPU_H */
