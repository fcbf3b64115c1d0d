// mp_arith.cuh -- branch-free multicomponent arithmetic on the CUDA cores.
//
// Device restatement of Kouya, arXiv 2603.14926, Section 2:
//   Algorithms 1-3  (QuickTwoSum, TwoSum, FMA TwoProd)
//   Algorithms 4, 6 (DWAdd sloppy, DWBFAdd), 7, 8 (DWMul, DWBFMul)
//   Algorithms 11, 12 (TWBFAdd, TWBFMul), 13, 14 (QWBFAdd, QDBFMul)
//   Algorithms 9, 10 (TWAdd, TWMul) and the QD library's quad-word add and
//   multiply, with their renormalisations (the conventional baseline)
// on binary64 (FP64 pipe) or binary32 (FP32 pipe) components.
//
// Every floating-point step is an explicit round-to-nearest-even intrinsic
// (__dadd_rn/__dsub_rn/__dmul_rn/__fma_rn and the binary32 forms), so the
// compiler can neither contract a*b+c nor reassociate: each algorithm runs as
// exactly the operation sequence the paper prints.  Negation and the "-p" of
// TwoProd's FMA are sign-operand modifiers, not instructions.  Tensor cores
// are not used: an FP64 DMMA returns no rounding error, which every step here
// needs.
#pragma once
#include <cstdint>
#include <type_traits>

#include "mp_eft_int.cuh"

namespace mp {

template <typename T> struct fpu;

template <> struct fpu<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

template <> struct fpu<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};

// ---------------------------------------------------------------------------
// Algorithms 1-3
// ---------------------------------------------------------------------------

// Algorithm 1: s = a + b, e = b - (s - a); exact when |a| >= |b|.
template <typename T>
__device__ __forceinline__ void quick_two_sum(T a, T b, T &s, T &e)
{
    using F = fpu<T>;
    T s_ = F::add(a, b);
    e = F::sub(b, F::sub(s_, a));
    s = s_;
}

// Algorithm 2: s = a + b, v = s - a, e = (a - (s - v)) + (b - v); exact.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e)
{
    using F = fpu<T>;
    T s_ = F::add(a, b);
    T v = F::sub(s_, a);
    e = F::add(F::sub(a, F::sub(s_, v)), F::sub(b, v));
    s = s_;
}

// Algorithm 3: p = a * b, e = FMA(a, b, -p); exact.
template <typename T>
__device__ __forceinline__ void two_prod(T a, T b, T &p, T &e)
{
    using F = fpu<T>;
    T p_ = F::mul(a, b);
    e = F::fma(a, b, -p_);
    p = p_;
}

// ---------------------------------------------------------------------------
// Engines.  The multicomponent algorithms below are written once against an
// engine that supplies Algorithms 1-3 and the plain add and multiply; the
// engine decides which pipe executes them.
//
// NativeEngine<T>: every step on the FP64 (or FP32) pipe, as printed.
// HybridEngine<QTS>: binary64 only.  TwoSum's s from one FP64 add, its error e
//   from the integer pipes (mp_eft_int.cuh); with QTS also QuickTwoSum's error
//   where Algorithm 1 is exact (exponent(a) >= exponent(b), or a zero operand);
//   with TP also TwoProd's error (p from one FP64 multiply, the error term from
//   the low 64 bits of the integer significand product); with SUB also a
//   subnormal TwoSum error term.  The plain operations
//   stay on the FP64 pipe.  Outside the
//   integer path's domain, and for QuickTwoSum outside its exact case, the
//   engine raises failed(); callers then recompute the result with
//   NativeEngine, so every output is the FP64 sequence's bits.
// ---------------------------------------------------------------------------

template <typename T> struct NativeEngine {
    __device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) { mp::two_sum(a, b, s, e); }
    __device__ __forceinline__ void quick_two_sum(T a, T b, T &s, T &e) { mp::quick_two_sum(a, b, s, e); }
    __device__ __forceinline__ void two_prod(T a, T b, T &p, T &e) { mp::two_prod(a, b, p, e); }
    __device__ __forceinline__ T add(T a, T b) { return fpu<T>::add(a, b); }
    __device__ __forceinline__ T mul(T a, T b) { return fpu<T>::mul(a, b); }
    __device__ __forceinline__ bool failed() const { return false; }
    __device__ __forceinline__ uint32_t bad_flags() const { return 0; }
    __device__ __forceinline__ void set_bad_flags(uint32_t) {}
};

template <bool QTS, bool TP = false, bool SUB = false> struct HybridEngine {
    uint32_t bad = 0;
    __device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
    {
        const double s_ = __dadd_rn(a, b);
        e = __longlong_as_double((long long)eft_int::two_sum_err<SUB>((uint64_t)__double_as_longlong(a),
                                                                       (uint64_t)__double_as_longlong(b),
                                                                       (uint64_t)__double_as_longlong(s_), bad));
        s = s_;
    }
    __device__ __forceinline__ void quick_two_sum(double a, double b, double &s, double &e)
    {
        if (!QTS) {
            mp::quick_two_sum(a, b, s, e);
            return;
        }
        const double s_ = __dadd_rn(a, b);
        const uint64_t A = (uint64_t)__double_as_longlong(a), B = (uint64_t)__double_as_longlong(b);
        const uint64_t Aa = A & 0x7FFFFFFFFFFFFFFFull, Ba = B & 0x7FFFFFFFFFFFFFFFull;
        // Algorithm 1 is exact when exponent(a) >= exponent(b) or a = 0; with b = 0 its e is b itself
        bad |= (uint32_t)!(Aa >= (Ba & 0x7FF0000000000000ull) || Aa == 0 || Ba == 0);
        const uint64_t E = eft_int::two_sum_err(A, B, (uint64_t)__double_as_longlong(s_), bad);
        e = __longlong_as_double((long long)(Ba == 0 ? B : E));
        s = s_;
    }
    __device__ __forceinline__ void two_prod(double a, double b, double &p, double &e)
    {
        if (!TP) {
            mp::two_prod(a, b, p, e);
            return;
        }
        const double p_ = __dmul_rn(a, b);
        e = __longlong_as_double((long long)eft_int::two_prod_err((uint64_t)__double_as_longlong(a),
                                                                   (uint64_t)__double_as_longlong(b),
                                                                   (uint64_t)__double_as_longlong(p_), bad));
        p = p_;
    }
    __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ bool failed() const { return bad != 0; }
    __device__ __forceinline__ uint32_t bad_flags() const { return bad; }
    __device__ __forceinline__ void set_bad_flags(uint32_t v) { bad = v; }
};

// A K-component number, component 0 leading.  Always held in registers.
template <typename T, int K> struct mpv {
    T c[K];
};

// ---------------------------------------------------------------------------
// Double word
// ---------------------------------------------------------------------------

// Algorithm 4 (DWAdd, the sloppy add of the QD library)
template <typename T, class E>
__device__ __forceinline__ mpv<T, 2> dw_add_sloppy(const mpv<T, 2> &a, const mpv<T, 2> &b, E &g)
{
    T s, e;
    g.two_sum(a.c[0], b.c[0], s, e);
    e = g.add(e, g.add(a.c[1], b.c[1]));
    mpv<T, 2> r;
    g.quick_two_sum(s, e, r.c[0], r.c[1]);
    return r;
}

// Algorithm 6 (DWBFAdd)
template <typename T, class E>
__device__ __forceinline__ mpv<T, 2> dw_add_bf(const mpv<T, 2> &a, const mpv<T, 2> &b, E &g)
{
    T g1, g1e, g2, g2e, g3, g3e;
    g.two_sum(a.c[0], b.c[0], g1, g1e);
    g.two_sum(a.c[1], b.c[1], g2, g2e);
    g.quick_two_sum(g1, g2, g3, g3e);
    T g4 = g.add(g1e, g2e);
    T g5 = g.add(g4, g3e);
    mpv<T, 2> r;
    g.quick_two_sum(g3, g5, r.c[0], r.c[1]);
    return r;
}

// Algorithm 7 (DWMul; its undefined "QuickTwoProd" read as QuickTwoSum) and
// Algorithm 8 (DWBFMul) are the same operation sequence:
// (p00, pe00) = TwoProd(a0, b0); g1 = a0*b1 + a1*b0; g2 = pe00 + g1; QuickTwoSum(p00, g2).
template <typename T, class E>
__device__ __forceinline__ mpv<T, 2> dw_mul_bf(const mpv<T, 2> &a, const mpv<T, 2> &b, E &g)
{
    T p00, pe00;
    g.two_prod(a.c[0], b.c[0], p00, pe00);
    T p01 = g.mul(a.c[0], b.c[1]);
    T p10 = g.mul(a.c[1], b.c[0]);
    T g1 = g.add(p01, p10);
    T g2 = g.add(pe00, g1);
    mpv<T, 2> r;
    g.quick_two_sum(p00, g2, r.c[0], r.c[1]);
    return r;
}

// ---------------------------------------------------------------------------
// Triple word
// ---------------------------------------------------------------------------

// Algorithm 11 (TWBFAdd)
template <typename T, class E>
__device__ __forceinline__ mpv<T, 3> tw_add_bf(const mpv<T, 3> &A, const mpv<T, 3> &B, E &g)
{
    T a1, b1, c1, d1, e1, f1, a2, c2, d2, e2, a3, d3, b3, c3, c5, d5, b6, c6, b7;
    mpv<T, 3> r;
    g.two_sum(A.c[0], B.c[0], a1, b1);
    g.two_sum(A.c[1], B.c[1], c1, d1);
    g.two_sum(A.c[2], B.c[2], e1, f1);
    g.quick_two_sum(a1, c1, a2, c2);
    T b2 = g.add(b1, f1);
    g.two_sum(d1, e1, d2, e2);
    g.quick_two_sum(a2, d2, a3, d3);
    g.two_sum(b2, c2, b3, c3);
    T c4 = g.add(c3, e2);
    g.two_sum(c4, d3, c5, d5);
    g.two_sum(b3, c5, b6, c6);
    g.quick_two_sum(a3, b6, r.c[0], b7);
    T c7 = g.add(c6, d5);
    g.quick_two_sum(b7, c7, r.c[1], r.c[2]);
    return r;
}

// Algorithm 12 (TWBFMul)
template <typename T, class E>
__device__ __forceinline__ mpv<T, 3> tw_mul_bf(const mpv<T, 3> &A, const mpv<T, 3> &B, E &g)
{
    T a0, b0, c0, e0, d0, f0, c1, d1, b2, c2, a3, b3, b5, c5, b6;
    mpv<T, 3> r;
    g.two_prod(A.c[0], B.c[0], a0, b0);
    g.two_prod(A.c[0], B.c[1], c0, e0);
    g.two_prod(A.c[1], B.c[0], d0, f0);
    T g0 = g.mul(A.c[0], B.c[2]);
    T h0 = g.mul(A.c[1], B.c[1]);
    T i0 = g.mul(A.c[2], B.c[0]);
    g.two_sum(c0, d0, c1, d1);
    T e1 = g.add(e0, f0);
    T g1 = g.add(g0, i0);
    g.two_sum(b0, c1, b2, c2);
    T g2 = g.add(g1, h0);
    g.quick_two_sum(a0, b2, a3, b3);
    T c3 = g.add(c2, d1);
    T e3 = g.add(e1, g2);
    T c4 = g.add(c3, e3);
    g.quick_two_sum(b3, c4, b5, c5);
    g.quick_two_sum(a3, b5, r.c[0], b6);
    g.quick_two_sum(b6, c5, r.c[1], r.c[2]);
    return r;
}

// ---------------------------------------------------------------------------
// Quad word
// ---------------------------------------------------------------------------

// Algorithm 13 (QWBFAdd)
template <typename T, class E>
__device__ __forceinline__ mpv<T, 4> qw_add_bf(const mpv<T, 4> &A, const mpv<T, 4> &B, E &g)
{
    T a1, b1, c1, d1, e1, f1, g1, h1, a2, c2, d2, e2, f2, g2, b3, g3, c3, d3, e3, f3,
        a4, c4, d4, e4, b5, d5, b6, c6, d6, e6, a7, b7, c7, d7, b8, c8, b10, c10, d10, c11;
    mpv<T, 4> r;
    g.two_sum(A.c[0], B.c[0], a1, b1);
    g.two_sum(A.c[1], B.c[1], c1, d1);
    g.two_sum(A.c[2], B.c[2], e1, f1);
    g.two_sum(A.c[3], B.c[3], g1, h1);
    g.quick_two_sum(a1, c1, a2, c2);
    T b2 = g.add(b1, h1);
    g.two_sum(d1, e1, d2, e2);
    g.two_sum(f1, g1, f2, g2);
    g.two_sum(b2, g2, b3, g3);
    g.quick_two_sum(c2, d2, c3, d3);
    g.two_sum(e2, f2, e3, f3);
    g.quick_two_sum(a2, c3, a4, c4);
    g.quick_two_sum(d3, e3, d4, e4);
    g.two_sum(b3, d4, b5, d5);
    T e5 = g.add(e4, f3);
    g.two_sum(b5, c4, b6, c6);
    g.two_sum(d5, e5, d6, e6);
    g.quick_two_sum(a4, b6, a7, b7);
    g.quick_two_sum(c6, d6, c7, d7);
    T e8 = g.add(e6, g3);
    g.quick_two_sum(b7, c7, b8, c8);
    T d9 = g.add(d7, e8);
    g.quick_two_sum(a7, b8, r.c[0], b10);
    g.quick_two_sum(c8, d9, c10, d10);
    g.quick_two_sum(b10, c10, r.c[1], c11);
    g.quick_two_sum(c11, d10, r.c[2], r.c[3]);
    return r;
}

// Algorithm 14 (QDBFMul)
template <typename T, class E>
__device__ __forceinline__ mpv<T, 4> qw_mul_bf(const mpv<T, 4> &A, const mpv<T, 4> &B, E &g)
{
    T a0, b0, c0, e0, d0, f0, g0, j0, h0, k0, i0, l0, c1, d1, e1, f1, g1, i1, b2, c2, e2, h2,
        a3, b3, c3, d3, e3, g3, c4, e4, c6, d6, b7, c7, b8, c8, d8, c9;
    mpv<T, 4> r;
    g.two_prod(A.c[0], B.c[0], a0, b0);
    g.two_prod(A.c[0], B.c[1], c0, e0);
    g.two_prod(A.c[1], B.c[0], d0, f0);
    g.two_prod(A.c[0], B.c[2], g0, j0);
    g.two_prod(A.c[1], B.c[1], h0, k0);
    g.two_prod(A.c[2], B.c[0], i0, l0);
    T m0 = g.mul(A.c[0], B.c[3]);
    T n0 = g.mul(A.c[1], B.c[2]);
    T o0 = g.mul(A.c[2], B.c[1]);
    T p0 = g.mul(A.c[3], B.c[0]);
    g.two_sum(c0, d0, c1, d1);
    g.two_sum(e0, f0, e1, f1);
    g.two_sum(g0, i0, g1, i1);
    T j1 = g.add(j0, l0);
    T m1 = g.add(m0, p0);
    T n1 = g.add(n0, o0);
    g.two_sum(b0, c1, b2, c2);
    g.two_sum(e1, h0, e2, h2);
    T f2 = g.add(f1, j1);
    T i2 = g.add(i1, k0);
    T m2 = g.add(m1, n1);
    g.quick_two_sum(a0, b2, a3, b3);
    g.quick_two_sum(c2, d1, c3, d3);
    g.two_sum(e2, g1, e3, g3);
    T f3 = g.add(f2, m2);
    T h3 = g.add(h2, i2);
    g.two_sum(c3, e3, c4, e4);
    T d4 = g.add(d3, h3);
    T f4 = g.add(f3, g3);
    T d5 = g.add(d4, e4);
    g.two_sum(c4, d5, c6, d6);
    g.two_sum(b3, c6, b7, c7);
    T d7 = g.add(d6, f4);
    g.quick_two_sum(a3, b7, r.c[0], b8);
    g.two_sum(c7, d7, c8, d8);
    g.two_sum(b8, c8, r.c[1], c9);
    g.quick_two_sum(c9, d8, r.c[2], r.c[3]);
    return r;
}

// ---------------------------------------------------------------------------
// Conventional (renormalising) triple and quad word: the "standard" side of
// Table 4.  TWAdd / TWMul are Algorithms 9 / 10; the renormalisations and the
// quad-word add / multiply, which the paper names but does not print, follow
// the QD library's published description (Hida, Li and Bailey, ARITH-15,
// 2001).  Their zero tests are real branches here: the point of this baseline
// is the data-dependent control flow that the branch-free algorithms remove.
// A zero test looks at the bit pattern (+0 and -0 are zero), which decides
// exactly like an IEEE compare but issues on the integer pipe.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool nonzero(double x)
{
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}
__device__ __forceinline__ bool nonzero(float x) { return (__float_as_uint(x) << 1) != 0u; }

// TWRenormalize of (x0, x1, x2, x3): a bottom-up sweep of QuickTwoSums, then a
// top-down one that opens a new component wherever an error term is nonzero
// (always five QuickTwoSums); the first three of the four components are kept.
template <typename T, class E>
__device__ __forceinline__ mpv<T, 3> tw_renorm(T x0, T x1, T x2, T x3, E &g)
{
    T s, t0, t1, t2, t3;
    g.quick_two_sum(x2, x3, s, t3);
    g.quick_two_sum(x1, s, s, t2);
    g.quick_two_sum(x0, s, t0, t1);
    T s0 = t0, s1 = t1, s2 = T(0), s3;
    if (nonzero(t1)) {
        g.quick_two_sum(s1, t2, s1, s2);
        if (nonzero(s2))
            g.quick_two_sum(s2, t3, s2, s3);
        else
            g.quick_two_sum(s1, t3, s1, s2);
    } else {
        g.quick_two_sum(s0, t2, s0, s1);
        if (nonzero(s1))
            g.quick_two_sum(s1, t3, s1, s2);
        else
            g.quick_two_sum(s0, t3, s0, s1);
    }
    mpv<T, 3> r;
    r.c[0] = s0;
    r.c[1] = s1;
    r.c[2] = s2;
    return r;
}

// QWRenormalize of (x0, ..., x4): the same two sweeps into four components; once
// only the last component is still open, the remaining term is added into it.
template <typename T, class E>
__device__ __forceinline__ mpv<T, 4> qw_renorm(T x0, T x1, T x2, T x3, T x4, E &g)
{
    T s, t0, t1, t2, t3, t4;
    g.quick_two_sum(x3, x4, s, t4);
    g.quick_two_sum(x2, s, s, t3);
    g.quick_two_sum(x1, s, s, t2);
    g.quick_two_sum(x0, s, t0, t1);
    T s0 = t0, s1 = t1, s2 = T(0), s3 = T(0);
    if (nonzero(t1)) {
        g.quick_two_sum(s1, t2, s1, s2);
        if (nonzero(s2)) {
            g.quick_two_sum(s2, t3, s2, s3);
            if (nonzero(s3))
                s3 = g.add(s3, t4);
            else
                g.quick_two_sum(s2, t4, s2, s3);
        } else {
            g.quick_two_sum(s1, t3, s1, s2);
            if (nonzero(s2))
                g.quick_two_sum(s2, t4, s2, s3);
            else
                g.quick_two_sum(s1, t4, s1, s2);
        }
    } else {
        g.quick_two_sum(s0, t2, s0, s1);
        if (nonzero(s1)) {
            g.quick_two_sum(s1, t3, s1, s2);
            if (nonzero(s2))
                g.quick_two_sum(s2, t4, s2, s3);
            else
                g.quick_two_sum(s1, t4, s1, s2);
        } else {
            g.quick_two_sum(s0, t3, s0, s1);
            if (nonzero(s1))
                g.quick_two_sum(s1, t4, s1, s2);
            else
                g.quick_two_sum(s0, t4, s0, s1);
        }
    }
    mpv<T, 4> r;
    r.c[0] = s0;
    r.c[1] = s1;
    r.c[2] = s2;
    r.c[3] = s3;
    return r;
}

// Algorithm 9 (TWAdd).  The three component-wise sums and their errors are the
// written-out form of three TwoSums (Algorithm 2's operation sequence).
template <typename T, class E>
__device__ __forceinline__ mpv<T, 3> tw_add_conv(const mpv<T, 3> &A, const mpv<T, 3> &B, E &g)
{
    T s0, s1, s2, t0, t1, t2, i1, i2, i3;
    g.two_sum(A.c[0], B.c[0], s0, t0);
    g.two_sum(A.c[1], B.c[1], s1, t1);
    g.two_sum(A.c[2], B.c[2], s2, t2);
    g.two_sum(s1, t0, s1, t0);
    g.two_sum(s2, t0, i1, i2);
    g.two_sum(t1, i1, s2, i3);
    g.two_sum(i2, i3, t0, t1);
    t0 = g.add(g.add(t0, t1), t2);
    return tw_renorm<T>(s0, s1, s2, t0, g);
}

// (a, b, c) -> (a + b + c, error, error) by three TwoSums (the QD library's three-sum).
template <typename T, class E> __device__ __forceinline__ void three_sum(T &a, T &b, T &c, E &g)
{
    T i1, i2, i3;
    g.two_sum(a, b, i1, i2);
    g.two_sum(c, i1, a, i3);
    g.two_sum(i2, i3, b, c);
}

// Algorithm 10 (TWMul); its final "TwoSum(q3, s1)" is read as TwoSum(t0, s1),
// the order-eps^3 sum t0 plus s1.  The unused s2 and final t1 are not formed.
template <typename T, class E>
__device__ __forceinline__ mpv<T, 3> tw_mul_conv(const mpv<T, 3> &A, const mpv<T, 3> &B, E &g)
{
    T p0, q0, p1, q1, p2, q2, p3, q3, p4, q4, p5, q5, s0, s1, t0, t1;
    g.two_prod(A.c[0], B.c[0], p0, q0);
    g.two_prod(A.c[0], B.c[1], p1, q1);
    g.two_prod(A.c[1], B.c[0], p2, q2);
    g.two_prod(A.c[0], B.c[2], p3, q3);
    g.two_prod(A.c[1], B.c[1], p4, q4);
    g.two_prod(A.c[2], B.c[0], p5, q5);
    three_sum<T>(p1, p2, q0, g);
    three_sum<T>(p2, q1, q2, g);
    three_sum<T>(p3, p4, p5, g);
    g.two_sum(p2, p3, s0, t0);
    g.two_sum(q1, p4, s1, t1);
    g.two_sum(s1, t0, s1, t0);
    g.two_sum(q0, q3, q0, q3);
    g.two_sum(q4, q5, q4, q5);
    T u;
    g.two_sum(q0, q4, t0, u);
    g.two_sum(t0, s1, t0, t1);
    return tw_renorm<T>(p0, p1, s0, t0, g);
}

// The QD library's quad-word add ("sloppy"): component-wise TwoSums, the errors
// folded in by a TwoSum, a three-sum and a three-sum with a plain add for its
// error, then QWRenormalize(s0, s1, s2, s3, t0).
template <typename T, class E>
__device__ __forceinline__ mpv<T, 4> qw_add_conv(const mpv<T, 4> &A, const mpv<T, 4> &B, E &g)
{
    T s0, s1, s2, s3, t0, t1, t2, t3, i1, i2, i3;
    g.two_sum(A.c[0], B.c[0], s0, t0);
    g.two_sum(A.c[1], B.c[1], s1, t1);
    g.two_sum(A.c[2], B.c[2], s2, t2);
    g.two_sum(A.c[3], B.c[3], s3, t3);
    g.two_sum(s1, t0, s1, t0);
    three_sum<T>(s2, t0, t1, g);
    g.two_sum(s3, t0, i1, i2);
    g.two_sum(t2, i1, s3, i3);
    t0 = g.add(i2, i3);
    t0 = g.add(g.add(t0, t1), t3);
    return qw_renorm<T>(s0, s1, s2, s3, t0, g);
}

// The QD library's quad-word multiply (accurate form): Algorithm 10's steps
// through the order-eps^2 terms; the order-eps^3 terms (errors q0, q3, q4, q5,
// products a0b3, a1b2, a2b1, a3b0, and s1) summed as double words; the
// order-eps^4 terms (a1b3, a2b2, a3b1, errors q6..q9, s2) added left to right
// into the low word; then QWRenormalize(p0, p1, s0, t0, t1).
template <typename T, class E>
__device__ __forceinline__ mpv<T, 4> qw_mul_conv(const mpv<T, 4> &A, const mpv<T, 4> &B, E &g)
{
    T p0, q0, p1, q1, p2, q2, p3, q3, p4, q4, p5, q5, p6, q6, p7, q7, p8, q8, p9, q9;
    T s0, s1, s2, t0, t1, r0, r1;
    g.two_prod(A.c[0], B.c[0], p0, q0);
    g.two_prod(A.c[0], B.c[1], p1, q1);
    g.two_prod(A.c[1], B.c[0], p2, q2);
    g.two_prod(A.c[0], B.c[2], p3, q3);
    g.two_prod(A.c[1], B.c[1], p4, q4);
    g.two_prod(A.c[2], B.c[0], p5, q5);
    three_sum<T>(p1, p2, q0, g);
    three_sum<T>(p2, q1, q2, g);
    three_sum<T>(p3, p4, p5, g);
    g.two_sum(p2, p3, s0, t0);
    g.two_sum(q1, p4, s1, t1);
    s2 = g.add(q2, p5);
    g.two_sum(s1, t0, s1, t0);
    s2 = g.add(s2, g.add(t0, t1));
    g.two_prod(A.c[0], B.c[3], p6, q6);
    g.two_prod(A.c[1], B.c[2], p7, q7);
    g.two_prod(A.c[2], B.c[1], p8, q8);
    g.two_prod(A.c[3], B.c[0], p9, q9);
    g.two_sum(q0, q3, q0, q3);
    g.two_sum(q4, q5, q4, q5);
    g.two_sum(p6, p7, p6, p7);
    g.two_sum(p8, p9, p8, p9);
    g.two_sum(q0, q4, t0, t1);
    t1 = g.add(t1, g.add(q3, q5));
    g.two_sum(p6, p8, r0, r1);
    r1 = g.add(r1, g.add(p7, p9));
    g.two_sum(t0, r0, q3, q4);
    q4 = g.add(q4, g.add(t1, r1));
    g.two_sum(q3, s1, t0, t1);
    t1 = g.add(t1, q4);
    T u = g.add(g.mul(A.c[1], B.c[3]), g.mul(A.c[2], B.c[2]));
    u = g.add(u, g.mul(A.c[3], B.c[1]));
    u = g.add(u, q6);
    u = g.add(u, q7);
    u = g.add(u, q8);
    u = g.add(u, q9);
    u = g.add(u, s2);
    t1 = g.add(t1, u);
    return qw_renorm<T>(p0, p1, s0, t0, t1, g);
}

// ---------------------------------------------------------------------------
// Precision tags: component type, K, add, multiply, reciprocal Newton steps.
// ---------------------------------------------------------------------------

#define MP_PREC_TAG(NAME, TYPE, KK, ADDF, MULF, NEWTON, FP64PIPE)                             \
    struct NAME {                                                                           \
        using T = TYPE;                                                                     \
        static constexpr int K = KK;                                                        \
        static constexpr int newton_steps = NEWTON;                                         \
        static constexpr bool fp64 = FP64PIPE;                                              \
        using V = mpv<TYPE, KK>;                                                            \
        template <class E> static __device__ __forceinline__ V add(const V &a, const V &b, E &g) \
        {                                                                                   \
            return ADDF(a, b, g);                                                           \
        }                                                                                   \
        template <class E> static __device__ __forceinline__ V mul(const V &a, const V &b, E &g) \
        {                                                                                   \
            return MULF(a, b, g);                                                           \
        }                                                                                   \
        static __device__ __forceinline__ V add(const V &a, const V &b)                     \
        {                                                                                   \
            NativeEngine<TYPE> g;                                                           \
            return ADDF(a, b, g);                                                           \
        }                                                                                   \
        static __device__ __forceinline__ V mul(const V &a, const V &b)                     \
        {                                                                                   \
            NativeEngine<TYPE> g;                                                           \
            return MULF(a, b, g);                                                           \
        }                                                                                   \
    };

MP_PREC_TAG(P_dd, double, 2, dw_add_bf<double>, dw_mul_bf<double>, 2, true)
MP_PREC_TAG(P_ddc, double, 2, dw_add_sloppy<double>, dw_mul_bf<double>, 2, true)
MP_PREC_TAG(P_td, double, 3, tw_add_bf<double>, tw_mul_bf<double>, 2, true)
MP_PREC_TAG(P_qd, double, 4, qw_add_bf<double>, qw_mul_bf<double>, 3, true)
MP_PREC_TAG(P_tdc, double, 3, tw_add_conv<double>, tw_mul_conv<double>, 2, true)
MP_PREC_TAG(P_qdc, double, 4, qw_add_conv<double>, qw_mul_conv<double>, 3, true)
MP_PREC_TAG(P_ds, float, 2, dw_add_bf<float>, dw_mul_bf<float>, 2, false)
MP_PREC_TAG(P_tf, float, 3, tw_add_bf<float>, tw_mul_bf<float>, 2, false)
MP_PREC_TAG(P_qf, float, 4, qw_add_bf<float>, qw_mul_bf<float>, 3, false)
#undef MP_PREC_TAG

// The engine the library's kernels use by default: hybrid for binary64
// components (every result still the FP64 sequence's bits, see above), native
// for binary32 components (their FP32 pipe is 64x wider, no gain).
template <class P>
using FastEngine =
    typename std::conditional<P::fp64, HybridEngine<false>, NativeEngine<typename P::T>>::type;

// ---------------------------------------------------------------------------
// Helpers over K-component values
// ---------------------------------------------------------------------------

template <class P> __device__ __forceinline__ typename P::V vzero()
{
    typename P::V r;
#pragma unroll
    for (int c = 0; c < P::K; c++) r.c[c] = typename P::T(0);
    return r;
}

template <class P> __device__ __forceinline__ typename P::V vone()
{
    typename P::V r = vzero<P>();
    r.c[0] = typename P::T(1);
    return r;
}

// Subtraction = negate every component of b, then add (Section 2).
template <class P> __device__ __forceinline__ typename P::V vneg(const typename P::V &a)
{
    typename P::V r;
#pragma unroll
    for (int c = 0; c < P::K; c++) r.c[c] = -a.c[c];
    return r;
}

template <class P>
__device__ __forceinline__ typename P::V vsub(const typename P::V &a, const typename P::V &b)
{
    return P::add(a, vneg<P>(b));
}

template <class P, class E>
__device__ __forceinline__ typename P::V vsub(const typename P::V &a, const typename P::V &b, E &g)
{
    return P::add(a, vneg<P>(b), g);
}

// Load / store element i of a K-array in plane layout (component c at base[c*ps + i]).
template <class P>
__device__ __forceinline__ typename P::V vload(const typename P::T *__restrict__ base, int64_t ps,
                                               int64_t i)
{
    typename P::V r;
#pragma unroll
    for (int c = 0; c < P::K; c++) r.c[c] = base[c * ps + i];
    return r;
}

template <class P>
__device__ __forceinline__ void vstore(typename P::T *__restrict__ base, int64_t ps, int64_t i,
                                       const typename P::V &v)
{
#pragma unroll
    for (int c = 0; c < P::K; c++) base[c * ps + i] = v.c[c];
}

// Reciprocal by Newton's method (Section 2 leaves the scheme open): y0 = 1/x[0]
// (one correctly rounded division), then newton_steps times e = 1 - x*y, y = y + y*e.
template <class P, class E> __device__ __forceinline__ typename P::V vrecip(const typename P::V &x, E &g)
{
    using T = typename P::T;
    typename P::V y = vzero<P>();
    y.c[0] = fpu<T>::div(T(1), x.c[0]);
    const typename P::V one = vone<P>();
#pragma unroll 1
    for (int s = 0; s < P::newton_steps; s++) {
        typename P::V t = P::mul(x, y, g);
        typename P::V e = vsub<P>(one, t, g);
        y = P::add(y, P::mul(y, e, g), g);
    }
    return y;
}

template <class P> __device__ __forceinline__ typename P::V vrecip(const typename P::V &x)
{
    NativeEngine<typename P::T> g;
    return vrecip<P>(x, g);
}

// Complex product with four real products: re = ar*br - ai*bi, im = ar*bi + ai*br.
template <class P, class E>
__device__ __forceinline__ void cmul(const typename P::V &ar, const typename P::V &ai, const typename P::V &br,
                                     const typename P::V &bi, typename P::V &cr, typename P::V &ci, E &g)
{
    typename P::V t1 = P::mul(ar, br, g);
    typename P::V t2 = P::mul(ai, bi, g);
    typename P::V t3 = P::mul(ar, bi, g);
    typename P::V t4 = P::mul(ai, br, g);
    cr = vsub<P>(t1, t2, g);
    ci = P::add(t3, t4, g);
}

template <class P>
__device__ __forceinline__ void cmul(const typename P::V &ar, const typename P::V &ai, const typename P::V &br,
                                     const typename P::V &bi, typename P::V &cr, typename P::V &ci)
{
    NativeEngine<typename P::T> g;
    cmul<P>(ar, ai, br, bi, cr, ci, g);
}

// Complex quotient a / b = (a * conj b) * recip(br^2 + bi^2).
template <class P, class E>
__device__ __forceinline__ void cdiv(const typename P::V &ar, const typename P::V &ai, const typename P::V &br,
                                     const typename P::V &bi, typename P::V &cr, typename P::V &ci, E &g)
{
    typename P::V n2 = P::add(P::mul(br, br, g), P::mul(bi, bi, g), g);
    typename P::V r = vrecip<P>(n2, g);
    typename P::V tr, ti;
    cmul<P>(ar, ai, br, vneg<P>(bi), tr, ti, g);
    cr = P::mul(tr, r, g);
    ci = P::mul(ti, r, g);
}

template <class P>
__device__ __forceinline__ void cdiv(const typename P::V &ar, const typename P::V &ai, const typename P::V &br,
                                     const typename P::V &bi, typename P::V &cr, typename P::V &ci)
{
    NativeEngine<typename P::T> g;
    cdiv<P>(ar, ai, br, bi, cr, ci, g);
}

}  // namespace mp
