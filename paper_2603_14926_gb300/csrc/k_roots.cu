// k_roots.cu -- batched Durand-Kerner all-roots solver (Section 4.2, Eq. 4)
// with Aberth starting values (Eq. 5), in complex multicomponent arithmetic.
//
// One block solves one polynomial.  Its monic coefficients and the current
// Jacobi iterate live in shared memory; the next iterate is written to the
// polynomial's slice of the caller's `roots` output (global memory this block
// alone owns) and copied back after the sweep's barrier, which halves the shared
// memory per block (four 128-thread blocks per SM at degree 500 in QD).  Thread
// t owns roots t, t + blockDim, ...  A sweep computes, for every owned root i,
//   q(z_i) by complex Horner over the coefficients (shared-memory broadcasts),
//   prod_{j != i} (z_i - z_j) over the current iterate (broadcasts),
//   w_i = q / prod, z_i' = z_i - w_i,
// then the block reduces delta = max |w_i| and zmax = max |z_i'| (binary64
// maxima on leading components: exact, so the reduction order cannot change
// them) and every thread takes the same stopping decision.  Per root and sweep
// this is n (4 mul + 3 add) + (n - 1) (4 mul + 4 add) multicomponent operations:
// about 1569 n FP64 instructions in QD, all on the FP64 pipe.
//
// Batching: mode 0 is one persistent launch: SMs x blocks_per_sm blocks pop
// polynomial indices from an atomic counter in the workspace (optionally in
// descending degree order, computed on the device), so uneven degrees balance
// across the GPU without host involvement; the launch is capturable in a CUDA
// graph.  Mode 1 is the plain per-polynomial launch loop (one single-block
// launch per polynomial) running the same device code, hence the same bits.
//
// Every step restates the operation order of the CPU oracle; see mpgpu.h for
// the stopping rule, the extended exponent of q and of the product, and the
// starting values.  There are no inter-block waits; the optional watchdog is a
// per-polynomial clock64 budget that ends the iteration with status 3.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <mutex>

#include "mp_arith.cuh"
#include "mp_common.cuh"

namespace mp {

enum { DK_CAP = 0, DK_CONVERGED = 1, DK_STAGNATED = 2, DK_TIMEOUT = 3, DK_BREAKDOWN = 4 };

// ---------------------------------------------------------------------------
// Binary64 helpers with fixed operation sequences (shared with nothing: the
// CPU oracle restates the same definitions independently).
// ---------------------------------------------------------------------------

__device__ __forceinline__ double pow2(int e)  // exact 2^e for -1022 <= e <= 1023
{
    return __longlong_as_double((long long)(e + 1023) << 52);
}

__device__ __forceinline__ int bexp(double x)  // biased exponent field
{
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// x = mant * 2^e with mant in [0.5, 1), for finite x > 0 (C frexp semantics).
__device__ __forceinline__ double frexp_pos(double x, int &e)
{
    int adj = 0;
    if (bexp(x) == 0) {  // subnormal: scale into the normal range first (exact)
        x = __dmul_rn(x, pow2(54));
        adj = -54;
    }
    long long u = __double_as_longlong(x);
    e = (int)((u >> 52) & 0x7ff) - 1022 + adj;
    u = (u & ~(0x7ffLL << 52)) | (1022LL << 52);
    return __longlong_as_double(u);
}

// x * 2^q correctly rounded (C ldexp), for x in [1, 2) and any q.
__device__ __forceinline__ double ldexp_pos(double x, long long q)
{
    if (q > 1023) return __dmul_rn(__dmul_rn(x, pow2(1023)), pow2((int)(q - 1023 > 1023 ? 1023 : q - 1023)));
    if (q >= -1022) return __dmul_rn(x, pow2((int)q));
    long long q2 = q + 54;
    if (q2 < -1022) return 0.0 * x;
    return __dmul_rn(__dmul_rn(x, pow2((int)q2)), pow2(-54));
}

__constant__ double kPI = 0x1.921fb54442d18p+1;
__constant__ double kLN2 = 0x1.62e42fefa39efp-1;

// cos and sin of theta in [0, 2 pi): Taylor series of cos/sin(theta - pi), 18 terms.
__device__ void dk_cos_sin(double theta, double &c, double &s)
{
    const double phi = __dsub_rn(theta, kPI);
    const double mx2 = -__dmul_rn(phi, phi);
    double ct = 1.0, cs = 1.0, st = phi, ss = phi;
    for (int k = 1; k <= 17; k++) {
        ct = __ddiv_rn(__dmul_rn(ct, mx2), (double)((2 * k - 1) * (2 * k)));
        st = __ddiv_rn(__dmul_rn(st, mx2), (double)((2 * k) * (2 * k + 1)));
        cs = __dadd_rn(cs, ct);
        ss = __dadd_rn(ss, st);
    }
    c = -cs;
    s = -ss;
}

// log2 f, f in [1, 2): 2 atanh((f-1)/(f+1)) / ln 2, series to 18 terms.
__device__ double dk_log2_1to2(double f)
{
    const double u = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double u2 = __dmul_rn(u, u);
    double pw = u, sum = u;
    for (int k = 1; k <= 17; k++) {
        pw = __dmul_rn(pw, u2);
        sum = __dadd_rn(sum, __ddiv_rn(pw, (double)(2 * k + 1)));
    }
    return __ddiv_rn(__dmul_rn(2.0, sum), kLN2);
}

// 2^t, t in [0, 1): Taylor series of exp(t ln 2), 21 terms.
__device__ double dk_exp2_0to1(double t)
{
    const double y = __dmul_rn(t, kLN2);
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 20; k++) {
        term = __ddiv_rn(__dmul_rn(term, y), (double)k);
        sum = __dadd_rn(sum, term);
    }
    return sum;
}

// v^(1/m) for v > 0, m >= 1; NaN for a non-finite v (as frexp/ldexp propagate it),
// which the radius maximum then ignores.
__device__ double dk_nthroot(double v, long long m)
{
    if (!(v < __longlong_as_double(0x7ff0000000000000LL))) return __longlong_as_double(0x7ff8000000000000LL);
    int e;
    const double mant = frexp_pos(v, e);
    const double f = __dmul_rn(2.0, mant);
    const long long ee = (long long)e - 1;
    const long long q = ee >= 0 ? ee / m : -((-ee + m - 1) / m);
    const long long s = ee - q * m;
    const double t = __ddiv_rn(__dadd_rn((double)s, dk_log2_1to2(f)), (double)m);
    return ldexp_pos(dk_exp2_0to1(t), q);
}

// x := x * 2^s componentwise, |s| <= 1000.
template <class P> __device__ __forceinline__ void vscale(typename P::V &x, int s)
{
    const double f = pow2(s);
#pragma unroll
    for (int c = 0; c < P::K; c++) x.c[c] = __dmul_rn(x.c[c], f);
}

template <class P> __device__ __forceinline__ void vscale_big(typename P::V &x, long long d)
{
    while (d > 512) {
        vscale<P>(x, 512);
        d -= 512;
    }
    while (d < -512) {
        vscale<P>(x, -512);
        d += 512;
    }
    if (d != 0) vscale<P>(x, (int)d);
}

constexpr int DK_RESCALE = 256;

// ---------------------------------------------------------------------------
// Shared-memory layout of one polynomial's solve
// ---------------------------------------------------------------------------

// Split sweeps (a small polynomial in a wide block): the product chains' exponents
// and domain flags for the threads that finish the roots.
constexpr int DK_SPLIT_MAX = 128;

struct DKShared {
    double delta, zmax, center, radius;
    int bad, stop, nnz, pad;
    double red[2][32];
    int redi[32];
    long long split_e[DK_SPLIT_MAX];
    int split_bad[DK_SPLIT_MAX];
};

template <class P> struct DKArgs {
    int64_t npoly;
    const int64_t *coef_off;
    const double *coef;
    int64_t pcoef;
    const double *z0;
    int64_t pz0;
    double *roots;
    int64_t proots;
    int32_t *iters;   // nullptr: do not write statistics
    int32_t *status;
    double tol;
    int32_t max_iter, win, kmin;
    double radius;
    long long watchdog;
    int32_t max_degree;
    const int32_t *order;  // nullptr: natural order
    unsigned long long *counter;  // persistent work queue (64-bit: pops past the end never wrap)
    double *gscratch;      // nullptr: coefficients and iterate in shared memory; else per-block slots
    int64_t gstride;       // doubles per block slot of gscratch
};

// block-wide max of two doubles and OR of a flag; result in sh
__device__ void block_max2(DKShared &sh, double a, double b, int bad)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a = fmax(a, __shfl_down_sync(0xffffffffu, a, off));
        b = fmax(b, __shfl_down_sync(0xffffffffu, b, off));
        bad |= __shfl_down_sync(0xffffffffu, bad, off);
    }
    if (lane == 0) {
        sh.red[0][warp] = a;
        sh.red[1][warp] = b;
        sh.redi[warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        int f = 0;
        for (int w = 0; w < nw; w++) {
            x = fmax(x, sh.red[0][w]);
            y = fmax(y, sh.red[1][w]);
            f |= sh.redi[w];
        }
        sh.delta = x;
        sh.zmax = y;
        sh.bad = f;
    }
    __syncthreads();
}

// The hybrid engine of the solver packs subnormal TwoSum error terms too: from
// the second sweep on, some updates meet operands whose lower components fall
// through the bottom of the binary64 range (imaginary parts of iterates that
// converge to real roots, for one), and with the default engine every such root
// was recomputed on the FP64 pipe (about 46,000 roots per sweep of the batched
// workload, each a full update run by a few lanes of a warp).
using DKHybrid = HybridEngine<false, false, true>;

// Roots recomputed on the FP64 pipe because the hybrid engine left its domain
// (all precisions; read by mp_roots_hybrid_fallbacks).
static __device__ unsigned long long mp_dk_fallbacks;

// The hybrid engine's multicomponent add and multiply, called out of line.  The
// root update holds about fifteen of them per step; inlined, the hybrid code
// overflows the instruction cache.  Each call runs its own engine and hands its
// domain flag back with the result.
template <class P> struct HybridResult {
    typename P::V v;
    uint32_t bad;
};

template <class P>
__device__ __noinline__ HybridResult<P> hybrid_add_call(typename P::V a, typename P::V b)
{
    DKHybrid h;
    const typename P::V r = P::add(a, b, h);
    return {r, h.bad};
}

template <class P>
__device__ __noinline__ HybridResult<P> hybrid_mul_call(typename P::V a, typename P::V b)
{
    DKHybrid h;
    const typename P::V r = P::mul(a, b, h);
    return {r, h.bad};
}

// A precision tag whose add and multiply on the hybrid engine are those calls
// (the native engine stays inline).
template <class P> struct OutlinedHybrid : P {
    using V = typename P::V;
    static __device__ __forceinline__ V add(const V &a, const V &b, DKHybrid &g)
    {
        const HybridResult<P> r = hybrid_add_call<P>(a, b);
        g.bad |= r.bad;
        return r.v;
    }
    static __device__ __forceinline__ V mul(const V &a, const V &b, DKHybrid &g)
    {
        const HybridResult<P> r = hybrid_mul_call<P>(a, b);
        g.bad |= r.bad;
        return r.v;
    }
    template <class E> static __device__ __forceinline__ V add(const V &a, const V &b, E &g)
    {
        return P::add(a, b, g);
    }
    template <class E> static __device__ __forceinline__ V mul(const V &a, const V &b, E &g)
    {
        return P::mul(a, b, g);
    }
    static __device__ __forceinline__ V add(const V &a, const V &b) { return P::add(a, b); }
    static __device__ __forceinline__ V mul(const V &a, const V &b) { return P::mul(a, b); }
};

// One Horner step of q(z_i) on coefficient kk, with the extended exponent Eq.
template <class P, class E>
__device__ __forceinline__ void dk_horner_step(const double *c, int64_t cap, int64_t kk, const typename P::V &zr,
                                               const typename P::V &zi, typename P::V &hr, typename P::V &hi,
                                               long long &Eq, E &g)
{
    using V = typename P::V;
    V a = vload<P>(c, cap, kk);
    if (Eq > 1000) a = vzero<P>();
    else if (Eq > 0) vscale<P>(a, (int)-Eq);
    V t1 = P::mul(hr, zr, g);
    V t2 = P::mul(hi, zi, g);
    t1 = vsub<P>(t1, t2, g);
    t1 = P::add(t1, a, g);
    V t3 = P::mul(hr, zi, g);
    V t4 = P::mul(hi, zr, g);
    hi = P::add(t3, t4, g);
    hr = t1;
    const int be = max(bexp(hr.c[0]), bexp(hi.c[0]));
    if (be >= 1023 + DK_RESCALE + 1) {
        vscale<P>(hr, -DK_RESCALE);
        vscale<P>(hi, -DK_RESCALE);
        Eq += DK_RESCALE;
    }
}

// One step of prod_{j != i} (z_i - z_j) with j given, with the extended exponent Ed.
template <class P, class E>
__device__ __forceinline__ void dk_product_step(const double *z, int64_t zc, int64_t j, const typename P::V &zr,
                                                const typename P::V &zi, typename P::V &dr, typename P::V &di,
                                                long long &Ed, E &g)
{
    using V = typename P::V;
    constexpr int K = P::K;
    const V tr = vsub<P>(zr, vload<P>(z, zc, j), g);
    const V ti = vsub<P>(zi, vload<P>(z + K * zc, zc, j), g);
    cmul<P>(dr, di, tr, ti, dr, di, g);
    const int be = max(bexp(dr.c[0]), bexp(di.c[0]));
    if (be >= 1023 + DK_RESCALE + 1) {
        vscale<P>(dr, -DK_RESCALE);
        vscale<P>(di, -DK_RESCALE);
        Ed += DK_RESCALE;
    } else if (be <= 1023 - DK_RESCALE - 1 && (dr.c[0] != 0.0 || di.c[0] != 0.0)) {
        vscale<P>(dr, DK_RESCALE);
        vscale<P>(di, DK_RESCALE);
        Ed -= DK_RESCALE;
    }
}

// w_i = q(z_i) / prod, rescaled by 2^(Eq - Ed), and y_i = z_i - w_i.
template <class P, class E>
__device__ __forceinline__ void dk_finish(const typename P::V &hr, const typename P::V &hi, long long Eq,
                                          const typename P::V &dr, const typename P::V &di, long long Ed,
                                          const typename P::V &zr, const typename P::V &zi, typename P::V &yr,
                                          typename P::V &yi, typename P::V &wr, typename P::V &wi, E &g)
{
    cdiv<P>(hr, hi, dr, di, wr, wi, g);
    vscale_big<P>(wr, Eq - Ed);
    vscale_big<P>(wi, Eq - Ed);
    yr = vsub<P>(zr, wr, g);
    yi = vsub<P>(zi, wi, g);
}

// One root's Durand-Kerner update (Eq. 4): w_i = q(z_i) / prod_{j != i} (z_i - z_j)
// with extended exponents for both factors, y_i = z_i - w_i; every multicomponent
// operation on the engine g.  q(z_i) (Horner, coefficients n-1 down to 0) and the
// product (j ascending) are independent recurrences: one loop advances both, so
// the two dependency chains overlap; each keeps its own order and exponent.
template <class P, class E>
__device__ __forceinline__ void dk_update(int64_t i, int64_t n, const double *c, int64_t cap, const double *z,
                                          int64_t zc, const typename P::V &zr, const typename P::V &zi,
                                          typename P::V &yr, typename P::V &yi, typename P::V &wr,
                                          typename P::V &wi, E &g)
{
    using V = typename P::V;
    V hr = vload<P>(c, cap, n), hi = vzero<P>();
    long long Eq = 0;
    V dr = vone<P>(), di = vzero<P>();
    long long Ed = 0;
    for (int64_t t = 0; t < n; t++) {
        dk_horner_step<P>(c, cap, n - 1 - t, zr, zi, hr, hi, Eq, g);
        if (t != i) dk_product_step<P>(z, zc, t, zr, zi, dr, di, Ed, g);
    }
    dk_finish<P>(hr, hi, Eq, dr, di, Ed, zr, zi, yr, yi, wr, wi, g);
}

// The same update on the FP64 pipe, out of line: taken only when the hybrid
// engine left its domain, so it need not share the hot path's registers.
template <class P>
__device__ __noinline__ void dk_update_native(int64_t i, int64_t n, const double *c, int64_t cap, const double *z,
                                              int64_t zc, const typename P::V &zr, const typename P::V &zi,
                                              typename P::V &yr, typename P::V &yi, typename P::V &wr,
                                              typename P::V &wi)
{
    NativeEngine<double> nat;
    dk_update<P>(i, n, c, cap, z, zc, zr, zi, yr, yi, wr, wi, nat);
}

// Set-up of one polynomial's solve, by every thread of the block: monic
// coefficients into c (K planes, stride cap) and the starting values into z
// (2K planes, stride zc).
template <class P>
__device__ void dk_setup(const DKArgs<P> &A, int64_t n, int64_t off, int64_t ro, double *c, int64_t cap, double *z,
                         int64_t zc, DKShared &sh)
{
    using V = typename P::V;
    constexpr int K = P::K;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t i = tid; i <= n; i += nt)
        for (int cc = 0; cc < K; cc++) c[cc * cap + i] = A.coef[cc * A.pcoef + off + i];
    __syncthreads();
    // monic q_n = p_n / a_n unless a_n == 1 exactly
    bool monic = c[n] == 1.0;
    for (int cc = 1; cc < K; cc++) monic = monic && c[cc * cap + n] == 0.0;
    if (!monic) {
        const V inv = vrecip<P>(vload<P>(c, cap, n));
        __syncthreads();
        for (int64_t i = tid; i < n; i += nt) vstore<P>(c, cap, i, P::mul(vload<P>(c, cap, i), inv));
        __syncthreads();
        if (tid == 0)
            for (int cc = 0; cc < K; cc++) c[cc * cap + n] = cc == 0 ? 1.0 : 0.0;
        __syncthreads();
    }

    // starting values
    if (A.z0) {
        for (int64_t i = tid; i < n; i += nt)
            for (int cc = 0; cc < 2 * K; cc++) z[cc * zc + i] = A.z0[cc * A.pz0 + ro + i];
    } else {
        double r = 0.0;
        if (A.radius > 0.0) {
            r = A.radius;
        } else {
            int cnt = 0;
            for (int64_t i = tid; i < n; i += nt) cnt += c[i] != 0.0;
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if ((tid & 31) == 0) sh.redi[tid >> 5] = cnt;
            __syncthreads();
            if (tid == 0) {
                int s = 0;
                for (int w = 0; w < (nt + 31) / 32; w++) s += sh.redi[w];
                sh.nnz = s;
            }
            __syncthreads();
            const double nnz = (double)sh.nnz;
            for (int64_t i = tid; i < n; i += nt) {
                if (c[i] == 0.0) continue;
                const double v = fabs(__dmul_rn(nnz, c[i]));
                const double rt = dk_nthroot(v, n - i);
                if (rt > r) r = rt;
            }
            block_max2(sh, r, 0.0, 0);
            r = sh.delta;
            if (r == 0.0) r = 1.0;
        }
        const double center = -__ddiv_rn(c[n - 1], (double)n);
        for (int64_t i = tid; i < n; i += nt) {
            const double th = __dadd_rn(__ddiv_rn(__dmul_rn(2.0 * (double)i, kPI), (double)n),
                                        __ddiv_rn(3.0, 2.0 * (double)n));
            double cs, sn;
            dk_cos_sin(th, cs, sn);
            for (int cc = 0; cc < 2 * K; cc++) z[cc * zc + i] = 0.0;
            z[i] = __dadd_rn(center, __dmul_rn(r, cs));
            z[K * zc + i] = __dmul_rn(r, sn);
        }
    }
    __syncthreads();
}

template <class P, class E>
__device__ void dk_solve(const DKArgs<P> &A, int64_t b, DKShared &sh, double *smem)
{
    using V = typename P::V;
    constexpr int K = P::K;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t off = A.coef_off[b];
    const int64_t n = A.coef_off[b + 1] - off - 1;
    const int64_t ro = off - b;  // root offset
    if (n <= 0 || n > A.max_degree) {
        if (tid == 0 && A.iters) {
            A.iters[b] = 0;
            A.status[b] = n <= 0 ? DK_CONVERGED : DK_BREAKDOWN;
        }
        return;
    }
    const int64_t cap = (int64_t)A.max_degree + 1;  // coefficient plane stride
    const int64_t zc = A.max_degree;                // iterate plane stride
    // K planes of coefficients, then 2K planes of the current iterate: in shared
    // memory, or (degrees above the shared-memory bound) in this block's slot of
    // the caller's workspace, which only this block touches
    double *c = A.gscratch ? A.gscratch + (int64_t)blockIdx.x * A.gstride : smem;
    double *z = c + K * cap;
    double *zn = A.roots + ro;                      // 2K planes, stride proots: next iterate
    const int64_t pn = A.proots;

    dk_setup<P>(A, n, off, ro, c, cap, z, zc, sh);

    const bool split = nt % 64 == 0 && n <= nt / 2 && n <= DK_SPLIT_MAX;
    // Product chains of a split sweep start 64 threads (two warps) after the Horner
    // chains when both fit in two warps each, else at the block's upper half: the
    // two chains of a root then run on different SM sub-partitions (warp w issues
    // on sub-partition w mod 4).
    const int poff = (n <= 64 && nt >= 128) ? 64 : nt / 2;
    // Roots are dealt to threads from a warp offset that rotates with the
    // polynomial and the sweep, so the partial last round of a sweep (and the
    // chains of a small polynomial) does not always load the same warps -- the
    // same sub-partitions -- of every block.  Each root's arithmetic is unchanged.
    const int nwarps = nt % 32 == 0 ? nt / 32 : 0;
    const long long t0 = clock64();
    int st = DK_CAP, it = A.max_iter;
    double best = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    int since = 0;
    for (int k = 1; k <= A.max_iter; k++) {
        double dmax = 0.0, zm = 0.0;
        int bad = 0;
        const int rot = nwarps > 1 ? 32 * (int)((b + k) % nwarps) : 0;
        const int vt = (tid + nt - rot) % nt;  // this thread's place in the dealing order
        using PU = typename std::conditional<std::is_same<E, DKHybrid>::value, OutlinedHybrid<P>, P>::type;
        if (split) {
            // Two threads per root: places poff .. poff+n-1 of the dealing order run
            // the product chains and leave them in the root's next-iterate slot,
            // places 0 .. n-1 run the Horner chains and then finish the roots.  Each
            // warp carries one chain instead of two, and every chain keeps its order.
            if (vt >= poff && vt - poff < n) {
                const int64_t i = vt - poff;
                const V zr = vload<P>(z, zc, i), zi = vload<P>(z + K * zc, zc, i);
                V dr = vone<P>(), di = vzero<P>();
                long long Ed = 0;
                E g;
                for (int64_t j = 0; j < n; j++)
                    if (j != i) dk_product_step<PU>(z, zc, j, zr, zi, dr, di, Ed, g);
                vstore<P>(zn, pn, i, dr);
                vstore<P>(zn + K * pn, pn, i, di);
                sh.split_e[i] = Ed;
                sh.split_bad[i] = g.failed() ? 1 : 0;
            }
            V zr = vzero<P>(), zi = vzero<P>(), hr = vzero<P>(), hi = vzero<P>();
            long long Eq = 0;
            E g;
            if (vt < n) {
                zr = vload<P>(z, zc, vt);
                zi = vload<P>(z + K * zc, zc, vt);
                hr = vload<P>(c, cap, n);
                for (int64_t kk = n - 1; kk >= 0; kk--) dk_horner_step<PU>(c, cap, kk, zr, zi, hr, hi, Eq, g);
            }
            __syncthreads();  // the products are in place
            if (vt < n) {
                const int64_t i = vt;
                const V dr = vload<P>(zn, pn, i), di = vload<P>(zn + K * pn, pn, i);
                V yr, yi, wr, wi;
                dk_finish<PU>(hr, hi, Eq, dr, di, sh.split_e[i], zr, zi, yr, yi, wr, wi, g);
                if (g.failed() || sh.split_bad[i]) {
                    atomicAdd(&mp_dk_fallbacks, 1ull);
                    dk_update_native<P>(i, n, c, cap, z, zc, zr, zi, yr, yi, wr, wi);
                }
                vstore<P>(zn, pn, i, yr);
                vstore<P>(zn + K * pn, pn, i, yi);
                const double d = __dadd_rn(fabs(wr.c[0]), fabs(wi.c[0]));
                const double m = __dadd_rn(fabs(yr.c[0]), fabs(yi.c[0]));
                if (!(d == d) || isinf(d) || !(m == m) || isinf(m)) bad = 1;
                if (d > dmax) dmax = d;
                if (m > zm) zm = m;
            }
        } else {
            for (int64_t i = vt; i < n; i += nt) {
                const V zr = vload<P>(z, zc, i), zi = vload<P>(z + K * zc, zc, i);
                V yr, yi, wr, wi;
                E g;
                dk_update<PU>(i, n, c, cap, z, zc, zr, zi, yr, yi, wr, wi, g);
                if (g.failed()) {
                    atomicAdd(&mp_dk_fallbacks, 1ull);
                    dk_update_native<P>(i, n, c, cap, z, zc, zr, zi, yr, yi, wr, wi);
                }
                vstore<P>(zn, pn, i, yr);
                vstore<P>(zn + K * pn, pn, i, yi);
                const double d = __dadd_rn(fabs(wr.c[0]), fabs(wi.c[0]));
                const double m = __dadd_rn(fabs(yr.c[0]), fabs(yi.c[0]));
                if (!(d == d) || isinf(d) || !(m == m) || isinf(m)) bad = 1;
                if (d > dmax) dmax = d;
                if (m > zm) zm = m;
            }
        }
        block_max2(sh, dmax, zm, bad);  // barrier: every read of the current iterate is done
        for (int64_t i = tid; i < n; i += nt)  // copy back (after the barrier any thread may)
            for (int cc = 0; cc < 2 * K; cc++) z[cc * zc + i] = zn[cc * pn + i];
        __syncthreads();
        const double delta = sh.delta, zmax = sh.zmax;
        const double scale = zmax > 1.0 ? zmax : 1.0;
        if (sh.bad) { st = DK_BREAKDOWN; it = k; break; }
        if (delta <= __dmul_rn(A.tol, scale)) { st = DK_CONVERGED; it = k; break; }
        if (delta < best) { best = delta; since = 0; } else { since++; }
        if (k >= A.kmin && since >= A.win && best <= __dmul_rn(pow2(-26 * K), scale)) {
            st = DK_STAGNATED;
            it = k;
            break;
        }
        if (A.watchdog > 0) {
            if (tid == 0) sh.stop = (clock64() - t0) > A.watchdog;
            __syncthreads();
            const int stop = sh.stop;
            __syncthreads();
            if (stop) { st = DK_TIMEOUT; it = k; break; }
        }
    }
    for (int64_t i = tid; i < n; i += nt)  // (the start values when no sweep ran)
        for (int cc = 0; cc < 2 * K; cc++) zn[cc * pn + i] = z[cc * zc + i];
    if (tid == 0 && A.iters) {
        A.iters[b] = it;
        A.status[b] = st;
    }
    __syncthreads();
}

// Register budgets: the native engine at its natural size (3 blocks of 128
// threads per SM fit), the hybrid engine capped at 128 so that 2 blocks of 256
// threads stay resident (its integer dependency chains need the warps).
template <class E> struct DKLaunch {
    static constexpr int min_blocks = 0, default_threads = 128;
};
template <> struct DKLaunch<DKHybrid> {
    static constexpr int min_blocks = 2, default_threads = 256;
};

template <class P, class E>
__global__ void __launch_bounds__(256, DKLaunch<E>::min_blocks) k_dk_persistent(DKArgs<P> A)
{
    extern __shared__ __align__(16) double dk_smem[];
    __shared__ DKShared sh;
    __shared__ unsigned long long next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(A.counter, 1ull);
        __syncthreads();
        const unsigned long long p = next;
        __syncthreads();
        if (p >= (unsigned long long)A.npoly) break;
        dk_solve<P, E>(A, A.order ? A.order[p] : (int64_t)p, sh, dk_smem);
    }
}

template <class P, class E>
__global__ void __launch_bounds__(256, DKLaunch<E>::min_blocks) k_dk_single(DKArgs<P> A, int64_t p)
{
    extern __shared__ __align__(16) double dk_smem[];
    __shared__ DKShared sh;
    dk_solve<P, E>(A, A.order ? A.order[p] : p, sh, dk_smem);
}

// ---------------------------------------------------------------------------
// Cluster solve (mode 2): one polynomial per thread-block cluster of C CTAs on
// C SMs, for latency (one or a few polynomials of degree <= 32 C).  A single
// block is bound by its SM's FP64 pipe; here CTA r owns roots r m .. r m + m - 1
// (m = ceil(n / C)) and every complex step of a root's two recurrences is split
// over a lane pair: the even lane forms the real part, the odd lane the
// imaginary part, each with the same two products and add(s) in the same order
// as the one-lane step, and the pair swaps its halves by shuffle.  So each
// root's Horner value, product and update are bit-identical to the one-block
// solver's.  Each CTA holds the coefficients and the whole current iterate in
// shared memory; after a sweep every CTA writes its new roots into every CTA's
// next-iterate buffer and its (delta, zmax, flags) into every CTA's slot
// array through distributed shared memory, then one cluster barrier (release /
// acquire) publishes them, and every CTA takes the same decision from the same
// exact maxima.  Buffers alternate with the sweep's parity, so a CTA that runs
// ahead never overwrites what another still reads.
// ---------------------------------------------------------------------------

constexpr int DK_CLUSTER_THREADS = 128;  // two Horner and two product warps at m = 32
constexpr int DK_CLUSTER_MAX = 8;        // portable cluster size: degrees <= 256

template <class P> __device__ __forceinline__ typename P::V pair_swap(const typename P::V &v)
{
    typename P::V r;
#pragma unroll
    for (int c = 0; c < P::K; c++) r.c[c] = __shfl_xor_sync(0xffffffffu, v.c[c], 1);
    return r;
}

// Horner step of q(z_i) on coefficient kk, split over a lane pair (im = 0: real
// part, 1: imaginary part).  One-lane form: t1 = hr zr, t2 = hi zi,
// hr' = (t1 - t2) + a; t3 = hr zi, t4 = hi zr, hi' = t3 + t4.
template <class P, class E>
__device__ __forceinline__ void dk_horner_pair(const double *c, int64_t cap, int64_t kk, const typename P::V &zr,
                                               const typename P::V &zi, typename P::V &hr, typename P::V &hi,
                                               long long &Eq, int im, E &g)
{
    using V = typename P::V;
    V a = vload<P>(c, cap, kk);
    if (Eq > 1000) a = vzero<P>();
    else if (Eq > 0) vscale<P>(a, (int)-Eq);
    const V u = P::mul(hr, im ? zi : zr, g);
    const V v = P::mul(hi, im ? zr : zi, g);
    V w = P::add(u, im ? v : vneg<P>(v), g);
    if (!im) w = P::add(w, a, g);
    const V o = pair_swap<P>(w);
    hr = im ? o : w;
    hi = im ? w : o;
    const int be = max(bexp(hr.c[0]), bexp(hi.c[0]));
    if (be >= 1023 + DK_RESCALE + 1) {
        vscale<P>(hr, -DK_RESCALE);
        vscale<P>(hi, -DK_RESCALE);
        Eq += DK_RESCALE;
    }
}

// Product step (z_i - z_j) split over a lane pair: each lane forms one part of
// the difference, the pair swaps them, then each lane forms one part of the
// complex product in cmul's order (re = t1 - t2, im = t3 + t4).  `take` false
// (j == i) computes the same instructions and keeps the old product, so every
// lane of the warp reaches every shuffle.
template <class P, class E>
__device__ __forceinline__ void dk_product_pair(const double *z, int64_t zc, int64_t j, bool take, const typename P::V &zr,
                                                const typename P::V &zi, typename P::V &dr, typename P::V &di,
                                                long long &Ed, int im, E &g)
{
    using V = typename P::V;
    constexpr int K = P::K;
    const uint32_t bad0 = g.bad_flags();
    const V d = vsub<P>(im ? zi : zr, vload<P>(z + (im ? K * zc : 0), zc, j), g);
    const V od = pair_swap<P>(d);
    const V tr = im ? od : d, ti = im ? d : od;
    const V u = P::mul(dr, im ? ti : tr, g);
    const V v = P::mul(di, im ? tr : ti, g);
    const V w = P::add(u, im ? v : vneg<P>(v), g);
    const V o = pair_swap<P>(w);
    V nr = im ? o : w, ni = im ? w : o;
    long long nE = Ed;
    const int be = max(bexp(nr.c[0]), bexp(ni.c[0]));
    if (be >= 1023 + DK_RESCALE + 1) {
        vscale<P>(nr, -DK_RESCALE);
        vscale<P>(ni, -DK_RESCALE);
        nE += DK_RESCALE;
    } else if (be <= 1023 - DK_RESCALE - 1 && (nr.c[0] != 0.0 || ni.c[0] != 0.0)) {
        vscale<P>(nr, DK_RESCALE);
        vscale<P>(ni, DK_RESCALE);
        nE -= DK_RESCALE;
    }
    if (take) {
        dr = nr;
        di = ni;
        Ed = nE;
    } else {
        g.set_bad_flags(bad0);
    }
}

// The same two steps split over a lane quad (role 0..3 = lane & 3): each lane
// forms one of the four real products of the complex product, the quad swaps
// them in pairs (roles 0 <-> 1, 2 <-> 3) to form the real part (roles 0, 1:
// t1 - t2) and the imaginary part (roles 2, 3: t3 + t4) in the one-lane
// order, and a second swap (roles 0 <-> 2, 1 <-> 3) hands both parts to every
// lane.  Lanes that form the same part form it from the same operands, so they
// agree bit for bit.  One multiply per lane and step instead of two.
template <class P> __device__ __forceinline__ typename P::V quad_swap(const typename P::V &v, int mask)
{
    typename P::V r;
#pragma unroll
    for (int c = 0; c < P::K; c++) r.c[c] = __shfl_xor_sync(0xffffffffu, v.c[c], mask);
    return r;
}

template <class P, class E>
__device__ __forceinline__ void dk_horner_quad(const double *c, int64_t cap, int64_t kk, const typename P::V &zr,
                                               const typename P::V &zi, typename P::V &hr, typename P::V &hi,
                                               long long &Eq, int role, E &g)
{
    using V = typename P::V;
    V a = vload<P>(c, cap, kk);
    if (Eq > 1000) a = vzero<P>();
    else if (Eq > 0) vscale<P>(a, (int)-Eq);
    // role 0: t1 = hr zr, 1: t2 = hi zi, 2: t3 = hr zi, 3: t4 = hi zr
    const V t = P::mul((role & 1) ? hi : hr, (role == 1 || role == 2) ? zi : zr, g);
    const V o = quad_swap<P>(t, 1);
    // roles 0, 1: t1 + (-t2); roles 2, 3: t3 + t4 -- one add for the whole warp
    const V x = (role & 1) ? o : t, y = (role & 1) ? t : o;
    V w = P::add(x, role < 2 ? vneg<P>(y) : y, g);
    if (role < 2) w = P::add(w, a, g);
    const V ow = quad_swap<P>(w, 2);
    hr = role < 2 ? w : ow;
    hi = role < 2 ? ow : w;
    const int be = max(bexp(hr.c[0]), bexp(hi.c[0]));
    if (be >= 1023 + DK_RESCALE + 1) {
        vscale<P>(hr, -DK_RESCALE);
        vscale<P>(hi, -DK_RESCALE);
        Eq += DK_RESCALE;
    }
}

template <class P, class E>
__device__ __forceinline__ void dk_product_quad(const double *z, int64_t zc, int64_t j, bool take,
                                                const typename P::V &zr, const typename P::V &zi, typename P::V &dr,
                                                typename P::V &di, long long &Ed, int role, E &g)
{
    using V = typename P::V;
    constexpr int K = P::K;
    const uint32_t bad0 = g.bad_flags();
    // roles 0, 2: tr = zr - z_j (real), roles 1, 3: ti = zi - z_j (imaginary)
    const int part = role & 1;
    const V d = vsub<P>(part ? zi : zr, vload<P>(z + (part ? K * zc : 0), zc, j), g);
    const V od = quad_swap<P>(d, 1);
    const V tr = part ? od : d, ti = part ? d : od;
    // role 0: t1 = dr tr, 1: t2 = di ti, 2: t3 = dr ti, 3: t4 = di tr
    const V t = P::mul((role & 1) ? di : dr, (role == 1 || role == 2) ? ti : tr, g);
    const V o = quad_swap<P>(t, 1);
    // roles 0, 1: t1 + (-t2); roles 2, 3: t3 + t4 -- one add for the whole warp
    const V x = (role & 1) ? o : t, y = (role & 1) ? t : o;
    const V w = P::add(x, role < 2 ? vneg<P>(y) : y, g);
    const V ow = quad_swap<P>(w, 2);
    V nr = role < 2 ? w : ow, ni = role < 2 ? ow : w;
    long long nE = Ed;
    const int be = max(bexp(nr.c[0]), bexp(ni.c[0]));
    if (be >= 1023 + DK_RESCALE + 1) {
        vscale<P>(nr, -DK_RESCALE);
        vscale<P>(ni, -DK_RESCALE);
        nE += DK_RESCALE;
    } else if (be <= 1023 - DK_RESCALE - 1 && (nr.c[0] != 0.0 || ni.c[0] != 0.0)) {
        vscale<P>(nr, DK_RESCALE);
        vscale<P>(ni, DK_RESCALE);
        nE -= DK_RESCALE;
    }
    if (take) {
        dr = nr;
        di = ni;
        Ed = nE;
    } else {
        g.set_bad_flags(bad0);
    }
}

template <class P, class E, int L>
__global__ void __launch_bounds__(DK_CLUSTER_THREADS) k_dk_cluster(DKArgs<P> A)
{
    namespace cg = cooperative_groups;
    using V = typename P::V;
    constexpr int K = P::K;
    using PU = typename std::conditional<std::is_same<E, DKHybrid>::value, OutlinedHybrid<P>, P>::type;
    extern __shared__ __align__(16) double dk_smem[];
    __shared__ DKShared sh;
    __shared__ double slot[2][DK_CLUSTER_MAX][4];  // per sweep parity and CTA: delta, zmax, bad, stop
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x / C;
    const int64_t off = A.coef_off[b];
    const int64_t n = A.coef_off[b + 1] - off - 1;
    const int64_t ro = off - b;
    if (n <= 0 || n > A.max_degree) {  // the same for every CTA of the cluster: no barrier is reached
        if (rank == 0 && tid == 0) {
            A.iters[b] = 0;
            A.status[b] = n <= 0 ? DK_CONVERGED : DK_BREAKDOWN;
        }
        return;
    }
    const int64_t cap = (int64_t)A.max_degree + 1, zc = A.max_degree;
    const int64_t m = (n + C - 1) / C;                  // roots per CTA (<= 64 / L)
    double *c = dk_smem;                                // K planes
    double *zbuf[2] = {c + K * cap, c + K * cap + 2 * K * zc};  // 2K planes each
    double *pbuf = c + K * cap + 4 * K * zc;            // 2K planes of m: the products
    long long *pE = reinterpret_cast<long long *>(pbuf + 2 * K * m);
    int *pbad = reinterpret_cast<int *>(pE + m);

    dk_setup<P>(A, n, off, ro, c, cap, zbuf[0], zc, sh);
    cluster.sync();  // every CTA of the cluster runs before any remote write

    const int64_t r0 = (int64_t)rank * m;
    const int64_t cnt = n - r0 < m ? (n - r0 > 0 ? n - r0 : 0) : m;  // roots this CTA owns
    const int hw = (int)((L * m + 31) / 32);            // warps of Horner lane groups, then as many of product ones
    const int warp = tid >> 5, im = tid & (L - 1);      // a lane's role within its group
    const bool horner = warp < hw, prod = !horner && warp < 2 * hw;
    const int64_t q = horner ? tid / L : (tid - 32 * hw) / L;   // group (root) index within the CTA
    const bool valid = (horner || prod) && q < cnt;
    const int64_t i = cnt > 0 ? r0 + (q < cnt ? q : cnt - 1) : 0;  // ghost pairs repeat a valid root

    const long long t0 = clock64();
    int st = DK_CAP, it = A.max_iter;
    double best = __longlong_as_double(0x7ff0000000000000LL);
    int since = 0;
    for (int k = 1; k <= A.max_iter; k++) {
        const int par = (k - 1) & 1;
        double *z = zbuf[par], *zn = zbuf[par ^ 1];
        const V zr = vload<P>(z, zc, i), zi = vload<P>(z + K * zc, zc, i);
        V hr = vzero<P>(), hi = vzero<P>();
        long long Eq = 0;
        uint32_t hbad = 0;
        E g;
        if (prod) {
            V dr = vone<P>(), di = vzero<P>();
            long long Ed = 0;
            if (L == 4)
                for (int64_t j = 0; j < n; j++) dk_product_quad<PU>(z, zc, j, j != i, zr, zi, dr, di, Ed, im, g);
            else
                for (int64_t j = 0; j < n; j++) dk_product_pair<PU>(z, zc, j, j != i, zr, zi, dr, di, Ed, im, g);
            uint32_t fb = g.bad_flags() | __shfl_xor_sync(0xffffffffu, g.bad_flags(), 1);
            if (L == 4) fb |= __shfl_xor_sync(0xffffffffu, fb, 2);
            if (valid && !im) {
                vstore<P>(pbuf, m, q, dr);
                vstore<P>(pbuf + K * m, m, q, di);
                pE[q] = Ed;
                pbad[q] = fb != 0;
            }
        } else if (horner) {
            hr = vload<P>(c, cap, n);
            if (L == 4)
                for (int64_t kk = n - 1; kk >= 0; kk--) dk_horner_quad<PU>(c, cap, kk, zr, zi, hr, hi, Eq, im, g);
            else
                for (int64_t kk = n - 1; kk >= 0; kk--) dk_horner_pair<PU>(c, cap, kk, zr, zi, hr, hi, Eq, im, g);
            hbad = g.bad_flags() | __shfl_xor_sync(0xffffffffu, g.bad_flags(), 1);
            if (L == 4) hbad |= __shfl_xor_sync(0xffffffffu, hbad, 2);
        }
        __syncthreads();  // the products are in place
        double dmax = 0.0, zm = 0.0;
        int bad = 0;
        if (horner && valid && !im) {
            const V dr = vload<P>(pbuf, m, q), di = vload<P>(pbuf + K * m, m, q);
            V yr, yi, wr, wi;
            E gf;
            dk_finish<PU>(hr, hi, Eq, dr, di, pE[q], zr, zi, yr, yi, wr, wi, gf);
            if (gf.failed() || hbad || pbad[q]) {
                atomicAdd(&mp_dk_fallbacks, 1ull);
                dk_update_native<P>(i, n, c, cap, z, zc, zr, zi, yr, yi, wr, wi);
            }
            for (int r = 0; r < C; r++) {  // the new root into every CTA's next-iterate buffer
                double *dst = cluster.map_shared_rank(zn, r);
                vstore<P>(dst, zc, i, yr);
                vstore<P>(dst + K * zc, zc, i, yi);
            }
            const double d = __dadd_rn(fabs(wr.c[0]), fabs(wi.c[0]));
            const double mm = __dadd_rn(fabs(yr.c[0]), fabs(yi.c[0]));
            if (!(d == d) || isinf(d) || !(mm == mm) || isinf(mm)) bad = 1;
            dmax = d;
            zm = mm;
        }
        block_max2(sh, dmax, zm, bad);
        if (tid == 0) {
            const double stop = (A.watchdog > 0 && rank == 0 && (clock64() - t0) > A.watchdog) ? 1.0 : 0.0;
            for (int r = 0; r < C; r++) {
                double *dst = cluster.map_shared_rank(&slot[par][rank][0], r);
                dst[0] = sh.delta;
                dst[1] = sh.zmax;
                dst[2] = sh.bad ? 1.0 : 0.0;
                dst[3] = stop;
            }
        }
        cluster.sync();  // new iterate and every CTA's maxima visible everywhere
        double delta = 0.0, zmax = 0.0;
        bool anybad = false;
        for (int r = 0; r < C; r++) {
            delta = fmax(delta, slot[par][r][0]);
            zmax = fmax(zmax, slot[par][r][1]);
            anybad = anybad || slot[par][r][2] != 0.0;
        }
        const bool stop = slot[par][0][3] != 0.0;
        const double scale = zmax > 1.0 ? zmax : 1.0;
        if (anybad) { st = DK_BREAKDOWN; it = k; break; }
        if (delta <= __dmul_rn(A.tol, scale)) { st = DK_CONVERGED; it = k; break; }
        if (delta < best) { best = delta; since = 0; } else { since++; }
        if (k >= A.kmin && since >= A.win && best <= __dmul_rn(pow2(-26 * K), scale)) {
            st = DK_STAGNATED;
            it = k;
            break;
        }
        if (stop) { st = DK_TIMEOUT; it = k; break; }
    }
    // the newest iterate: the buffer the last sweep wrote (the start values when none ran)
    double *zf = zbuf[it < 1 ? 0 : (it & 1)];
    for (int64_t j = tid; j < cnt; j += blockDim.x)
        for (int cc = 0; cc < 2 * K; cc++) A.roots[cc * A.proots + ro + r0 + j] = zf[cc * zc + r0 + j];
    if (rank == 0 && tid == 0) {
        A.iters[b] = it;
        A.status[b] = st;
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// Descending-degree order (ties by index): order[rank(p)] = p.
__global__ void k_dk_order(int64_t npoly, const int64_t *__restrict__ coef_off, int32_t *__restrict__ order)
{
    __shared__ int64_t deg[1024];
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < npoly; p0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + threadIdx.x;
        const int64_t dp = p < npoly ? coef_off[p + 1] - coef_off[p] : 0;
        int64_t rank = 0;
        for (int64_t q0 = 0; q0 < npoly; q0 += blockDim.x) {
            __syncthreads();
            if (q0 + threadIdx.x < npoly)
                deg[threadIdx.x] = coef_off[q0 + threadIdx.x + 1] - coef_off[q0 + threadIdx.x];
            __syncthreads();
            const int64_t lim = npoly - q0 < blockDim.x ? npoly - q0 : blockDim.x;
            for (int64_t j = 0; j < lim; j++) {
                const int64_t dq = deg[j], q = q0 + j;
                rank += (dq > dp) || (dq == dp && q < p);
            }
        }
        if (p < npoly) order[rank] = (int32_t)p;
    }
}

template <class P>
__global__ void __launch_bounds__(256) k_dk_start(int64_t npoly, const int64_t *coef_off, const double *coef,
                                                  int64_t pcoef, double radius, int32_t max_degree, double *zout,
                                                  int64_t pz)
{
    // Same start as dk_solve (monic normalisation included), without iterating.
    extern __shared__ __align__(16) double dk_smem[];
    __shared__ DKShared sh;
    DKArgs<P> A{};
    A.npoly = npoly;
    A.coef_off = coef_off;
    A.coef = coef;
    A.pcoef = pcoef;
    A.z0 = nullptr;
    A.roots = zout;
    A.proots = pz;
    A.iters = nullptr;  // start values only: no per-polynomial statistics
    A.status = nullptr;
    A.max_iter = 0;
    A.tol = 1.0;
    A.win = 1;
    A.kmin = 1;
    A.radius = radius;
    A.watchdog = 0;
    A.max_degree = max_degree;
    A.order = nullptr;
    for (int64_t b = blockIdx.x; b < npoly; b += gridDim.x) dk_solve<P, NativeEngine<double>>(A, b, sh, dk_smem);
}

template <class P> static size_t dk_smem_bytes(int32_t max_degree)
{
    return (size_t)P::K * sizeof(double) * ((size_t)(max_degree + 1) + 2 * (size_t)max_degree);
}

constexpr size_t DK_SMEM_LIMIT = 227 * 1024 - 4096;  // leaves room for the static DKShared

template <class P> static int32_t dk_max_degree()
{
    return (int32_t)((DK_SMEM_LIMIT / (P::K * sizeof(double)) - 1) / 3);
}

static size_t dk_ws(int64_t npoly) { return 256 + (size_t)(npoly > 0 ? npoly : 0) * sizeof(int32_t); }

// Degrees above the shared-memory bound keep each block's coefficients and
// iterate in a slot of the workspace (after the queue and the order array).
// The persistent grid is capped at DK_GLOBAL_SLOTS_PER_SM blocks per SM.
constexpr int DK_GLOBAL_SLOTS_PER_SM = 4;
constexpr int32_t DK_GLOBAL_MAX_DEGREE = 1 << 20;

template <class P> static int64_t dk_slot_doubles(int32_t max_degree)
{
    return (int64_t)P::K * ((int64_t)max_degree + 1) + 2 * (int64_t)P::K * max_degree;
}

static size_t dk_slots_offset(int64_t npoly) { return (dk_ws(npoly) + 255) / 256 * 256; }

template <class P> static size_t dk_ws_deg(int64_t npoly, int32_t max_degree)
{
    if (max_degree <= dk_max_degree<P>()) return dk_ws(npoly);
    const int64_t slots = (int64_t)sm_count() * DK_GLOBAL_SLOTS_PER_SM;
    return dk_slots_offset(npoly) + (size_t)slots * (size_t)dk_slot_doubles<P>(max_degree) * sizeof(double);
}

// The persistent batched launch (mode 0) or one launch per polynomial (mode 1).
// Lanes per root of a cluster solve: four (one real product of each complex
// product per lane) while one CTA per 16 roots fits in a portable cluster, else
// two.  Cluster size: one CTA per 64 / lanes roots of the largest degree, at
// least 2, at most DK_CLUSTER_MAX (0 when the degree is too large).
static int dk_cluster_lanes(int32_t max_degree) { return max_degree <= 16 * DK_CLUSTER_MAX ? 4 : 2; }

static int dk_cluster_size(int32_t max_degree)
{
    const int per = 64 / dk_cluster_lanes(max_degree);
    const int c = (max_degree + per - 1) / per;
    if (c > DK_CLUSTER_MAX) return 0;
    return c < 2 ? 2 : c;
}

template <class P> static size_t dk_cluster_smem(int32_t max_degree, int C)
{
    const size_t m = ((size_t)max_degree + C - 1) / C;
    return sizeof(double) * ((size_t)P::K * (max_degree + 1) + 4 * (size_t)P::K * max_degree + 2 * (size_t)P::K * m) +
           m * (sizeof(long long) + sizeof(int)) + 16;
}

template <class P, class E>
static mp_status dk_run(const DKArgs<P> &A, const mp_roots_opts *o, int64_t npoly, int threads, size_t smem,
                        cudaStream_t st)
{
    if (o->mode == 2) {
        const int C = dk_cluster_size(o->max_degree);
        const int L = dk_cluster_lanes(o->max_degree);
        const size_t cs = dk_cluster_smem<P>(o->max_degree, C);
        if (C == 0 || npoly * C > 0x7fffffff) return MP_EINVAL;
        auto kern = L == 4 ? k_dk_cluster<P, E, 4> : k_dk_cluster<P, E, 2>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs);
        if (e != cudaSuccess) return cuda_status(e);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(npoly * C), 1, 1);
        cfg.blockDim = dim3(DK_CLUSTER_THREADS, 1, 1);
        cfg.dynamicSmemBytes = cs;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cuda_status(cudaLaunchKernelEx(&cfg, kern, A));
    }
    if (o->mode == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_dk_persistent<P, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
        int per_sm = o->blocks_per_sm;
        if (per_sm <= 0) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dk_persistent<P, E>, threads, smem);
            if (e != cudaSuccess) return cuda_status(e);
            if (per_sm < 1) per_sm = 1;
        }
        if (A.gscratch && per_sm > DK_GLOBAL_SLOTS_PER_SM) per_sm = DK_GLOBAL_SLOTS_PER_SM;
        int64_t grid = (int64_t)sm_count() * per_sm;
        if (grid > npoly) grid = npoly;
        e = cudaMemsetAsync(A.counter, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return cuda_status(e);
        k_dk_persistent<P, E><<<(unsigned)grid, threads, smem, st>>>(A);
        return launch_status();
    }
    cudaError_t e = cudaFuncSetAttribute(k_dk_single<P, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    for (int64_t p = 0; p < npoly; p++) {
        k_dk_single<P, E><<<1, threads, smem, st>>>(A, p);
        mp_status r = launch_status();
        if (r != MP_OK) return r;
    }
    return MP_OK;
}

template <class P>
static mp_status roots_launch(int64_t npoly, const int64_t *coef_off, const double *coef, int64_t pcoef,
                              const double *z0, int64_t pz0, double *roots, int64_t proots, int32_t *iters,
                              int32_t *status, const mp_roots_opts *o, void *ws, size_t ws_bytes, mp_stream s)
{
    if (npoly < 0 || o == nullptr) return MP_EINVAL;
    if (npoly == 0) return MP_OK;
    if (npoly > 0x7fffffff || coef_off == nullptr || coef == nullptr || roots == nullptr || iters == nullptr ||
        status == nullptr || pcoef < 1 || proots < 1 || (z0 && pz0 < 1))
        return MP_EINVAL;
    if (o->max_degree <= 0 || o->max_degree > DK_GLOBAL_MAX_DEGREE) return MP_EINVAL;
    const bool global = o->max_degree > dk_max_degree<P>();
    if (o->mode < 0 || o->mode > 2) return MP_EINVAL;
    if (o->mode == 2 && (dk_cluster_size(o->max_degree) == 0 || o->sort)) return MP_EINVAL;
    if (o->engine < 0 || o->engine > 2) return MP_EINVAL;
    const bool hybrid = o->engine != 2;  // 0 = automatic: the hybrid engine
    // Hybrid default: the smallest multiple of 64 threads that still splits every
    // sweep (two threads per root, so 2 x max_degree), at most 256.  Small blocks
    // let more of them share an SM: 4096 Chebyshev problems of degree 32 took
    // 0.79 s in 64-thread blocks against 1.30 s in 256-thread ones, degree 64
    // 6.13 s in 128-thread blocks against 6.71 s; same bits.
    const int64_t split_threads = (2 * (int64_t)o->max_degree + 63) / 64 * 64;
    const int hybrid_threads = split_threads < DKLaunch<DKHybrid>::default_threads
                                   ? (int)split_threads
                                   : DKLaunch<DKHybrid>::default_threads;
    const int threads = o->threads > 0 ? o->threads
                                       : (hybrid ? hybrid_threads : DKLaunch<NativeEngine<double>>::default_threads);
    if (threads % 32 != 0 || threads > 256) return MP_EINVAL;
    if (o->sort && npoly > (1 << 16)) return MP_EINVAL;
    if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 8 != 0) return MP_EINVAL;
    if (ws_bytes < dk_ws_deg<P>(npoly, o->max_degree)) return MP_ENOMEM;
    cudaStream_t st = as_stream(s);
    DKArgs<P> A{};
    A.npoly = npoly;
    A.coef_off = coef_off;
    A.coef = coef;
    A.pcoef = pcoef;
    A.z0 = z0;
    A.pz0 = pz0;
    A.roots = roots;
    A.proots = proots;
    A.iters = iters;
    A.status = status;
    A.tol = o->tol > 0 ? o->tol : ldexp(1.0, -(53 * P::K - 6));
    A.max_iter = o->max_iter > 0 ? o->max_iter : 1000;
    A.win = o->stag_window > 0 ? o->stag_window : 5;
    A.kmin = o->stag_min_iter > 0 ? o->stag_min_iter : 10;
    A.radius = o->radius;
    A.watchdog = o->watchdog_cycles;
    A.max_degree = o->max_degree;
    A.counter = static_cast<unsigned long long *>(ws);
    int32_t *order = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + 256);
    A.order = nullptr;
    A.gscratch = global ? reinterpret_cast<double *>(static_cast<char *>(ws) + dk_slots_offset(npoly)) : nullptr;
    A.gstride = global ? dk_slot_doubles<P>(o->max_degree) : 0;
    const size_t smem = global ? 0 : dk_smem_bytes<P>(o->max_degree);
    if (o->sort) {
        k_dk_order<<<grid_for(npoly, 256, 4), 256, 0, st>>>(npoly, coef_off, order);
        mp_status e = launch_status();
        if (e != MP_OK) return e;
        A.order = order;
    }
    return hybrid ? dk_run<P, DKHybrid>(A, o, npoly, threads, smem, st)
                  : dk_run<P, NativeEngine<double>>(A, o, npoly, threads, smem, st);
}

template <class P>
static mp_status roots_init_launch(int64_t npoly, const int64_t *coef_off, const double *coef, int64_t pcoef,
                                   double radius, int32_t max_degree, double *z, int64_t pz, mp_stream s)
{
    if (npoly < 0) return MP_EINVAL;
    if (npoly == 0) return MP_OK;
    if (coef_off == nullptr || coef == nullptr || z == nullptr || pcoef < 1 || pz < 1) return MP_EINVAL;
    if (max_degree <= 0 || max_degree > dk_max_degree<P>()) return MP_EINVAL;
    const size_t smem = dk_smem_bytes<P>(max_degree);
    cudaError_t e = cudaFuncSetAttribute(k_dk_start<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    k_dk_start<P><<<grid_for(npoly, 1, 4), 256, smem, as_stream(s)>>>(npoly, coef_off, coef, pcoef, radius,
                                                                      max_degree, z, pz);
    return launch_status();
}

}  // namespace mp

using namespace mp;

extern "C" {

#define MP_EXPORT_ROOTS(S, PT)                                                                        \
    size_t mp_roots_workspace_##S(int64_t npoly) { return dk_ws(npoly); }                             \
    size_t mp_roots_workspace_deg_##S(int64_t npoly, int32_t max_degree)                              \
    {                                                                                                 \
        if (npoly < 0 || max_degree <= 0 || max_degree > DK_GLOBAL_MAX_DEGREE) return 0;              \
        return dk_ws_deg<PT>(npoly, max_degree);                                                      \
    }                                                                                                 \
    int32_t mp_roots_max_degree_##S(void) { return dk_max_degree<PT>(); }                             \
    mp_status mp_roots_init_##S(int64_t npoly, const int64_t *coef_off, const double *coef,            \
                                int64_t pcoef, double radius, int32_t max_degree, double *z, int64_t pz, \
                                mp_stream s)                                                          \
    {                                                                                                 \
        return roots_init_launch<PT>(npoly, coef_off, coef, pcoef, radius, max_degree, z, pz, s);     \
    }                                                                                                 \
    mp_status mp_roots_##S(int64_t npoly, const int64_t *coef_off, const double *coef, int64_t pcoef,  \
                           const double *z0, int64_t pz0, double *roots, int64_t proots, int32_t *iters, \
                           int32_t *status, const mp_roots_opts *opts, void *ws, size_t ws_bytes,      \
                           mp_stream s)                                                               \
    {                                                                                                 \
        return roots_launch<PT>(npoly, coef_off, coef, pcoef, z0, pz0, roots, proots, iters, status,  \
                                opts, ws, ws_bytes, s);                                               \
    }

mp_status mp_roots_hybrid_fallbacks(unsigned long long *count)
{
    if (count == nullptr) return MP_EINVAL;
    return cuda_status(cudaMemcpyFromSymbol(count, mp_dk_fallbacks, sizeof(unsigned long long)));
}

MP_EXPORT_ROOTS(dd, P_dd)
MP_EXPORT_ROOTS(ddc, P_ddc)
MP_EXPORT_ROOTS(td, P_td)
MP_EXPORT_ROOTS(qd, P_qd)

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched roots for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or pass in a workspace: code running
// inside a pre-sized memory pool that must not grow, plugins and JIT hosts whose
// allocator is owned by someone else, or a real-time loop where an allocation
// could stall.  mp_roots_noalloc_qd gives them the QD Durand-Kerner solver with
// its workspace (the persistent queue's counter and the degree order) in a
// fixed array that the library itself holds in device memory.  It runs exactly
// the kernels of mp_roots_qd, so its results are the same bits.
//
// The array is 256 + 4 * MP_NOALLOC_MAX_POLYS bytes (64.25 KiB), allocated by
// the CUDA runtime when the library is loaded and held by every GPU that loads
// it until the process exits.  Calls share it: two calls whose kernels overlap
// on the GPU (different streams, or a later call enqueued before an earlier one
// finished on a stream that does not order them) race on it.  Of its contents
// only the queue counter must start at zero; the persistent launch clears it
// (cudaMemsetAsync on the call's stream) before every solve, and the order
// array is written before it is read in the same call.
// ---------------------------------------------------------------------------

// MP_NOALLOC_MAX_POLYS (16384 polynomials) is defined in mpgpu.h.
static __device__ __align__(256) unsigned char mp_roots_noalloc_scratch[256 + 4 * (size_t)MP_NOALLOC_MAX_POLYS];

namespace {

// Device address of mp_roots_noalloc_scratch, looked up once per device with
// that device current (host code cannot use the array's name as a device
// pointer).  Host threads may call concurrently: the lookup and the cache are
// guarded by a mutex.  The cache is not refreshed after cudaDeviceReset (which
// unloads the library's device code and may move the array): a process that
// resets a device must not call this entry point on that device again.
mp_status roots_noalloc_scratch(void **out)
{
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return MP_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, mp_roots_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        addr[dev] = p;
    }
    *out = addr[dev];
    return MP_OK;
}

}  // namespace

extern "C" mp_status mp_roots_noalloc_qd(int64_t npoly, const int64_t *coef_off, const double *coef, int64_t pcoef,
                                         const double *z0, int64_t pz0, double *roots, int64_t proots,
                                         int32_t *iters, int32_t *status, const mp_roots_opts *opts, mp_stream s)
{
    if (npoly < 0 || opts == nullptr) return MP_EINVAL;
    if (npoly > MP_NOALLOC_MAX_POLYS) return MP_ENOMEM;  // more order entries than the array holds
    // above the shared-memory bound the solver keeps per-block slots in its workspace
    if (opts->max_degree > dk_max_degree<P_qd>()) return MP_ENOMEM;
    if (npoly == 0) return MP_OK;
    void *ws = nullptr;
    mp_status st = roots_noalloc_scratch(&ws);
    if (st != MP_OK) return st;
    return roots_launch<P_qd>(npoly, coef_off, coef, pcoef, z0, pz0, roots, proots, iters, status, opts, ws,
                              sizeof(mp_roots_noalloc_scratch), s);
}
