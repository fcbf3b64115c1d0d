// k_poly.cu -- polynomial evaluation (Section 4.1), its adjoint, and the
// construction of polynomials from their roots, in multicomponent arithmetic.
//
// Evaluation: one thread per (polynomial, point), Horner's rule with the
// coefficients read as warp-uniform broadcasts.  Real arguments cost one
// multiply and one add per coefficient (209 FP64 instructions in QD), complex
// arguments four multiplies and three adds.
//
// Adjoint, dy -> (dcoef, dx):
//   dx: one thread per point, simultaneous Horner recurrence for p'.
//   dcoef_i = sum over points m (ascending) of dy_m x_m^i.  One warp per
//   polynomial; lane L takes the points L, L+32, ... in turn and runs each
//   point's powers dy_m x_m^i up the coefficients, while the partial sums S_i
//   travel along the lanes (register shuffles) and from lane 31 back to lane 0
//   through dcoef itself.  Each coefficient is folded over the points in
//   ascending order with the powers formed by repeated multiplication -- the
//   oracle's order, so the result is bit-identical.  No workspace.
//
// Polynomials from roots: one block per polynomial, the coefficient vector in
// shared memory, one factor (x - r) or (x^2 + Bx + C) per synchronised stage,
// all coefficients of a stage in parallel.
//
// Evaluation and dx run on FastEngine<P> (binary64: TwoSum's error term on the
// integer pipes); a point whose integer path left its domain is recomputed
// with the FP64 pipe, so every result is the FP64 sequence's bits.  The
// coefficient sweep runs on the hybrid engine that also packs subnormal error
// terms (see k_poly_dcoef); when any lane of the warp left its domain the whole
// polynomial is redone on the FP64 pipe, because the lanes pass partial sums to
// each other.
#include <cuda_runtime.h>

#include "mp_arith.cuh"
#include "mp_common.cuh"

namespace mp {

// ---------------------------------------------------------------------------
// Evaluation
// ---------------------------------------------------------------------------

template <class P, bool CPLX, class E>
__device__ __forceinline__ void horner_point(int64_t n, const typename P::T *__restrict__ cb, int64_t pc,
                                             const typename P::V &zr, const typename P::V &zi, typename P::V &hr,
                                             typename P::V &hi, E &g)
{
    using V = typename P::V;
    hr = vload<P>(cb, pc, n);
    hi = vzero<P>();
    if (!CPLX) {
        for (int64_t i = n - 1; i >= 0; i--) hr = P::add(P::mul(hr, zr, g), vload<P>(cb, pc, i), g);
    } else {
        for (int64_t i = n - 1; i >= 0; i--) {
            V t1 = P::mul(hr, zr, g);
            V t2 = P::mul(hi, zi, g);
            t1 = vsub<P>(t1, t2, g);
            t1 = P::add(t1, vload<P>(cb, pc, i), g);
            V t3 = P::mul(hr, zi, g);
            V t4 = P::mul(hi, zr, g);
            hi = P::add(t3, t4, g);
            hr = t1;
        }
    }
}

template <class P, bool CPLX>
__global__ void __launch_bounds__(256) k_polyeval(int64_t npoly, const int64_t *__restrict__ coef_off,
                                                  const typename P::T *__restrict__ coef, int64_t pc,
                                                  int64_t npts, const typename P::T *__restrict__ xr,
                                                  const typename P::T *__restrict__ xi, int64_t px,
                                                  typename P::T *__restrict__ yr,
                                                  typename P::T *__restrict__ yi, int64_t py)
{
    using V = typename P::V;
    const int64_t total = npoly * npts;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const int64_t b = idx / npts;
        const int64_t off = coef_off[b];
        const int64_t n = coef_off[b + 1] - off - 1;
        const typename P::T *cb = coef + off;
        if (n < 0) {
            vstore<P>(yr, py, idx, vzero<P>());
            if (CPLX) vstore<P>(yi, py, idx, vzero<P>());
            continue;
        }
        const V zr = vload<P>(xr, px, idx);
        const V zi = CPLX ? vload<P>(xi, px, idx) : vzero<P>();
        V hr, hi;
        FastEngine<P> g;
        horner_point<P, CPLX>(n, cb, pc, zr, zi, hr, hi, g);
        if (g.failed()) {
            NativeEngine<typename P::T> nat;
            horner_point<P, CPLX>(n, cb, pc, zr, zi, hr, hi, nat);
        }
        vstore<P>(yr, py, idx, hr);
        if (CPLX) vstore<P>(yi, py, idx, hi);
    }
}

template <class P>
static mp_status polyeval_launch(int64_t npoly, const int64_t *coef_off, const typename P::T *coef,
                                 int64_t pc, int64_t npts, const typename P::T *xr,
                                 const typename P::T *xi, int64_t px, typename P::T *yr,
                                 typename P::T *yi, int64_t py, mp_stream s)
{
    if (npoly < 0 || npts < 0) return MP_EINVAL;
    const int64_t total = npoly * npts;
    if (total == 0) return MP_OK;
    if (coef_off == nullptr || coef == nullptr || pc < 1 || !planes_ok(xr, total, px) ||
        !planes_ok(yr, total, py))
        return MP_EINVAL;
    if ((xi == nullptr) != (yi == nullptr)) return MP_EINVAL;
    const unsigned g = grid_for(total, 256, 8);
    if (xi)
        k_polyeval<P, true><<<g, 256, 0, as_stream(s)>>>(npoly, coef_off, coef, pc, npts, xr, xi, px, yr,
                                                         yi, py);
    else
        k_polyeval<P, false><<<g, 256, 0, as_stream(s)>>>(npoly, coef_off, coef, pc, npts, xr, xi, px, yr,
                                                          yi, py);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Estrin's scheme (Section 4.1 compares it with Horner's; the standard pairwise
// tree): level 0 holds a_0 .. a_n, each level replaces adjacent pairs (lo, hi)
// by add(mul(hi, y_k), lo) with y_0 = x and y_{k+1} = mul(y_k, y_k), an unpaired
// last value moves up unchanged.  One thread per point streams the coefficients
// in ascending order through a binary counter: a new value meets the pending
// value of each level whose bit is set, as the tree pairs them, and the values
// still pending at the end are combined from the lowest level up, the lower one
// as `hi` -- exactly the tree's pass-through rule.  Same operations, same
// order, same bits as the oracle's level-by-level form.  Pending values and
// powers live in per-thread (local) arrays; degrees up to 2^(ESTRIN_LEVELS-1)-1.
// ---------------------------------------------------------------------------

constexpr int ESTRIN_LEVELS = 26;

// (r, i) := (lo_r, lo_i) + (hi_r, hi_i) * (yr, yi), in the order of the 4M
// complex product of Horner's complex form; real arguments use only r.
template <class P, bool CPLX, class E>
__device__ __forceinline__ void estrin_combine(const typename P::V &hr, const typename P::V &hi,
                                               const typename P::V &lr, const typename P::V &li,
                                               const typename P::V &yr, const typename P::V &yi,
                                               typename P::V &rr, typename P::V &ri, E &g)
{
    using V = typename P::V;
    if (!CPLX) {
        rr = P::add(P::mul(hr, yr, g), lr, g);
        return;
    }
    V t1 = P::mul(hr, yr, g);
    V t2 = P::mul(hi, yi, g);
    t1 = vsub<P>(t1, t2, g);
    V t3 = P::mul(hr, yi, g);
    V t4 = P::mul(hi, yr, g);
    t3 = P::add(t3, t4, g);
    rr = P::add(t1, lr, g);
    ri = P::add(t3, li, g);
}

template <class P, bool CPLX, class E>
__device__ __forceinline__ void estrin_point(int64_t n, const typename P::T *__restrict__ cb, int64_t pc,
                                             const typename P::V &zr, const typename P::V &zi, typename P::V &outr,
                                             typename P::V &outi, E &g)
{
    using V = typename P::V;
    V pr[ESTRIN_LEVELS], pi[ESTRIN_LEVELS];  // pending value of each level
    V yr[ESTRIN_LEVELS], yi[ESTRIN_LEVELS];  // y_k = x^(2^k)
    int ny = 1;
    yr[0] = zr;
    yi[0] = CPLX ? zi : vzero<P>();
    auto power = [&](int lev) {
        while (ny <= lev) {
            const V a = yr[ny - 1], b = yi[ny - 1];
            if (!CPLX) {
                yr[ny] = P::mul(a, a, g);
            } else {
                V t1 = P::mul(a, a, g);
                V t2 = P::mul(b, b, g);
                t1 = vsub<P>(t1, t2, g);
                V t3 = P::mul(a, b, g);
                V t4 = P::mul(b, a, g);
                yi[ny] = P::add(t3, t4, g);
                yr[ny] = t1;
            }
            ny++;
        }
    };
    uint64_t cnt = 0;
    for (int64_t i = 0; i <= n; i++) {
        V cr = vload<P>(cb, pc, i), ci = vzero<P>();
        int lev = 0;
        while ((cnt >> lev) & 1) {  // pair with the pending value (the lower coefficients) of this level
            power(lev);
            V rr, ri;
            estrin_combine<P, CPLX>(cr, ci, pr[lev], pi[lev], yr[lev], yi[lev], rr, ri, g);
            cr = rr;
            ci = ri;
            lev++;
        }
        pr[lev] = cr;
        pi[lev] = ci;
        cnt++;
    }
    V cr = vzero<P>(), ci = vzero<P>();
    bool have = false;
    for (int lev = 0; lev < ESTRIN_LEVELS && (cnt >> lev) != 0; lev++) {
        if (!((cnt >> lev) & 1)) continue;
        if (!have) {
            cr = pr[lev];
            ci = pi[lev];
            have = true;
        } else {
            power(lev);
            V rr, ri;
            estrin_combine<P, CPLX>(cr, ci, pr[lev], pi[lev], yr[lev], yi[lev], rr, ri, g);
            cr = rr;
            ci = ri;
        }
    }
    outr = cr;
    outi = ci;
}

template <class P, bool CPLX>
__global__ void __launch_bounds__(256) k_polyeval_estrin(int64_t npoly, const int64_t *__restrict__ coef_off,
                                                         const typename P::T *__restrict__ coef, int64_t pc,
                                                         int64_t npts, const typename P::T *__restrict__ xr,
                                                         const typename P::T *__restrict__ xi, int64_t px,
                                                         typename P::T *__restrict__ yr,
                                                         typename P::T *__restrict__ yi, int64_t py)
{
    using V = typename P::V;
    const int64_t total = npoly * npts;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const int64_t b = idx / npts;
        const int64_t off = coef_off[b];
        const int64_t n = coef_off[b + 1] - off - 1;
        V hr = vzero<P>(), hi = vzero<P>();
        if (n >= ((int64_t)1 << (ESTRIN_LEVELS - 1))) {  // beyond the per-thread level arrays: NaN
            for (int c = 0; c < P::K; c++) hr.c[c] = hi.c[c] = (typename P::T)NAN;
        } else if (n >= 0) {
            const V zr = vload<P>(xr, px, idx);
            const V zi = CPLX ? vload<P>(xi, px, idx) : vzero<P>();
            // The powers x^(2^k) of points with |x| < 1 reach the bottom of the
            // binary64 range (x^256 for |x| < 0.1 in QD), so the hybrid engine
            // here also packs subnormal TwoSum error terms; with the default one
            // every such point was recomputed on the FP64 pipe by a few lanes of
            // its warp (ncu: 41% lane efficiency on the FP64 pipe, 2.9x Horner).
            typename std::conditional<P::fp64, HybridEngine<false, false, true>, NativeEngine<typename P::T>>::type g;
            estrin_point<P, CPLX>(n, coef + off, pc, zr, zi, hr, hi, g);
            if (g.failed()) {
                NativeEngine<typename P::T> nat;
                estrin_point<P, CPLX>(n, coef + off, pc, zr, zi, hr, hi, nat);
            }
        }
        vstore<P>(yr, py, idx, hr);
        if (CPLX) vstore<P>(yi, py, idx, hi);
    }
}

template <class P>
static mp_status polyeval_estrin_launch(int64_t npoly, const int64_t *coef_off, const typename P::T *coef,
                                        int64_t pc, int64_t npts, const typename P::T *xr, const typename P::T *xi,
                                        int64_t px, typename P::T *yr, typename P::T *yi, int64_t py, mp_stream s)
{
    if (npoly < 0 || npts < 0) return MP_EINVAL;
    const int64_t total = npoly * npts;
    if (total == 0) return MP_OK;
    if (coef_off == nullptr || coef == nullptr || pc < 1 || !planes_ok(xr, total, px) ||
        !planes_ok(yr, total, py))
        return MP_EINVAL;
    if ((xi == nullptr) != (yi == nullptr)) return MP_EINVAL;
    const unsigned gsz = grid_for(total, 256, 8);
    if (xi)
        k_polyeval_estrin<P, true><<<gsz, 256, 0, as_stream(s)>>>(npoly, coef_off, coef, pc, npts, xr, xi, px, yr,
                                                                   yi, py);
    else
        k_polyeval_estrin<P, false><<<gsz, 256, 0, as_stream(s)>>>(npoly, coef_off, coef, pc, npts, xr, xi, px, yr,
                                                                    yi, py);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------

// dy_m p'(x_m) by the simultaneous Horner recurrence for p and p'.
template <class P, class E>
__device__ __forceinline__ typename P::V dx_point(int64_t n, const typename P::T *__restrict__ cb, int64_t pc,
                                                  const typename P::V &xm, const typename P::V &dym, E &g)
{
    using V = typename P::V;
    V h = vload<P>(cb, pc, n);
    V d = vzero<P>();
    for (int64_t i = n - 1; i >= 0; i--) {
        d = P::add(P::mul(d, xm, g), h, g);
        h = P::add(P::mul(h, xm, g), vload<P>(cb, pc, i), g);
    }
    return P::mul(dym, d, g);
}

// dx of point idx (polynomial idx / npts).
template <class P>
__device__ __forceinline__ void dx_one(int64_t idx, int64_t npts, const int64_t *__restrict__ coef_off,
                                       const typename P::T *__restrict__ coef, int64_t pc,
                                       const typename P::T *__restrict__ x, int64_t px,
                                       const typename P::T *__restrict__ dy, int64_t pdy,
                                       typename P::T *__restrict__ dx, int64_t pdx)
{
    using V = typename P::V;
    const int64_t b = idx / npts;
    const int64_t off = coef_off[b];
    const int64_t n = coef_off[b + 1] - off - 1;
    if (n < 0) {
        vstore<P>(dx, pdx, idx, vzero<P>());
        return;
    }
    const typename P::T *cb = coef + off;
    const V xm = vload<P>(x, px, idx);
    const V dym = vload<P>(dy, pdy, idx);
    FastEngine<P> g;
    V r = dx_point<P>(n, cb, pc, xm, dym, g);
    if (g.failed()) {
        NativeEngine<typename P::T> nat;
        r = dx_point<P>(n, cb, pc, xm, dym, nat);
    }
    vstore<P>(dx, pdx, idx, r);
}

template <class P>
__global__ void __launch_bounds__(256) k_poly_dx(int64_t npoly, const int64_t *__restrict__ coef_off,
                                                 const typename P::T *__restrict__ coef, int64_t pc,
                                                 int64_t npts, const typename P::T *__restrict__ x,
                                                 int64_t px, const typename P::T *__restrict__ dy,
                                                 int64_t pdy, typename P::T *__restrict__ dx, int64_t pdx)
{
    const int64_t total = npoly * npts;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride)
        dx_one<P>(idx, npts, coef_off, coef, pc, x, px, dy, pdy, dx, pdx);
}

// Warps per block of the coefficient adjoint.  One warp per polynomial and one
// warp per block: with 1024 polynomials the block scheduler then spreads 6 or 7
// warps over each SM; four-warp blocks left some SMs twice the work of others
// (245 ms against 270 ms on 1024 polynomials x degree 256 x 4096 points).
constexpr int DCOEF_WARPS = 1;

// The coefficient adjoint of one polynomial (one warp).  Lane L takes the points
// m = 32g + L, g = 0, 1, ..., one after another, and spends Q = max(n + 1, 32)
// steps on each: at local step i <= n it adds w_i = dy_m x_m^i to S_i, the fold
// of w_i over the points before m, and forms w_{i+1} = w_i x_m (w_0 = dy_m).  That partial sum comes from lane L-1, which handled point
// m - 1 at the same local step one step earlier (a register shuffle); lane 0
// takes it from the group before, parked in dcoef_i by lane 31 Q - 31 >= 1
// steps earlier (and overwritten by lane 31 only 31 steps after the read).
// Points past npts pass the sum on unchanged, so lane 31's last write of each
// S_i is the whole fold.  Every coefficient is folded over the points in
// ascending order with the powers formed by repeated multiplication: the
// oracle's order and operations, so the result is bit-identical.  Returns true
// when any lane's engine failed; the caller then redoes the polynomial on the
// FP64 pipe (dy and x are never overwritten, and nothing is read from dcoef
// before it was written in the same sweep).
template <class P, class E>
__device__ __forceinline__ bool dcoef_ring(int64_t n, int64_t off, int64_t base, int64_t npts,
                                           const typename P::T *__restrict__ x, int64_t px,
                                           const typename P::T *__restrict__ dy, int64_t pdy,
                                           typename P::T *dcoef, int64_t pdc, E &g)
{
    using V = typename P::V;
    const int lane = threadIdx.x & 31;
    const int64_t Q = n + 1 > 32 ? n + 1 : 32;
    const int64_t groups = (npts + 31) / 32;
    const int64_t steps = groups * Q + 31;
    int64_t i = -lane;  // local step within the current point (negative: not started)
    int64_t m = lane;   // current point
    bool have = false;  // m < npts
    const V zero = vzero<P>();
    V w = zero, xm = zero, carry = zero;
    for (int64_t t = 0; t < steps; t++) {
        V s = carry;  // lane L-1's partial sum from the step before
        bool act = false;
        if (i >= 0) {
            if (i == 0) {
                have = m < npts;
                if (have) {
                    xm = vload<P>(x, px, base + m);
                    w = vload<P>(dy, pdy, base + m);  // w_0
                }
            }
            act = have && i <= n;
            if (lane == 0 && i <= n) {
                if (m < 32) {
                    s = zero;
                } else {
#pragma unroll
                    for (int c = 0; c < P::K; c++) s.c[c] = __ldcg(dcoef + c * pdc + off + i);
                }
            }
        }
        // S_i += w_i and w_{i+1} = w_i x_m are independent: both are issued
        // unconditionally (zero operands where a lane has nothing to do, so the
        // engine sees no spurious operands) and their instructions interleave.
        const bool nxt = act && i < n;
        const V sum = P::add(act ? s : zero, act ? w : zero, g);
        const V pw = P::mul(nxt ? w : zero, nxt ? xm : zero, g);
        if (act) s = sum;
        if (nxt) w = pw;
        if (lane == 31 && i >= 0 && i <= n) {
#pragma unroll
            for (int c = 0; c < P::K; c++) __stcg(dcoef + c * pdc + off + i, s.c[c]);
        }
        __syncwarp();  // orders lane 31's write before lane 0's read Q - 31 steps later
#pragma unroll
        for (int c = 0; c < P::K; c++) carry.c[c] = __shfl_up_sync(0xffffffffu, s.c[c], 1);
        if (++i == Q) {
            i = 0;
            m += 32;
        }
    }
    return __any_sync(0xffffffffu, g.failed());
}

// The coefficient adjoint of polynomial b (one whole warp).
template <class P>
__device__ __forceinline__ void dcoef_poly(int64_t b, int64_t npts, const int64_t *__restrict__ coef_off,
                                           const typename P::T *__restrict__ x, int64_t px,
                                           const typename P::T *__restrict__ dy, int64_t pdy,
                                           typename P::T *dcoef, int64_t pdc)
{
    const int lane = threadIdx.x & 31;
    const int64_t off = coef_off[b];
    const int64_t n = coef_off[b + 1] - off - 1;
    if (n < 0) return;
    if (npts == 0) {  // an empty fold
        for (int64_t i = lane; i <= n; i += 32) vstore<P>(dcoef, pdc, off + i, vzero<P>());
        return;
    }
    const int64_t base = b * npts;  // this polynomial's points
    // The sweep is bound by the FP64 pipe (one QD multiply and one add per
    // coefficient and point), so it runs on the hybrid engine for binary64
    // components, in the form that also packs subnormal error terms: the running
    // powers dy x^i of points with |x| < 1 fall through the bottom of the
    // binary64 range at high i, and with the default engine every polynomial
    // holding such a point restarted on the FP64 pipe.  Any other failure
    // restarts the polynomial there.
    typename std::conditional<P::fp64, HybridEngine<false, false, true>, NativeEngine<typename P::T>>::type g;
    if (dcoef_ring<P>(n, off, base, npts, x, px, dy, pdy, dcoef, pdc, g)) {
        NativeEngine<typename P::T> nat;
        dcoef_ring<P>(n, off, base, npts, x, px, dy, pdy, dcoef, pdc, nat);
    }
}

template <class P>
__global__ void __launch_bounds__(32 * DCOEF_WARPS)
    k_poly_dcoef(int64_t npoly, const int64_t *__restrict__ coef_off, int64_t npts,
                 const typename P::T *__restrict__ x, int64_t px, const typename P::T *__restrict__ dy,
                 int64_t pdy, typename P::T *dcoef, int64_t pdc)
{
    const int64_t b = (int64_t)blockIdx.x * DCOEF_WARPS + (threadIdx.x >> 5);
    if (b >= npoly) return;  // whole warp
    dcoef_poly<P>(b, npts, coef_off, x, px, dy, pdy, dcoef, pdc);
}

// The adjoint needs no workspace: the coefficient sweep parks its partial sums
// in dcoef itself.  The size query stays in the interface and answers 0.
template <class P> static size_t backward_ws(int64_t, int64_t) { return 0; }

template <class P>
static mp_status polyeval_backward_launch(int64_t npoly, const int64_t *coef_off, const typename P::T *coef,
                                          int64_t pc, int64_t npts, const typename P::T *x, int64_t px,
                                          const typename P::T *dy, int64_t pdy, typename P::T *dcoef,
                                          int64_t pdc, typename P::T *dx, int64_t pdx, void *ws,
                                          size_t ws_bytes, mp_stream s)
{
    if (npoly < 0 || npts < 0) return MP_EINVAL;
    const int64_t total = npoly * npts;
    if (npoly == 0) return MP_OK;
    if (coef_off == nullptr || coef == nullptr || pc < 1) return MP_EINVAL;
    if (total > 0 && (!planes_ok(x, total, px) || !planes_ok(dy, total, pdy))) return MP_EINVAL;
    // every argument check before the first launch: an error return enqueues nothing
    if (dx && total > 0 && pdx < total) return MP_EINVAL;
    if (dcoef && pdc < 1) return MP_EINVAL;
    (void)ws;  // no workspace needed (backward_ws)
    (void)ws_bytes;
    if (dx && total > 0) {
        k_poly_dx<P><<<grid_for(total, 256, 8), 256, 0, as_stream(s)>>>(npoly, coef_off, coef, pc, npts, x,
                                                                         px, dy, pdy, dx, pdx);
        mp_status st = launch_status();
        if (st != MP_OK) return st;
    }
    if (dcoef) {
        const int64_t blocks = (npoly + DCOEF_WARPS - 1) / DCOEF_WARPS;
        k_poly_dcoef<P><<<(unsigned)blocks, 32 * DCOEF_WARPS, 0, as_stream(s)>>>(npoly, coef_off, npts, x, px,
                                                                                 dy, pdy, dcoef, pdc);
        return launch_status();
    }
    return MP_OK;
}

// ---------------------------------------------------------------------------
// Polynomials from roots
// ---------------------------------------------------------------------------

constexpr int BUILD_THREADS = 128;

template <class P>
__global__ void __launch_bounds__(BUILD_THREADS)
    k_poly_from_roots(int64_t npoly, const int64_t *__restrict__ coef_off, const double *__restrict__ rootdata,
                      const double *__restrict__ delta, int32_t max_degree, typename P::T *__restrict__ coef,
                      int64_t pc)
{
    using T = typename P::T;
    using V = typename P::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t b = blockIdx.x;
    const int64_t off = coef_off[b];
    const int64_t n = coef_off[b + 1] - off - 1;
    if (n < 0 || n > max_degree) return;
    const int64_t cap = (int64_t)max_degree + 1;  // plane stride of the work vectors
    T *p = reinterpret_cast<T *>(smem_raw);
    T *q = p + P::K * cap;
    T *cq = q + P::K * cap;  // C of each quadratic factor, plane stride cap/2+1
    const int64_t pq = cap / 2 + 1;
    const double *rd = rootdata + (off - b);
    const double *dl = delta + (off - b);
    const int64_t npair = n / 2;
    for (int64_t k = threadIdx.x; k < npair; k += blockDim.x) {
        V re = vzero<P>(), im = vzero<P>();
        re.c[0] = rd[2 * k];
        im.c[0] = rd[2 * k + 1];
        vstore<P>(cq, pq, k, P::add(P::mul(re, re), P::mul(im, im)));
    }
    if (threadIdx.x == 0) vstore<P>(p, cap, 0, vone<P>());
    __syncthreads();
    int64_t d = 0;
    if (n % 2) {
        V r = vzero<P>();
        r.c[0] = rd[n - 1];
        for (int64_t i = threadIdx.x; i <= d + 1; i += blockDim.x) {
            V acc = i >= 1 ? vload<P>(p, cap, i - 1) : vzero<P>();
            if (i <= d) acc = P::add(acc, vneg<P>(P::mul(r, vload<P>(p, cap, i))));
            vstore<P>(q, cap, i, acc);
        }
        __syncthreads();
        T *t = p; p = q; q = t;
        d += 1;
    }
    for (int64_t k = 0; k < npair; k++) {
        V B = vzero<P>();
        B.c[0] = -2.0 * rd[2 * k];  // power-of-two scale: exact
        const V C = vload<P>(cq, pq, k);
        for (int64_t i = threadIdx.x; i <= d + 2; i += blockDim.x) {
            V acc = i >= 2 ? vload<P>(p, cap, i - 2) : vzero<P>();
            if (i >= 1 && i - 1 <= d) acc = P::add(acc, P::mul(B, vload<P>(p, cap, i - 1)));
            if (i <= d) acc = P::add(acc, P::mul(C, vload<P>(p, cap, i)));
            vstore<P>(q, cap, i, acc);
        }
        __syncthreads();
        T *t = p; p = q; q = t;
        d += 2;
    }
    for (int64_t i = threadIdx.x; i <= n; i += blockDim.x) {
        V a = vload<P>(p, cap, i);
        if (i < n) {
            V f = vone<P>();
            f.c[1] = dl[i];
            a = P::mul(a, f);
        }
        vstore<P>(coef + off, pc, i, a);
    }
}

constexpr int32_t BUILD_MAX_DEGREE = 2048;

template <class P>
static mp_status poly_from_roots_launch(int64_t npoly, const int64_t *coef_off, const double *rootdata,
                                        const double *delta, int32_t max_degree, typename P::T *coef,
                                        int64_t pc, mp_stream s)
{
    if (npoly < 0 || max_degree < 0 || max_degree > BUILD_MAX_DEGREE) return MP_EINVAL;
    if (npoly == 0) return MP_OK;
    if (coef_off == nullptr || coef == nullptr || pc < 1) return MP_EINVAL;
    if (max_degree > 0 && (rootdata == nullptr || delta == nullptr)) return MP_EINVAL;
    const int64_t cap = (int64_t)max_degree + 1;
    const size_t smem = (size_t)P::K * sizeof(typename P::T) * (2 * cap + cap / 2 + 1);
    if (npoly > 0x7fffffff) return MP_EINVAL;
    cudaError_t e = cudaFuncSetAttribute(k_poly_from_roots<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    k_poly_from_roots<P><<<(unsigned)npoly, BUILD_THREADS, smem, as_stream(s)>>>(npoly, coef_off, rootdata,
                                                                                  delta, max_degree, coef, pc);
    return launch_status();
}

}  // namespace mp

using namespace mp;

extern "C" {

#define MP_EXPORT_POLY(S, PT)                                                                       \
    mp_status mp_polyeval_##S(int64_t npoly, const int64_t *coef_off, const PT::T *coef,           \
                              int64_t pcoef, int64_t npts, const PT::T *x_re, const PT::T *x_im,    \
                              int64_t px, PT::T *y_re, PT::T *y_im, int64_t py, mp_stream s)       \
    {                                                                                               \
        return polyeval_launch<PT>(npoly, coef_off, coef, pcoef, npts, x_re, x_im, px, y_re, y_im, \
                                   py, s);                                                          \
    }                                                                                               \
    mp_status mp_polyeval_estrin_##S(int64_t npoly, const int64_t *coef_off, const PT::T *coef,    \
                                     int64_t pcoef, int64_t npts, const PT::T *x_re,                \
                                     const PT::T *x_im, int64_t px, PT::T *y_re, PT::T *y_im,       \
                                     int64_t py, mp_stream s)                                       \
    {                                                                                               \
        return polyeval_estrin_launch<PT>(npoly, coef_off, coef, pcoef, npts, x_re, x_im, px, y_re, \
                                          y_im, py, s);                                             \
    }                                                                                               \
    size_t mp_polyeval_backward_workspace_##S(int64_t npoly, int64_t npts)                          \
    {                                                                                               \
        return backward_ws<PT>(npoly, npts);                                                        \
    }                                                                                               \
    mp_status mp_polyeval_backward_##S(int64_t npoly, const int64_t *coef_off, const PT::T *coef,  \
                                       int64_t pcoef, int64_t npts, const PT::T *x, int64_t px,     \
                                       const PT::T *dy, int64_t pdy, PT::T *dcoef, int64_t pdc,     \
                                       PT::T *dx, int64_t pdx, void *ws, size_t ws_bytes,           \
                                       mp_stream s)                                                 \
    {                                                                                               \
        return polyeval_backward_launch<PT>(npoly, coef_off, coef, pcoef, npts, x, px, dy, pdy,     \
                                            dcoef, pdc, dx, pdx, ws, ws_bytes, s);                  \
    }

MP_EXPORT_POLY(dd, P_dd)
MP_EXPORT_POLY(ddc, P_ddc)
MP_EXPORT_POLY(td, P_td)
MP_EXPORT_POLY(qd, P_qd)
MP_EXPORT_POLY(ds, P_ds)
MP_EXPORT_POLY(tf, P_tf)
MP_EXPORT_POLY(qf, P_qf)

#define MP_EXPORT_BUILD(S, PT)                                                                      \
    mp_status mp_poly_from_roots_##S(int64_t npoly, const int64_t *coef_off, const double *rootdata, \
                                     const double *delta, int32_t max_degree, double *coef,          \
                                     int64_t pcoef, mp_stream s)                                     \
    {                                                                                               \
        return poly_from_roots_launch<PT>(npoly, coef_off, rootdata, delta, max_degree, coef, pcoef, \
                                          s);                                                       \
    }

MP_EXPORT_BUILD(dd, P_dd)
MP_EXPORT_BUILD(ddc, P_ddc)
MP_EXPORT_BUILD(td, P_td)
MP_EXPORT_BUILD(qd, P_qd)

}  // extern "C"
