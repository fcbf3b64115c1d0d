// k_blas1.cu -- elementwise add/multiply/reciprocal, AXPY, dot and GEMV over
// K-arrays (component planes), plus the library's status helpers and the
// FP64/FP32 pipe-peak microbenchmark.
//
// All arithmetic is the branch-free multicomponent arithmetic of mp_arith.cuh
// (Section 2, Algorithms 1-14).  These kernels are FP64-pipe bound for the
// binary64 precisions (one QD multiply-add is 209 FP64 instructions against
// 96 bytes of AXPY traffic), so each thread simply takes one element per
// grid-stride step; loads of each plane are coalesced across the warp.  The
// add, multiply, AXPY, dot and GEMV folds run on FastEngine<P> (binary64: the
// hybrid engine, TwoSum's error term on the integer pipes); an element or a
// thread's partial sum whose integer path left its domain is recomputed with
// the FP64 pipe, so every result is the FP64 sequence's bits.
#include <cuda_runtime.h>

#include <cstdio>

#include "mp_arith.cuh"
#include "mp_common.cuh"

namespace mp {

int &last_cuda_error()
{
    static thread_local int e = 0;
    return e;
}

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 1;
        cached[dev] = v;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// Elementwise
// ---------------------------------------------------------------------------

enum { EW_ADD = 0, EW_MUL = 1, EW_RECIP = 2 };

template <class P, int OP>
__global__ void __launch_bounds__(256) k_elementwise(int64_t n, const typename P::T *__restrict__ a,
                                                     int64_t pa, const typename P::T *__restrict__ b,
                                                     int64_t pb, typename P::T *__restrict__ c,
                                                     int64_t pc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        typename P::V x = vload<P>(a, pa, i);
        typename P::V z;
        if (OP == EW_RECIP) {
            z = vrecip<P>(x);
        } else {
            typename P::V y = vload<P>(b, pb, i);
            FastEngine<P> g;
            z = OP == EW_ADD ? P::add(x, y, g) : P::mul(x, y, g);
            if (g.failed()) z = OP == EW_ADD ? P::add(x, y) : P::mul(x, y);
        }
        vstore<P>(c, pc, i, z);
    }
}

template <class P, int OP>
static mp_status ew_launch(int64_t n, const typename P::T *a, int64_t pa, const typename P::T *b,
                           int64_t pb, typename P::T *c, int64_t pc, mp_stream s)
{
    if (n < 0 || !planes_ok(a, n, pa) || !planes_ok(c, n, pc)) return MP_EINVAL;
    if (OP != EW_RECIP && !planes_ok(b, n, pb)) return MP_EINVAL;
    if (n == 0) return MP_OK;
    k_elementwise<P, OP><<<grid_for(n, 256, 8), 256, 0, as_stream(s)>>>(n, a, pa, b, pb, c, pc);
    return launch_status();
}

// ---------------------------------------------------------------------------
// AXPY: y_i = add(mul(alpha, x_i), y_i)
// ---------------------------------------------------------------------------

// At least 2 (QD), 3 (three components) or 4 (two) blocks of 256 threads per SM.
template <class P>
__global__ void __launch_bounds__(256, P::K == 4 ? 2 : (P::K == 3 ? 3 : 4)) k_axpy(int64_t n, typename P::V alpha,
                                              const typename P::T *__restrict__ x, int64_t px,
                                              typename P::T *__restrict__ y, int64_t py)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        typename P::V xi = vload<P>(x, px, i);
        typename P::V yi = vload<P>(y, py, i);
        FastEngine<P> g;
        typename P::V r = P::add(P::mul(alpha, xi, g), yi, g);
        if (g.failed()) r = P::add(P::mul(alpha, xi), yi);
        vstore<P>(y, py, i, r);
    }
}

template <class P>
static mp_status axpy_launch(int64_t n, const typename P::T *alpha, const typename P::T *x,
                             int64_t px, typename P::T *y, int64_t py, mp_stream s)
{
    if (n < 0 || alpha == nullptr || !planes_ok(x, n, px) || !planes_ok(y, n, py)) return MP_EINVAL;
    if (n == 0) return MP_OK;
    typename P::V a;
    for (int c = 0; c < P::K; c++) a.c[c] = alpha[c];
    k_axpy<P><<<grid_for(n, 256, 8), 256, 0, as_stream(s)>>>(n, a, x, px, y, py);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Reductions: warp shuffle tree and block tree with the multicomponent add.
// ---------------------------------------------------------------------------

template <class P> __device__ __forceinline__ typename P::V warp_reduce(typename P::V v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        typename P::V o;
#pragma unroll
        for (int c = 0; c < P::K; c++) o.c[c] = __shfl_down_sync(0xffffffffu, v.c[c], off);
        v = P::add(v, o);
    }
    return v;  // valid in lane 0
}

// Block of `nthreads` (multiple of 32, <= 1024): returns the total in thread 0.
template <class P> __device__ __forceinline__ typename P::V block_reduce(typename P::V v)
{
    __shared__ typename P::T red[P::K][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    v = warp_reduce<P>(v);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < P::K; c++) red[c][warp] = v.c[c];
    __syncthreads();
    if (warp == 0) {
        typename P::V w = vzero<P>();
        if (lane < nwarp)
#pragma unroll
            for (int c = 0; c < P::K; c++) w.c[c] = red[c][lane];
        w = warp_reduce<P>(w);
        v = w;
    }
    return v;
}

constexpr int DOT_THREADS = 256;

template <class P>
__global__ void __launch_bounds__(DOT_THREADS) k_dot_partial(int64_t n, const typename P::T *__restrict__ x,
                                                             int64_t px, const typename P::T *__restrict__ y,
                                                             int64_t py, typename P::T *__restrict__ part);

// One full wave of resident blocks (SMs x blocks per SM), so every block folds the
// same number of elements and no partial last wave idles the FP64 pipe.  The count
// depends only on the device, so results are reproducible on a given GPU model.
template <class P> static int64_t dot_blocks(int64_t n)
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dot_partial<P>, DOT_THREADS, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        cached[dev] = sm_count() * per_sm;
    }
    int64_t g = (n + DOT_THREADS - 1) / DOT_THREADS;
    if (g > cached[dev]) g = cached[dev];
    return g < 1 ? 1 : g;
}

// A thread's share of the dot: elements i0, i0 + stride, ...  Binary64 components
// (FP64-pipe bound) fold them into one accumulator; binary32 components, whose
// FP32 pipe is fast enough for the add chain's latency to show, fold them
// round-robin into DOT_ACC accumulators combined in order at the end -- a fixed
// order, so the result is still deterministic and within the same bound.
constexpr int DOT_ACC = 4;

template <class P, class E>
__device__ __forceinline__ typename P::V dot_fold(int64_t n, const typename P::T *__restrict__ x, int64_t px,
                                                  const typename P::T *__restrict__ y, int64_t py, int64_t i0,
                                                  int64_t stride, E &g)
{
    using V = typename P::V;
    constexpr int NA = P::fp64 ? 1 : DOT_ACC;
    V acc[NA];
#pragma unroll
    for (int a = 0; a < NA; a++) acc[a] = vzero<P>();
    int64_t i = i0;
    for (; i + (NA - 1) * stride < n; i += NA * stride)
#pragma unroll
        for (int a = 0; a < NA; a++)
            acc[a] = P::add(acc[a], P::mul(vload<P>(x, px, i + a * stride), vload<P>(y, py, i + a * stride), g), g);
    for (int a = 0; i < n; i += stride, a++)
        acc[a] = P::add(acc[a], P::mul(vload<P>(x, px, i), vload<P>(y, py, i), g), g);
#pragma unroll
    for (int a = 1; a < NA; a++) acc[0] = P::add(acc[0], acc[a], g);
    return acc[0];
}

template <class P>
__global__ void __launch_bounds__(DOT_THREADS) k_dot_partial(int64_t n, const typename P::T *__restrict__ x,
                                                             int64_t px, const typename P::T *__restrict__ y,
                                                             int64_t py, typename P::T *__restrict__ part)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    FastEngine<P> g;
    typename P::V acc = dot_fold<P>(n, x, px, y, py, i0, stride, g);
    if (g.failed()) {  // the thread's fold again on the FP64 pipe
        NativeEngine<typename P::T> nat;
        acc = dot_fold<P>(n, x, px, y, py, i0, stride, nat);
    }
    acc = block_reduce<P>(acc);
    if (threadIdx.x == 0) vstore<P>(part, gridDim.x, blockIdx.x, acc);
}

template <class P>
__global__ void __launch_bounds__(DOT_THREADS) k_dot_final(int64_t g, const typename P::T *__restrict__ part,
                                                           typename P::T *__restrict__ out)
{
    typename P::V acc = vzero<P>();
    for (int64_t i = threadIdx.x; i < g; i += blockDim.x) acc = P::add(acc, vload<P>(part, g, i));
    acc = block_reduce<P>(acc);
    if (threadIdx.x == 0) vstore<P>(out, 1, 0, acc);
}

template <class P> static size_t dot_ws(int64_t n)
{
    return (size_t)dot_blocks<P>(n < 0 ? 0 : n) * P::K * sizeof(typename P::T);
}

template <class P>
static mp_status dot_launch(int64_t n, const typename P::T *x, int64_t px, const typename P::T *y,
                            int64_t py, typename P::T *result, void *ws, size_t ws_bytes, mp_stream s)
{
    if (n < 0 || result == nullptr || !planes_ok(x, n, px) || !planes_ok(y, n, py) || ws == nullptr)
        return MP_EINVAL;
    if (ws_bytes < dot_ws<P>(n)) return MP_ENOMEM;
    int64_t g = dot_blocks<P>(n);
    auto *part = static_cast<typename P::T *>(ws);
    k_dot_partial<P><<<(unsigned)g, DOT_THREADS, 0, as_stream(s)>>>(n, x, px, y, py, part);
    mp_status st = launch_status();
    if (st != MP_OK) return st;
    k_dot_final<P><<<1, DOT_THREADS, 0, as_stream(s)>>>(g, part, result);
    return launch_status();
}

// ---------------------------------------------------------------------------
// GEMV: one warp per row for short rows, one 256-thread block per row for long
// ones (many more, smaller work units than resident warps, so no tail wave)
// ---------------------------------------------------------------------------

template <class P>
__global__ void __launch_bounds__(256) k_gemv(int64_t m, int64_t n, const typename P::T *__restrict__ A,
                                              int64_t lda, int64_t pA, const typename P::T *__restrict__ x,
                                              int64_t px, typename P::T *__restrict__ y, int64_t py, int per_row)
{
    // per_row threads fold one row; blockDim / per_row rows per block
    const int t = threadIdx.x % per_row;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / per_row) + threadIdx.x / per_row;
    typename P::V acc = vzero<P>();
    if (row < m) {
        const typename P::T *Ar = A + row * lda;
        FastEngine<P> g;
        for (int64_t j = t; j < n; j += per_row)
            acc = P::add(acc, P::mul(vload<P>(Ar, pA, j), vload<P>(x, px, j), g), g);
        if (g.failed()) {  // the thread's fold again on the FP64 pipe
            acc = vzero<P>();
            for (int64_t j = t; j < n; j += per_row)
                acc = P::add(acc, P::mul(vload<P>(Ar, pA, j), vload<P>(x, px, j)));
        }
    }
    acc = warp_reduce<P>(acc);
    if (per_row > 32) {  // combine the row's warps (per_row / 32 of them) in shared memory
        __shared__ typename P::T red[P::K][8];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < P::K; c++) red[c][warp] = acc.c[c];
        __syncthreads();
        if (t == 0) {
            const int w0 = warp;  // first warp of this row
            typename P::V s = vload<P>(&red[0][0], 8, w0);
            for (int w = 1; w < per_row / 32; w++) s = P::add(s, vload<P>(&red[0][0], 8, w0 + w));
            acc = s;
        }
    }
    if (t == 0 && row < m) vstore<P>(y, py, row, acc);
}

// Threads per row: the smallest of 32, 64, 128, 256 that gives at least 8 full
// waves of warps (so the last, partial wave costs little), as long as each thread
// still folds at least 16 columns (so the reduction tree stays cheap).
static int gemv_threads_per_row(int64_t m, int64_t n)
{
    const int64_t resident_warps = (int64_t)sm_count() * 24;  // 3 blocks of 8 warps per SM
    int t = 32;
    while (t < 256 && m * (t / 32) < 8 * resident_warps && n / (2 * t) >= 16) t *= 2;
    return t;
}

template <class P>
static mp_status gemv_launch(int64_t m, int64_t n, const typename P::T *A, int64_t lda, int64_t pA,
                             const typename P::T *x, int64_t px, typename P::T *y, int64_t py,
                             mp_stream s)
{
    if (m < 0 || n < 0 || lda < n || !planes_ok(y, m, py) || !planes_ok(x, n, px)) return MP_EINVAL;
    if (m > 0 && n > 0 && (A == nullptr || pA < (m - 1) * lda + n)) return MP_EINVAL;
    if (m == 0) return MP_OK;
    const int per_row = gemv_threads_per_row(m, n);
    const int64_t blocks = (m + (256 / per_row) - 1) / (256 / per_row);
    if (blocks > 0x7fffffff) return MP_EINVAL;
    k_gemv<P><<<(unsigned)blocks, 256, 0, as_stream(s)>>>(m, n, A, lda, pA, x, px, y, py, per_row);
    return launch_status();
}

// ---------------------------------------------------------------------------
// Pipe-peak microbenchmark: 8 independent chains per thread.
// ---------------------------------------------------------------------------

// Packed binary32 pairs (sm_100+ PTX): two lanes per instruction.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm volatile("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <int KIND>
__global__ void k_peak(int64_t iters, double *sink)
{
    if (KIND == 11) {  // DFMA with one active lane per warp: the FP64 pipe's cost per warp instruction
        if ((threadIdx.x & 31) != 0) return;
        double a[8];
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = 1.0 + 1e-9 * (threadIdx.x + 8 * j);
        for (int64_t it = 0; it < iters; it++)
#pragma unroll
            for (int j = 0; j < 8; j++) a[j] = __fma_rn(a[j], 0.999999999, 1e-12);
        double s = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) s += a[j];
        if (s == 1234.5) sink[0] = s;
    } else if (KIND >= 7) {  // integer pipes; inline PTX so the chains cannot be folded
        unsigned a[8];
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = threadIdx.x * 7u + (unsigned)j;
        const unsigned b = 0x12345u, cc = 0x9abcu;
        for (int64_t it = 0; it < iters; it++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (KIND == 7) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(cc));
                if (KIND == 8) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(cc));
                if (KIND == 9) {
                    if (j & 1) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[j]) : "r"(b));
                    else asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(cc));
                }
                if (KIND == 10) asm volatile("{.reg .u32 t; clz.b32 t, %0; add.u32 %0, %0, t;}" : "+r"(a[j]));
            }
        }
        unsigned s = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) s ^= a[j];
        if (s == 0x7777777u) sink[0] = (double)s;
    } else if (KIND >= 5) {
        unsigned long long a[8];
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = 0x3f8000003f800000ULL + threadIdx.x + j;  // ~(1.0f, 1.0f)
        const unsigned long long b = 0x3f7fffff3f7fffffULL, cc = 0x2edbe6ff2edbe6ffULL;
        for (int64_t it = 0; it < iters; it++) {
#pragma unroll
            for (int j = 0; j < 8; j++) a[j] = KIND == 5 ? ffma2(a[j], b, cc) : fadd2(a[j], cc);
        }
        unsigned long long s = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) s ^= a[j];
        if (s == 12345ULL) sink[0] = (double)s;
    } else if (KIND <= 2) {
        double a[8];
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = 1.0 + 1e-9 * (threadIdx.x + 8 * j);
        const double b = 0.999999999, cc = 1e-12;
        for (int64_t it = 0; it < iters; it++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (KIND == 0) a[j] = __fma_rn(a[j], b, cc);
                if (KIND == 1) a[j] = __dadd_rn(a[j], cc);
                if (KIND == 2) a[j] = __dmul_rn(a[j], b);
            }
        }
        double s = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) s += a[j];
        if (s == 1234.5) sink[0] = s;
    } else {
        float a[8];
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = 1.0f + 1e-6f * (threadIdx.x + 8 * j);
        const float b = 0.9999999f, cc = 1e-9f;
        for (int64_t it = 0; it < iters; it++) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (KIND == 3) a[j] = __fmaf_rn(a[j], b, cc);
                if (KIND == 4) a[j] = __fadd_rn(a[j], cc);
            }
        }
        float s = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) s += a[j];
        if (s == 1234.5f) sink[0] = s;
    }
}

}  // namespace mp

using namespace mp;

extern "C" {

const char *mp_status_str(mp_status s)
{
    switch (s) {
    case MP_OK: return "ok";
    case MP_EINVAL: return "invalid argument";
    case MP_ECUDA: return "CUDA error";
    case MP_ENOMEM: return "workspace too small";
    case MP_ETIMEOUT: return "watchdog expired";
    case MP_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

int mp_last_cuda_error(void) { return last_cuda_error(); }

const char *mp_version(void) { return "mpgpu 0.1 (sm_103a)"; }

int mp_sm_count(void) { return sm_count(); }

mp_status mp_peak_run(int kind, int64_t iters, int blocks, int threads, float *ms, double *lane_ops,
                      mp_stream stream)
{
    if (kind < 0 || kind > 11 || iters <= 0 || blocks <= 0 || threads <= 0 || threads > 1024 ||
        ms == nullptr || lane_ops == nullptr)
        return MP_EINVAL;
    cudaStream_t s = as_stream(stream);
    cudaEvent_t e0, e1;
    mp_status st = cuda_status(cudaEventCreate(&e0));
    if (st != MP_OK) return st;
    st = cuda_status(cudaEventCreate(&e1));
    if (st != MP_OK) {
        cudaEventDestroy(e0);
        return st;
    }
    cudaEventRecord(e0, s);
    switch (kind) {
    case 0: k_peak<0><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 1: k_peak<1><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 2: k_peak<2><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 3: k_peak<3><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 4: k_peak<4><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 5: k_peak<5><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 6: k_peak<6><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 7: k_peak<7><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 8: k_peak<8><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 9: k_peak<9><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    case 10: k_peak<10><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    default: k_peak<11><<<blocks, threads, 0, s>>>(iters, nullptr); break;
    }
    st = launch_status();
    cudaEventRecord(e1, s);
    if (st == MP_OK) st = cuda_status(cudaEventSynchronize(e1));
    if (st == MP_OK) st = cuda_status(cudaEventElapsedTime(ms, e0, e1));
    *lane_ops = kind == 11 ? (double)blocks * ((threads + 31) / 32) * (double)iters * 8.0
                           : (double)blocks * threads * (double)iters * 8.0 *
                                 ((kind == 5 || kind == 6 || kind == 10) ? 2.0 : 1.0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

#define MP_EXPORT_BLAS1(S, PT)                                                                   \
    mp_status mp_add_##S(int64_t n, const PT::T *a, int64_t pa, const PT::T *b, int64_t pb,     \
                         PT::T *c, int64_t pc, mp_stream s)                                     \
    {                                                                                            \
        return ew_launch<PT, EW_ADD>(n, a, pa, b, pb, c, pc, s);                                 \
    }                                                                                            \
    mp_status mp_mul_##S(int64_t n, const PT::T *a, int64_t pa, const PT::T *b, int64_t pb,     \
                         PT::T *c, int64_t pc, mp_stream s)                                     \
    {                                                                                            \
        return ew_launch<PT, EW_MUL>(n, a, pa, b, pb, c, pc, s);                                 \
    }                                                                                            \
    mp_status mp_recip_##S(int64_t n, const PT::T *a, int64_t pa, PT::T *c, int64_t pc,         \
                           mp_stream s)                                                         \
    {                                                                                            \
        return ew_launch<PT, EW_RECIP>(n, a, pa, nullptr, 0, c, pc, s);                          \
    }                                                                                            \
    mp_status mp_axpy_##S(int64_t n, const PT::T *alpha, const PT::T *x, int64_t px, PT::T *y,  \
                          int64_t py, mp_stream s)                                              \
    {                                                                                            \
        return axpy_launch<PT>(n, alpha, x, px, y, py, s);                                       \
    }                                                                                            \
    size_t mp_dot_workspace_##S(int64_t n) { return dot_ws<PT>(n); }                             \
    mp_status mp_dot_##S(int64_t n, const PT::T *x, int64_t px, const PT::T *y, int64_t py,     \
                         PT::T *result, void *ws, size_t ws_bytes, mp_stream s)                 \
    {                                                                                            \
        return dot_launch<PT>(n, x, px, y, py, result, ws, ws_bytes, s);                         \
    }                                                                                            \
    mp_status mp_gemv_##S(int64_t m, int64_t n, const PT::T *A, int64_t lda, int64_t pA,        \
                          const PT::T *x, int64_t px, PT::T *y, int64_t py, mp_stream s)        \
    {                                                                                            \
        return gemv_launch<PT>(m, n, A, lda, pA, x, px, y, py, s);                               \
    }

MP_EXPORT_BLAS1(dd, P_dd)
MP_EXPORT_BLAS1(ddc, P_ddc)
MP_EXPORT_BLAS1(td, P_td)
MP_EXPORT_BLAS1(qd, P_qd)
MP_EXPORT_BLAS1(tdc, P_tdc)
MP_EXPORT_BLAS1(qdc, P_qdc)
MP_EXPORT_BLAS1(ds, P_ds)
MP_EXPORT_BLAS1(tf, P_tf)
MP_EXPORT_BLAS1(qf, P_qf)

}  // extern "C"
