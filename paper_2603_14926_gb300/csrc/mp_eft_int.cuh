// mp_eft_int.cuh -- the error term of TwoSum (Algorithm 2) computed exactly on the
// integer pipes, for binary64.
//
// TwoSum returns s = fl(a + b) and e = a + b - s, which is exactly representable
// (Section 2, Algorithms 1-2).  On this GPU the FP64 pipe retires about 2 lanes per
// clock per SM while the integer ALU and FMA pipes retire 64 each, so instead of
// the five further FP64 operations of Algorithm 2 the engine takes s from one FP64
// add and evaluates e = a + b - s in integer arithmetic:
//
//   every finite binary64 x with biased exponent E and fraction f is m * 2^(E' - 1075)
//   with E' = max(E, 1) and m = f + 2^52 [E > 0] (IEEE 754 binary64 encoding), so
//
//   e * 2^(1075 - u) = ma 2^(Ea' - u) + mb 2^(Eb' - u) - ms 2^(Es' - u),  u = min(Ea', Eb', Es'),
//
// with signs applied.  |e| <= ulp(s)/2 and e is a multiple of the smallest unit in
// play, so the right-hand side is an integer below 2^55 in magnitude: it can be
// evaluated modulo 2^64 (terms shifted by 64 or more vanish) and read back as a
// signed 64-bit value, then normalised and packed.  The result is bit-identical to
// the FP64 sequence of Algorithm 2 (+0 when the sum is exact) whenever
//   - a and b are finite with biased exponent <= 2045 (no intermediate of
//     Algorithm 2 can overflow), and
//   - e is zero or normal.
// Outside that domain the function raises `bad`; callers then recompute the whole
// result with the FP64 pipe, so every output stays exactly the paper's operation
// sequence.  A variant (SUBNORMAL) also packs a subnormal e exactly, for callers
// whose values reach the bottom of the binary64 range.
//
// The functions are also compiled for the host, where a unit test checks them
// against the host's binary64 arithmetic.
#pragma once
#include <cstdint>

#define MP_HD __host__ __device__ __forceinline__

namespace mp {
namespace eft_int {

MP_HD uint32_t lo32(uint64_t x) { return (uint32_t)x; }
MP_HD uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }
MP_HD uint64_t mk64(uint32_t h, uint32_t l) { return ((uint64_t)h << 32) | l; }
MP_HD int imin(int a, int b) { return a < b ? a : b; }

// 1 << k as a 32-bit word, 0 when k >= 32 (PTX clamps the shift count).
MP_HD uint32_t pow2_32(uint32_t k)
{
#ifdef __CUDA_ARCH__
    uint32_t r;
    asm("shl.b32 %0, 1, %1;" : "=r"(r) : "r"(k));
    return r;
#else
    return k < 32 ? 1u << k : 0u;
#endif
}

MP_HD int clz64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

MP_HD int clz32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

MP_HD int imax(int a, int b) { return a > b ? a : b; }

// high word of (hi:lo) << min(c, 32)
MP_HD uint32_t shl_hi(uint32_t lo, uint32_t hi, uint32_t c)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_lc(lo, hi, c);
#else
    return c >= 32 ? lo : c == 0 ? hi : (hi << c) | (lo >> (32 - c));
#endif
}

// low word of (hi:lo) >> 11
MP_HD uint32_t shr11_lo(uint32_t lo, uint32_t hi)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, 11);
#else
    return (lo >> 11) | (hi << 21);
#endif
}

// m * 2^k mod 2^64 for any k >= 0, as multiplications (FMA pipe) by 2^k.
MP_HD uint64_t shl_mod(uint64_t m, uint32_t k)
{
    const uint32_t plo = pow2_32(k), phi = pow2_32(k - 32u);  // k - 32 wraps to a huge count when k < 32
    const uint64_t r = (uint64_t)lo32(m) * plo;
    return mk64(hi32(r) + hi32(m) * plo + lo32(m) * phi, lo32(r));
}

// Biased exponent clamped to >= 1, and the integer significand (hidden bit only
// for E > 0), of the binary64 pattern x.
MP_HD void unpack(uint64_t x, int &e1, uint64_t &m)
{
    const uint32_t h = hi32(x);
    const int e = (int)((h >> 20) & 0x7FFu);
    e1 = e > 0 ? e : 1;
    m = mk64((h & 0xFFFFFu) | (e > 0 ? 0x100000u : 0u), lo32(x));
}

// e = a + b - s for s = fl(a + b), as a binary64 pattern.  `bad` is raised when
// the operands leave the domain stated above.  With SUBNORMAL the domain also
// takes in a subnormal e (the error of a sum of tiny operands): e is a multiple
// of 2^(u - 1075) below 2^-1022, so its fraction field is exactly mag * 2^(u - 1);
// the domain is then only "a and b finite with biased exponent <= 2045".
template <bool SUBNORMAL = false>
MP_HD uint64_t two_sum_err(uint64_t A, uint64_t B, uint64_t S, uint32_t &bad)
{
    int ea, eb, es;
    uint64_t ma, mb, ms;
    unpack(A, ea, ma);
    unpack(B, eb, mb);
    unpack(S, es, ms);
    const int u = imin(imin(ea, eb), es);
    const uint64_t ta = shl_mod(ma, (uint32_t)(ea - u)), tb = shl_mod(mb, (uint32_t)(eb - u));
    const uint64_t ts = shl_mod(ms, (uint32_t)(es - u));
    // Signs by the sign words k = 0 or all ones: (t ^ k) - k negates t when k is all
    // ones, and -x = ~x + 1, so
    //   ei = (ta^ka) - ka + (tb^kb) - kb - ((ts^ks) - ks)
    //      = (ta^ka) + (tb^kb) + (ts^~ks) + (1 + ks - ka - kb),
    // the last term a small constant in [0, 3].
    const uint64_t ka = (uint64_t)((int64_t)A >> 63), kb = (uint64_t)((int64_t)B >> 63),
                   ks = (uint64_t)((int64_t)S >> 63);
    const uint32_t cc = 1u + lo32(ks) - lo32(ka) - lo32(kb);
    const uint64_t ei = (ta ^ ka) + (tb ^ kb) + (ts ^ ~ks) + (uint64_t)cc;
    const uint64_t kn = (uint64_t)((int64_t)ei >> 63);
    const uint64_t mag = (ei ^ kn) - kn;
    // Normalise mag (< 2^55) to a leading one at bit 63 with one count-leading-zeros:
    // on the high word when it is nonzero, else on the low word (then lz = 32 + c).
    const uint32_t mh = hi32(mag), ml = lo32(mag);
    const bool z = mh == 0;
    const uint32_t x = z ? ml : mh, y = z ? 0u : ml;
    const int c = clz32(x);                          // 32 only when mag == 0
    const uint32_t nh = shl_hi(y, x, (uint32_t)c);   // high word of mag << lz (0 when mag == 0)
    const uint32_t nl = y << (c & 31);               // low word (y == 0 whenever c == 32)
    const int be = 11 - c - (z ? 32 : 0) + u;        // biased exponent of e
    // The hidden bit (bit 20 of nh >> 11) is 2^20 exactly when mag != 0, so multiplying
    // the exponent field by it packs +0 for mag == 0 with no select.
    const uint32_t f = nh >> 11, hb = f & 0x100000u;
    const uint32_t eh = (f + (uint32_t)(be - 1) * hb) | (hi32(kn) & 0x80000000u);
    const uint32_t el = shr11_lo(nl, nh);
    // |s| <= 2 max(|a|, |b|), so exponents of a and b <= 2045 bound s's by 2046
    if (SUBNORMAL) {
        bad |= (uint32_t)(imax(ea, eb) > 2045);
        const uint64_t sub = shl_mod(mag, (uint32_t)(u - 1)) | (kn & 0x8000000000000000ull);
        return (hb != 0 && be < 1) ? sub : mk64(eh, el);
    }
    bad |= (uint32_t)(imax(ea, eb) > 2045) | (uint32_t)(hb != 0 && be < 1);
    return mk64(eh, el);
}

// e = a*b - p for p = fl(a*b) (the error term of Algorithm 3's TwoProd, which
// FMA(a, b, -p) returns), as a binary64 pattern.  With ma, mb the integer
// significands and units 2^(Ea+Eb-2150), a*b = ma*mb exactly, and p = mp * 2^sh in
// those units with sh = Ep - Ea - Eb + 1075 in {52, 53, 54} for normal operands;
// |e| <= ulp(p)/2 < 2^54 units, so e = ma*mb - mp*2^sh evaluated modulo 2^64 (the
// low 64 bits of the 106-bit product, three multiplications on the FMA pipe) is
// exact as a signed value; its sign is then applied relative to p's.  Domain:
// a and b normal with p normal, or a zero operand (e = +0); e zero or normal;
// elsewhere `bad` is raised.
MP_HD uint64_t two_prod_err(uint64_t A, uint64_t B, uint64_t P, uint32_t &bad)
{
    int ea, eb, ep;
    uint64_t ma, mb, mp;
    unpack(A, ea, ma);
    unpack(B, eb, mb);
    unpack(P, ep, mp);
    const uint64_t lo = ma * mb;                                      // low 64 bits of the product
    const int sh = ep - ea - eb + 1075;
    const uint64_t ei = lo - shl_mod(mp, (uint32_t)sh);
    const uint64_t kn = (uint64_t)((int64_t)ei >> 63);
    const uint64_t mag = (ei ^ kn) - kn;
    const int lz = clz64(mag);
    const uint64_t norm = shl_mod(mag, (uint32_t)lz & 63u);
    const int be = ea + eb - 1064 - lz;                              // biased exponent of e
    const uint32_t sign = (hi32(A) ^ hi32(B) ^ hi32(kn)) & 0x80000000u;
    const uint32_t eh = ((hi32(norm) >> 11) + ((uint32_t)(be - 1) << 20)) | sign;
    const uint32_t el = shr11_lo(lo32(norm), hi32(norm));
    const uint32_t Ea = (hi32(A) >> 20) & 0x7FFu, Eb = (hi32(B) >> 20) & 0x7FFu, Ep = (hi32(P) >> 20) & 0x7FFu;
    const bool za = ((A << 1) == 0), zb = ((B << 1) == 0), zp = ((P << 1) == 0);
    bad |= (uint32_t)(Ea == 0 && !za && !zb) | (uint32_t)(Eb == 0 && !zb && !za) | (uint32_t)(Ea == 0x7FF) |
           (uint32_t)(Eb == 0x7FF) | (uint32_t)(Ep == 0x7FF) | (uint32_t)(Ep == 0 && !zp) |
           (uint32_t)(mag != 0 && be < 1) | (uint32_t)(!za && !zb && (sh < 52 || sh > 54));
    return mag == 0 ? 0 : mk64(eh, el);
}

}  // namespace eft_int
}  // namespace mp
