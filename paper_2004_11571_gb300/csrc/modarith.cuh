// Device modular arithmetic for word-size primes (paper Sect. 3.1).
//
// Integer products are built from 64-bit mul.lo / mul.hi.  Values are kept
// "lazy" in [0, 2p) inside loops and brought to [0, p) only where a result
// leaves the kernel; every bound below needs p < 2^62.
#pragma once
#include <cstdint>
#include "common.h"

namespace pe {

__device__ __forceinline__ uint64_t canon(uint64_t x, uint64_t p) { return x >= p ? x - p : x; }

// ---------------------------------------------------------------- Montgomery
// Montgomery reduction with R = 2^64: for a 128-bit x = hi*2^64 + lo < p*2^64,
// returns (x + q*p) / 2^64 with q = lo * (-p^-1) mod 2^64.  The low words of x
// and q*p add up to 0 mod 2^64, so they carry out exactly when lo != 0.
// Result < 2p whenever x < p*2^64.
__device__ __forceinline__ uint64_t mont_redc(uint64_t lo, uint64_t hi, const ModCtx &mc)
{
    const uint64_t q = lo * mc.pinv_neg;
    return hi + __umul64hi(q, mc.p) + (lo != 0 ? 1ull : 0ull);
}

// a*b*2^-64 mod p, lazy: a, b < 2p and 4p < 2^64 give a result < 2p.
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, const ModCtx &mc)
{
    return mont_redc(a * b, __umul64hi(a, b), mc);
}

// (x^e) in Montgomery form, canonical; xR is x in Montgomery form (< 2p).
__device__ __forceinline__ uint64_t mont_pow(uint64_t xR, uint64_t e, const ModCtx &mc)
{
    if (e == 0) return mc.r1;
    uint64_t r = xR;
    for (int b = 62 - __clzll(e); b >= 0; --b) {
        r = mont_mul(r, r, mc);
        if ((e >> b) & 1) r = mont_mul(r, xR, mc);
    }
    return canon(r, mc.p);
}

// --------------------------------------------------- Barrett, fixed multiplier
// Barrett's product with the quotient estimate scaled by the multiplier:
// wq = floor(w * 2^64 / p) for a multiplier w < p.  For any x < 2^64,
// q = floor(x * wq / 2^64) is floor(x*w/p) or one less, so x*w - q*p lies in
// [0, 2p) and is exact in 64-bit arithmetic.
__device__ __forceinline__ uint64_t barrett_mul(uint64_t x, uint64_t w, uint64_t wq, uint64_t p)
{
    return x * w - __umul64hi(x, wq) * p;
}

// The same product with a cheaper quotient: with x = x1*2^32 + x0 and
// wq = w1*2^32 + w0, x*wq = (x1*w1 + hi(x1*w0) + hi(x0*w1)) * 2^64 + R with
// 0 <= R < 3 * 2^64, so the estimate below is floor(x*wq / 2^64) minus 0, 1
// or 2.  The result therefore lies in [0, 4p), exact in 64 bits for
// p < 2^62, and stays a valid input (any x < 2^64) for the next product.
__device__ __forceinline__ uint64_t barrett_mul_lazy4(uint64_t x, uint64_t w, uint64_t wq, uint64_t p)
{
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    const uint32_t w0 = (uint32_t)wq, w1 = (uint32_t)(wq >> 32);
    const uint64_t q = (uint64_t)x1 * w1 + __umulhi(x1, w0) + __umulhi(x0, w1);
    return x * w - q * p;
}

// 32-bit words, p < 2^30: with wq = floor(w * 2^32 / p) and any x < 2^32,
// x*w - hi(x*wq)*p lies in [0, 2p) (same argument as above, one word).
__device__ __forceinline__ uint32_t barrett_mul32(uint32_t x, uint32_t w, uint32_t wq, uint32_t p)
{
    return x * w - __umulhi(x, wq) * p;
}

// The same value as barrett_mul_lazy4, with r = x*w + q*(2^64 - p) mod 2^64
// accumulated by 32-bit multiply-adds (two wide, four low) instead of two
// 64-bit products and a subtraction.  np = 2^64 - p.
__device__ __forceinline__ uint64_t barrett_mul_lazy4_mad(uint64_t x, uint64_t w, uint64_t wq, uint64_t np)
{
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
    const uint32_t q0w = (uint32_t)wq, q1w = (uint32_t)(wq >> 32);
    const uint64_t q = (uint64_t)x1 * q1w + __umulhi(x1, q0w) + __umulhi(x0, q1w);
    const uint32_t q0 = (uint32_t)q, q1 = (uint32_t)(q >> 32);
    const uint32_t n0 = (uint32_t)np, n1 = (uint32_t)(np >> 32);
    uint64_t t;
    uint32_t hi;
    asm("mad.wide.u32 %0, %1, %2, 0;" : "=l"(t) : "r"(x0), "r"(w0));
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(t) : "r"(q0), "r"(n0));
    hi = (uint32_t)(t >> 32);
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(hi) : "r"(x0), "r"(w1));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(hi) : "r"(x1), "r"(w0));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(hi) : "r"(q0), "r"(n1));
    asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(hi) : "r"(q1), "r"(n0));
    return ((uint64_t)hi << 32) | (uint32_t)t;
}

// Given mR = m * 2^64 mod p (canonical), the Barrett quotient of m is
// (m*2^64 - mR) / p, an exact division, hence equal to -mR * p^-1 mod 2^64.
__device__ __forceinline__ uint64_t barrett_quotient_from_mont(uint64_t mR, const ModCtx &mc)
{
    return (0ull - mR) * mc.pinv;
}

// ------------------------------------------------------ 96-bit accumulation
// acc(lo, hi) += x, with the carry of the 64-bit addition into hi.
__device__ __forceinline__ void add96(uint64_t &lo, uint32_t &hi, uint64_t x)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(lo), "+r"(hi) : "l"(x));
}

__device__ __forceinline__ void add96(uint64_t &lo, uint32_t &hi, uint64_t xlo, uint32_t xhi)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+l"(lo), "+r"(hi) : "l"(xlo), "r"(xhi));
}

// (hi*2^64 + lo) mod p, canonical, for hi < 2^32 and p < 2^62:
// hi*2^64 = hi*r1 (mod p) and lo = lo*1 by the fixed-multiplier product, each
// in [0, 2p); their sum is below 4p and two conditional subtractions finish.
__device__ __forceinline__ uint64_t reduce96(uint64_t lo, uint32_t hi, const ModCtx &mc)
{
    uint64_t a = barrett_mul((uint64_t)hi, mc.r1, mc.w64q, mc.p);
    uint64_t b = lo - __umul64hi(lo, mc.one_q) * mc.p;
    uint64_t s = a + b;
    s = s >= mc.p2 ? s - mc.p2 : s;
    return s >= mc.p ? s - mc.p : s;
}

// ------------------------------------------------ 192-bit exact sums
// (h, m, l) += a * b, exact (a, b < 2^64, h counts the carries out of 128 bits).
__device__ __forceinline__ void mac192(uint64_t &l, uint64_t &m, uint32_t &h, uint64_t a, uint64_t b)
{
    asm("mad.lo.cc.u64 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u64 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+l"(l), "+l"(m), "+r"(h)
        : "l"(a), "l"(b));
}

// x = h*2^128 + m*2^64 + l times fac/R^3 mod p, canonical, for h < p (sums of
// fewer than 2^64 products of values below 2^62 stay far under p * 2^128).
// With R = 2^64: REDC(l) = l/R, REDC((h, m + l/R)) = h + m/R + l/R^2 = x/R^2,
// and a Montgomery product by fac gives x fac / R^3: fac = R^3 mod p yields
// x mod p, fac = R^2 mod p yields x/R (a sum of products of Montgomery forms
// back in Montgomery form).
__device__ __forceinline__ uint64_t reduce192(uint64_t l, uint64_t m, uint32_t h, uint64_t fac, const ModCtx &mc)
{
    const uint64_t a = mont_redc(l, 0, mc);
    uint64_t lo;
    uint32_t hi = h;
    asm("add.cc.u64 %0, %2, %3;\n\taddc.u32 %1, %1, 0;" : "=l"(lo), "+r"(hi) : "l"(m), "l"(a));
    const uint64_t b = mont_redc(lo, hi, mc);
    return canon(mont_mul(b, fac, mc), mc.p);
}

// ------------------------------------------------- Algorithms 2 and 3 (FP64)
// Modular product of canonical x, y < p < 2^50 held in doubles, u = 1/(double)p.
// h + l = x*y exactly (FMA error-free product); c is the quotient within one;
// g = x*y - c*p is the remainder within p, then corrected into [0, p).
// Every operation is explicitly round-to-nearest, so no contraction can alter it.
__device__ __forceinline__ double fp64_mulmod(double x, double y, double p, double u)
{
    const double h = __dmul_rn(x, y);
    const double l = __fma_rn(x, y, -h);
    const double b = __dmul_rn(h, u);
    const double c = floor(b);
    const double d = __fma_rn(-c, p, h);
    double g = __dadd_rn(d, l);
    g = (g >= p) ? __dsub_rn(g, p) : g;
    g = (g < 0.0) ? __dadd_rn(g, p) : g;
    return g;
}

// Modular addition of canonical x, y < p < 2^50 held in doubles.
__device__ __forceinline__ double fp64_addmod(double x, double y, double p)
{
    const double s = __dadd_rn(x, y);
    return (s >= p) ? __dsub_rn(s, p) : s;
}

}  // namespace pe
