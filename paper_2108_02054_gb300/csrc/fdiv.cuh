// Correctly rounded FP64 division, and FP64 -> FP32 conversion, in integer
// arithmetic.
//
// On this part an FP64 division takes about 565 cycles (its refinement steps
// run on the FP64 pipe, 64 cycles per warp instruction), while 32-bit integer
// multiply-adds take about 5.  The coarsest LU divides a whole column by one
// pivot per elimination step, on its critical path, so the division is done
// here with integer multiplies instead:
//
//  - the divisor's significand, normalised to d in [2^63, 2^64), gets the
//    reciprocal v = floor((2^128 - 1) / d) - 2^64: a 44-bit seed on the FP32
//    pipe (the reciprocal approximation instruction and one Newton-Raphson
//    step in two-float arithmetic), one Newton-Raphson step in 64-bit fixed
//    point, then a correction by the exact remainder 2^128 - 1 - (2^64 + v) d
//    until it lies in [0, d);
//  - each dividend's significand becomes a two-word numerator (u1, u0) with
//    u1 < d, divided by the two-by-one division with a precomputed reciprocal
//    of Moller and Granlund ("Improved division by invariant integers", IEEE
//    Trans. Computers 60(2), 2011, Algorithm 4), which returns the exact
//    64-bit quotient Q in [2^63, 2^64) and its remainder;
//  - Q's top 53 bits are rounded to nearest, ties to even, from bit 10
//    (round) and bits 9..0 with the remainder (sticky).
//
// The result is the IEEE quotient num / den whenever the divisor is normal
// and the quotient is a normal number; zero dividends give the signed zero.
// Everything else (subnormal, infinite or NaN operands, results outside the
// normal range, a reciprocal whose correction did not settle) falls back to
// the hardware division, so the function equals num / den for every input.
#pragma once
#include <cstdint>

namespace amgpr {

struct DivRecip {
    double den;              // the divisor
    unsigned long long d;    // its significand << 11, in [2^63, 2^64)
    unsigned long long v;    // floor((2^128 - 1) / d) - 2^64
    unsigned long long sgn;  // its sign bit
    int e;                   // its unbiased exponent
    bool ok;                 // normal divisor and exact v
};

__device__ __forceinline__ float fdiv_rcp_seed(float f) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
    return r;
}

// high 64 bits of the signed product of an unsigned u and a signed s
__device__ __forceinline__ long long fdiv_mulhi_us(unsigned long long u, long long s) {
    const unsigned long long h = __umul64hi(u, (unsigned long long)s);
    return (long long)(s < 0 ? h - u : h);
}

__device__ __forceinline__ DivRecip div_recip(double den) {
    DivRecip R;
    const unsigned long long b = (unsigned long long)__double_as_longlong(den);
    const int eb = (int)((b >> 52) & 0x7ff);
    R.den = den;
    R.sgn = b & 0x8000000000000000ull;
    R.e = eb - 1023;
    const unsigned long long d = ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) << 11;
    R.d = d;
    // seed on the FP32 pipe: with D = d / 2^40 ~ dh + dl 2^-24 (48 bits),
    // r0 ~ 1 / dh and e = 1 - D r0 (two fmas), 1 / D ~ r0 + r0 e (~44 bits)
    const float dh = (float)(unsigned)(d >> 40), dl = (float)(unsigned)((d >> 16) & 0xffffffu) * 0x1p-24f;
    const float r0 = fdiv_rcp_seed(dh);
    const float e = fmaf(-dl, r0, fmaf(-dh, r0, 1.0f));
    const float c = r0 * e;
    // v0 = 2^88 (r0 + c) - 2^64 in 64-bit fixed point, from the floats' bits
    const unsigned rb = __float_as_uint(r0);
    const int re = (int)((rb >> 23) & 0xff) - 127;
    unsigned long long v = re == -24 ? (unsigned long long)(rb & 0x7fffffu) << 41 : (re > -24 ? ~0ull : 0ull);
    const unsigned cb = __float_as_uint(c);
    const int ce = (int)((cb >> 23) & 0xff) - 127 + 65;  // 2^88 c = +-(2^23 + m) 2^ce
    if ((cb & 0x7fffffffu) != 0u && ce >= 0 && ce < 40) {
        const unsigned long long mag = (unsigned long long)((cb & 0x7fffffu) | 0x800000u) << ce;
        if (cb >> 31) v = v > mag ? v - mag : 0ull;
        else v = v + mag < v ? ~0ull : v + mag;
    }
    // one Newton-Raphson step in 64-bit fixed point: y <- y + y (2^128 - d y) / 2^128
    {
        const unsigned long long lo = d * v, hi = __umul64hi(d, v);
        const unsigned long long ph = d + hi;  // d y = ph:lo (mod 2^128)
        const long long eh = (long long)(~ph + (lo == 0ull ? 1ull : 0ull));  // high word of -(ph:lo)
        v += (unsigned long long)(eh + fdiv_mulhi_us(v, eh));
    }
    // exact v: S = 2^128 - 1 - (2^64 + v) d must lie in [0, d).  After the
    // Newton step v is short by at most a few units, so a fixed sequence of
    // selects (one decrement, three increments) settles it without branches;
    // S is a 129-bit two's-complement value (sh, sm, sl) moved by +-d
    const unsigned long long lo = v * d, hi = __umul64hi(v, d);
    const unsigned long long ph = d + hi;
    unsigned long long sh = ph < d ? ~0ull : 0ull;  // (2^64 + v) d >= 2^128: S < 0
    unsigned long long sm = ~ph, sl = ~lo;
    {
        const unsigned long long neg = sh >> 63;  // S < 0: v -= 1, S += d
        const unsigned long long t = sl + (d & (0ull - neg));
        const unsigned long long cy = t < sl ? 1ull : 0ull;
        sl = t;
        const unsigned long long t2 = sm + cy;
        sh += t2 < sm ? 1ull : 0ull;
        sm = t2;
        v -= neg;
    }
#pragma unroll
    for (int it = 0; it < 3; ++it) {  // S >= d: v += 1, S -= d
        const unsigned long long big = (sh >> 63) == 0ull && (sm != 0ull || sl >= d) ? 1ull : 0ull;
        const unsigned long long t = sl - (d & (0ull - big));
        const unsigned long long bw = t > sl ? 1ull : 0ull;
        sl = t;
        const unsigned long long t2 = sm - bw;
        sh -= t2 > sm ? 1ull : 0ull;
        sm = t2;
        v += big;
    }
    R.v = v;
    R.ok = eb != 0 && eb != 0x7ff && sh == 0ull && sm == 0ull && sl < d;
    return R;
}

// num / den, rounded to nearest even (see above); R = div_recip(den)
__device__ __forceinline__ double div_rn(double num, const DivRecip &R) {
    const unsigned long long xb = (unsigned long long)__double_as_longlong(num);
    const int ex = (int)((xb >> 52) & 0x7ff);
    if (!R.ok || ex == 0 || ex == 0x7ff) {
        if (R.ok && (xb & 0x7fffffffffffffffull) == 0ull)
            return __longlong_as_double((long long)((xb ^ R.sgn) & 0x8000000000000000ull));
        return num / R.den;
    }
    const unsigned long long X = ((xb & 0x000fffffffffffffull) | 0x0010000000000000ull) << 11;
    unsigned long long u1, u0;
    int e = (ex - 1023) - R.e;
    if (X >= R.d) {
        u1 = X >> 1;
        u0 = X << 63;
    } else {
        u1 = X;
        u0 = 0ull;
        e -= 1;
    }
    // two-by-one division with the precomputed reciprocal
    unsigned long long q0 = R.v * u1, q1 = __umul64hi(R.v, u1);
    const unsigned long long s0 = q0 + u0;
    q1 += u1 + (s0 < q0 ? 1ull : 0ull) + 1ull;
    q0 = s0;
    unsigned long long rem = u0 - q1 * R.d;
    if (rem > q0) {
        q1 -= 1ull;
        rem += R.d;
    }
    if (rem >= R.d) {
        q1 += 1ull;
        rem -= R.d;
    }
    // round Q = q1 (bit 63 set) to 53 bits, nearest even
    unsigned long long m = q1 >> 11;
    const bool rnd = (q1 >> 10) & 1ull, sticky = (q1 & 0x3ffull) != 0ull || rem != 0ull;
    if (rnd && (sticky || (m & 1ull))) m += 1ull;
    if (m == 0x0020000000000000ull) {
        m >>= 1;
        e += 1;
    }
    const int be = e + 1023;
    if (be <= 0 || be >= 0x7ff) return num / R.den;
    return __longlong_as_double(
        (long long)(((xb ^ R.sgn) & 0x8000000000000000ull) | ((unsigned long long)be << 52) | (m & 0x000fffffffffffffull)));
}



// Whether x is finite, from its exponent bits (the FP64 compare would run on
// the FP64 pipe).
__device__ __forceinline__ bool finite_bits(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// (float)x rounded to nearest, ties to even, from the IEEE 754 formats: on
// this part the conversion instruction runs on the FP64 pipe (about as slow
// as an FP64 add), these integer steps do not.  Worth it where the FP64 pipe
// bounds a kernel (the finest level's copy-and-cast), not elsewhere (measured
// slower in the V-cycle kernels).  The 52-bit significand drops
// 29 bits (normal results) or more (subnormal results, shift 52 - (e + 149)
// for an unbiased exponent e), rounded from the dropped bits; a carry out of
// the significand moves to the next exponent (up to infinity).  Infinities
// and NaNs use the conversion instruction.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const int eb = (int)((b >> 52) & 0x7ff);
    if (eb == 0x7ff) return (float)x;
    const int e = eb - 1023;
    if (e > 127) return __uint_as_float(sgn | 0x7f800000u);
    const unsigned long long full = (b & 0x000fffffffffffffull) | (eb ? 0x0010000000000000ull : 0ull);
    // result = round(full * 2^(e - 52)) in units of the float's last place:
    // 2^(e - 23) for normal results, 2^-149 for subnormal ones
    const int sh = e >= -126 ? 29 : 52 - (e + 149);
    if (eb == 0 || sh > 63) return __uint_as_float(sgn);
    unsigned long long q = full >> sh;
    const unsigned long long rem = full & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) q += 1ull;
    unsigned bits;
    if (e >= -126) {
        // q in [2^23, 2^24]: the hidden bit and 23 fraction bits (2^24: a carry)
        bits = (unsigned)((unsigned long long)(e + 127) << 23) + (unsigned)(q - (1ull << 23));
        if (bits >= 0x7f800000u) bits = 0x7f800000u;
    } else {
        bits = (unsigned)q;  // subnormal (2^23: the smallest normal)
    }
    return __uint_as_float(sgn | bits);
}


}  // namespace amgpr
