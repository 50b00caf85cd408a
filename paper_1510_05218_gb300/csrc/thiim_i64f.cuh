// IEEE binary64 addition and multiplication on the integer pipe.
//
// GB300 issues FP64 adds, multiplies and fused multiply-adds on one FP64 pipe
// that retires about 1.7 instructions per SM and clock, while its integer
// units retire 64 (logic, shifts, multiply-adds, selects) to 128 (adds).  The
// FP64 sweep is bound by that pipe.  Part of its work can run instead on the
// integer units by computing the same IEEE 754 binary64 operation in integer
// arithmetic: the result of add() and mul() below is the correctly rounded
// (round to nearest, ties to even) binary64 sum or product, bit for bit what
// the FP64 pipe returns, so a kernel that uses them computes exactly what the
// pure-FP64 kernel computes.
//
// Method (the textbook construction of IEEE arithmetic, e.g. Goldberg, "What
// every computer scientist should know about floating-point arithmetic",
// 1991, and Muller et al., "Handbook of Floating-Point Arithmetic", ch. 7-8):
//   add: order the operands by magnitude, align the smaller significand to
//        the larger one's exponent keeping 10 extra low bits and a sticky bit
//        (OR of every bit shifted out), add or subtract the integers,
//        normalise with a leading-zero count, round the 53 leading bits to
//        nearest-even from the guard bit and the bits below it, and pack.
//        The sticky bit in the last place is exact for rounding: with 10 bits
//        below the result's last place (at most 2 of them lost to the
//        normalising shift when bits were shifted out) the true sum and the
//        computed one lie strictly between the same rounding boundaries.
//   mul: multiply the two 53-bit significands exactly (106-bit product), take
//        the 53 leading bits, round to nearest-even from the rest, add the
//        exponents and pack.
// Rounding may carry into the exponent; packing as (exponent - 1) * 2^52 +
// significand (hidden bit included) absorbs that carry, and an overflow to
// the top exponent produces the correctly rounded infinity.
//
// add_bits covers every operand pair (zeros, subnormals, overflow, infinities
// and NaN) without a branch.  mul covers products of normal numbers with a
// normal result or a zero factor; subnormal products, infinities and NaN use
// the FP64 pipe's own instruction.
//
// The functions also compile as plain C++ (no CUDA), where mul's fallback is
// the host's IEEE double arithmetic; the CPU test suite checks the integer
// path against the host bit for bit.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define I64F_FN __host__ __device__ __forceinline__
#else
#define I64F_FN inline
#endif

namespace thiim {
namespace i64f {

constexpr uint64_t SIGN = 0x8000000000000000ull;
constexpr uint64_t ABS = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t FRAC = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t HIDDEN = 0x0010000000000000ull;

// The bit reinterpretations are opaque moves on the device: seen through,
// the compiler rewrites "bits ^ sign" and "bits & ~sign" of a double as an
// FP64 negation or absolute value, which costs an FP64-pipe instruction
// when the consumer is integer code.
I64F_FN uint64_t bits(double x) {
#if defined(__CUDA_ARCH__)
    uint64_t u;
    asm("mov.b64 %0, %1;" : "=l"(u) : "d"(x));
    return u;
#else
    uint64_t u;
    memcpy(&u, &x, sizeof(u));
    return u;
#endif
}

I64F_FN double from_bits(uint64_t u) {
#if defined(__CUDA_ARCH__)
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(u));
    return x;
#else
    double x;
    memcpy(&x, &u, sizeof(x));
    return x;
#endif
}

// Leading zeros of a 64-bit value (64 for zero).
I64F_FN int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

I64F_FN uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }
I64F_FN int imin(int a, int b) { return a < b ? a : b; }

// High 64 bits of the 128-bit product.
I64F_FN uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// The FP64 pipe's own multiplication (mul's fallback for the rare cases).
I64F_FN double pipe_mul(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dmul_rn(a, b);
#else
    volatile double r = a * b;
    return r;
#endif
}

// Result of the integer path and whether it applies to these operands.
struct Res {
    uint64_t v;
    bool ok;
};

// NaN results: an invalid operation (Inf - Inf) returns the default NaN
// below and a NaN operand is returned quieted, as the FP64 pipe does
// (measured on GB300: Inf - Inf = 0xFFF8000000000000, NaN + 1 = the NaN
// with the quiet bit set).
constexpr uint64_t DEFAULT_NAN = 0xFFF8000000000000ull;
constexpr uint64_t QUIET = 0x0008000000000000ull;
constexpr uint64_t INF = 0x7FF0000000000000ull;

// a + b, round to nearest even, integer arithmetic only, for every operand
// pair (zeros, subnormals, overflow, infinities, NaN), without branches.
I64F_FN uint64_t add_bits(uint64_t A, uint64_t B) {
    const bool swap = (B & ABS) > (A & ABS);
    const uint64_t X = swap ? B : A, Y = swap ? A : B;   // |X| >= |Y|
    const uint64_t ax = X & ABS, ay = Y & ABS;
    const uint64_t sx = X & SIGN;
    const bool opp = ((X ^ Y) & SIGN) != 0;
    const uint32_t ex = (uint32_t)(ax >> 52);
    const uint32_t ey = (uint32_t)(ay >> 52);
    // significands with the hidden bit at 61 (9 extra low bits); a subnormal
    // or zero operand has no hidden bit and the exponent of the smallest
    // normals, 1
    const uint32_t ex1 = ex ? ex : 1u, ey1 = ey ? ey : 1u;
    const uint64_t mx = ((ax & FRAC) | (ex ? HIDDEN : 0)) << 9;
    const uint64_t my = ((ay & FRAC) | (ey ? HIDDEN : 0)) << 9;
    const uint32_t d = umin32(ex1 - ey1, 63u);                // my < 2^62: a shift of 63 clears it
    const uint64_t ys0 = my >> d;
    const uint64_t ys = ys0 | (uint64_t)((ys0 << d) != my);   // sticky bit
    const uint64_t m = opp ? mx - ys : mx + ys;            // < 2^63
    // normalise the leading one to bit 62, but not below the exponent of the
    // smallest normals: a subnormal result keeps exponent field 0 and is
    // exact (every double is a multiple of 2^-1074, and subnormal results
    // only arise when no bit was shifted out)
    const int lz = imin(clz64(m), (int)ex1 + 1);
    const uint64_t n = m << (lz - 1);
    const int e = (int)ex1 + 2 - lz;                       // biased exponent of n / 2^62, >= 1
    // round to nearest even at bit 10: + (2^9 - 1) + (bit 10), cannot overflow
    const uint64_t q = (n + 0x1FFull + ((n >> 10) & 1ull)) >> 10;
    // exponent field e - 1 plus the significand (its hidden bit carries into
    // the field; rounding up to 2^53 carries once more)
    uint64_t v = sx | (((uint64_t)(uint32_t)(e - 1) << 52) + q);
    v = e >= 2047 ? (sx | INF) : v;                        // overflow
    v = m == 0 ? (opp ? 0ull : sx) : v;                    // exact zero: +0, or the sign of two zeros
    // an infinite or NaN operand
    const uint64_t special = ax > INF ? (X | QUIET) : ((ay == INF) & opp ? DEFAULT_NAN : X);
    return ex == 0x7FFu ? special : v;
}

// a * b, round to nearest even, integer arithmetic only.  Covers normal
// operands with a normal product and a zero operand (times a finite one);
// subnormal operands or results, infinities and NaN are left to the FP64 pipe.
I64F_FN Res mul_int(uint64_t A, uint64_t B) {
    const uint32_t ea = (uint32_t)(A >> 52) & 0x7FFu;
    const uint32_t eb = (uint32_t)(B >> 52) & 0x7FFu;
    const uint64_t ma = (A & FRAC) | HIDDEN, mb = (B & FRAC) | HIDDEN;
    const uint64_t lo = ma * mb, hi = mulhi64(ma, mb);    // 106-bit product
    const uint32_t s = (uint32_t)(hi >> 41) & 1u;          // product >= 2^105
    const uint64_t q0 = s ? ((hi << 11) | (lo >> 53)) : ((hi << 12) | (lo >> 52));
    const uint64_t rem = lo & (s ? 0x1FFFFFFFFFFFFFull : 0xFFFFFFFFFFFFFull);
    const uint64_t half = s ? 0x10000000000000ull : 0x8000000000000ull;
    const uint64_t q = q0 + (uint64_t)((rem > half) | ((rem == half) & ((uint32_t)q0 & 1u)));
    const int e = (int)ea + (int)eb - 1023 + (int)s;
    const uint64_t sign = (A ^ B) & SIGN;
    const bool zero = ((A & ABS) == 0) | ((B & ABS) == 0);
    Res out;
    out.v = zero ? sign : (sign | (((uint64_t)(uint32_t)(e - 1) << 52) + q));
    out.ok = zero ? (ea != 0x7FFu && eb != 0x7FFu)
                  : ((ea - 1u < 2046u) && (eb - 1u < 2046u) && ((uint32_t)(e - 1) < 2046u));
    return out;
}

I64F_FN double add(double a, double b) { return from_bits(add_bits(bits(a), bits(b))); }

I64F_FN double sub(double a, double b) { return from_bits(add_bits(bits(a), bits(b) ^ SIGN)); }

I64F_FN double mul(double a, double b) {
    const Res r = mul_int(bits(a), bits(b));
    double v = from_bits(r.v);
    if (!r.ok) v = pipe_mul(a, b);
    return v;
}

}  // namespace i64f
}  // namespace thiim
