// Arithmetic policies of the fused sweep.
//
// The sweep body (thiim_sweep.cuh) is written once against a policy that
// says how a complex value is loaded, stored, added and updated:
//
//   Native<double>  complex128 storage, FP64 arithmetic.
//   Native<float>   complex64 storage, FP32 arithmetic.
//   Fp64Int<OFF>    complex128 storage, FP64 arithmetic with part of it on
//                   the integer pipe (thiim_i64f.cuh): bit-identical
//                   results to Native<double>, fewer FP64-pipe instructions.
//   PairArith<I,O>  complex128 data, arithmetic on pairs of FP32 numbers
//                   (hi + lo, "double-float").  GB300 executes FP64 at
//                   2 instructions/clk/SM but FP32 at 128, so the FP64 sweep
//                   is pipe-bound; the pair form moves the work to the FP32
//                   pipe.  Coefficients arrive pre-split as float4
//                   (re.hi, re.lo, im.hi, im.lo); fields are read as
//                   complex128 (I = 0) or as float4 pairs (I = 1) and written
//                   as complex128 (O = 0) or pairs (O = 1), so a multi-
//                   iteration call converts only on its first and last pass.
//
// Pair arithmetic (Dekker / Knuth error-free transformations):
//   two_sum(a, b)  -> s + e == a + b exactly (6 FP32 operations),
//   two_prod(a, b) -> p + e == a * b exactly (1 multiply + 1 FMA),
// so a product of pairs is exact up to the lo*lo term and the cross terms'
// rounding (relative 2^-48), and a sum of such products is accumulated with
// two_sum on the leading parts and plain FP32 on the error parts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "thiim_i64f.cuh"

namespace thiim {

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };

template <typename V>
__device__ __forceinline__ V ldg_as(const void *base, size_t i) {
    return __ldg(reinterpret_cast<const V *>(base) + i);
}
// L2 eviction priority of a load: createpolicy gives a cache policy that
// ld.global.L2::cache_hint applies to the lines it brings in.
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
template <typename V> __device__ __forceinline__ V ldg_hint(const void *base, size_t i, uint64_t pol);
template <> __device__ __forceinline__ double2 ldg_hint<double2>(const void *base, size_t i, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y) : "l"(reinterpret_cast<const double2 *>(base) + i), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ float2 ldg_hint<float2>(const void *base, size_t i, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(v.x), "=f"(v.y) : "l"(reinterpret_cast<const float2 *>(base) + i), "l"(pol));
    return v;
}
template <> __device__ __forceinline__ float4 ldg_hint<float4>(const void *base, size_t i, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(reinterpret_cast<const float4 *>(base) + i), "l"(pol));
    return v;
}

template <typename V>
__device__ __forceinline__ void stg_as(void *base, size_t i, V v) {
    reinterpret_cast<V *>(base)[i] = v;
}

// ---------------------------------------------------------------- native ----
template <typename R>
struct Native {
    typedef typename cplx_of<R>::type Z;
    static constexpr bool pairs = false;
    // resident 256-thread CTAs per SM asked of the register allocator
    static constexpr int min_blocks = sizeof(R) == 8 ? 3 : 5;
    // how much of the next phase's once-read data the sweep prefetches into L1
    static constexpr int l1_prefetch = sizeof(R) == 8 ? 2 : 1;
    __device__ static __forceinline__ Z zero() { Z z; z.x = R(0); z.y = R(0); return z; }
    __device__ static __forceinline__ Z ld_field(const void *b, size_t i) { return ldg_as<Z>(b, i); }
    __device__ static __forceinline__ Z ld_field_hint(const void *b, size_t i, uint64_t pol) {
        return ldg_hint<Z>(b, i, pol);
    }
    __device__ static __forceinline__ Z ld_coef(const void *b, size_t i) { return ldg_as<Z>(b, i); }
    __device__ static __forceinline__ void st_field(void *b, size_t i, Z v) { stg_as<Z>(b, i, v); }
    __device__ static __forceinline__ Z add(Z a, Z b) { Z r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
    __device__ static __forceinline__ Z sub(Z a, Z b) { Z r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
    // t*x + s + c*d (d carries the curl sign)
    __device__ static __forceinline__ Z upd_src(Z x, Z t, Z c, Z d, Z s) {
        Z r;
        r.x = fma(t.x, x.x, s.x); r.x = fma(-t.y, x.y, r.x); r.x = fma(c.x, d.x, r.x); r.x = fma(-c.y, d.y, r.x);
        r.y = fma(t.x, x.y, s.y); r.y = fma(t.y, x.x, r.y); r.y = fma(c.x, d.y, r.y); r.y = fma(c.y, d.x, r.y);
        return r;
    }
    __device__ static __forceinline__ Z upd(Z x, Z t, Z c, Z d) {
        Z r;
        r.x = t.x * x.x; r.x = fma(-t.y, x.y, r.x); r.x = fma(c.x, d.x, r.x); r.x = fma(-c.y, d.y, r.x);
        r.y = t.x * x.y; r.y = fma(t.y, x.x, r.y); r.y = fma(c.x, d.y, r.y); r.y = fma(c.y, d.x, r.y);
        return r;
    }
    __device__ static __forceinline__ double re(Z a) { return (double)a.x; }
    __device__ static __forceinline__ double im(Z a) { return (double)a.y; }
    // residual norms: FP64 sums of the three components' terms
    typedef double Acc;
    __device__ static __forceinline__ Acc acc_zero() { return 0.0; }
    __device__ static __forceinline__ double acc_value(Acc a) { return a; }
    __device__ static __forceinline__ double d2(Z a, Z b) {
        const double x = re(a) - re(b), y = im(a) - im(b);
        return x * x + y * y;
    }
    __device__ static __forceinline__ double n2(Z a) { const double x = re(a), y = im(a); return x * x + y * y; }
    __device__ static __forceinline__ void acc_d3(Acc &acc, Z a0, Z b0, Z a1, Z b1, Z a2, Z b2) {
        acc += d2(a0, b0) + d2(a1, b1) + d2(a2, b2);
    }
    __device__ static __forceinline__ void acc_n3(Acc &acc, Z a0, Z a1, Z a2) { acc += n2(a0) + n2(a1) + n2(a2); }
};

// ------------------------------------------- FP64 with integer-pipe ops ----
// The FP64 sweep issues about 145 FP64-pipe instructions per cell (132 without
// the halo): 86 fused multiply-adds, 41 additions (full-field sums and
// differences) and 18 multiplications (the leading product t*x of the updates
// without a source term).  GB300's FP64 pipe retires ~1.7 of them per SM and
// clock, its integer units 64-128.  OFF selects which operations run as
// integer-pipe binary64 arithmetic instead (thiim_i64f.cuh; bit 0: additions
// and subtractions, bit 2: the additions of the full-field sums only (A::add,
// not the differences A::sub), bit 1: the leading products); the fused
// multiply-adds stay on the FP64 pipe.  Every operation keeps its IEEE result, and the order of
// operations is Native<double>'s, so the results are bit-identical to it.
// Measured on GB300 it does not pay: an integer addition takes ~75 integer
// instructions (twice the pipe time of the FP64 instruction it replaces, in a
// pipe shared with the sweep's address and index work).  With the additions
// on the integer pipe the FP64-pipe cycles drop 28 % but the 512^3 sweep runs
// at 3621 against 3610 MLUP/s on the FP64 pipe alone (32 x 16 tiles), and
// with only the full-field sums there (bit 2) at 3533; the multiplications'
// rare-case fallback to the FP64 pipe is evaluated unconditionally by the
// compiler, so bit 1 saves nothing.  It stays as an option (off by default).
template <int OFF>
struct Fp64Int : Native<double> {
    static constexpr int min_blocks = 2;
    __device__ static __forceinline__ double dadd(double a, double b) {
        return (OFF & 5) ? i64f::add(a, b) : __dadd_rn(a, b);
    }
    __device__ static __forceinline__ double dsub(double a, double b) {
        return (OFF & 1) ? i64f::sub(a, b) : __dsub_rn(a, b);
    }
    __device__ static __forceinline__ double dmul(double a, double b) {
        return (OFF & 2) ? i64f::mul(a, b) : __dmul_rn(a, b);
    }
    __device__ static __forceinline__ Z add(Z a, Z b) { Z r; r.x = dadd(a.x, b.x); r.y = dadd(a.y, b.y); return r; }
    __device__ static __forceinline__ Z sub(Z a, Z b) { Z r; r.x = dsub(a.x, b.x); r.y = dsub(a.y, b.y); return r; }
    __device__ static __forceinline__ Z upd_src(Z x, Z t, Z c, Z d, Z s) {
        Z r;
        r.x = __fma_rn(t.x, x.x, s.x); r.x = __fma_rn(-t.y, x.y, r.x);
        r.x = __fma_rn(c.x, d.x, r.x); r.x = __fma_rn(-c.y, d.y, r.x);
        r.y = __fma_rn(t.x, x.y, s.y); r.y = __fma_rn(t.y, x.x, r.y);
        r.y = __fma_rn(c.x, d.y, r.y); r.y = __fma_rn(c.y, d.x, r.y);
        return r;
    }
    __device__ static __forceinline__ Z upd(Z x, Z t, Z c, Z d) {
        Z r;
        r.x = dmul(t.x, x.x); r.x = __fma_rn(-t.y, x.y, r.x);
        r.x = __fma_rn(c.x, d.x, r.x); r.x = __fma_rn(-c.y, d.y, r.x);
        r.y = dmul(t.x, x.y); r.y = __fma_rn(t.y, x.x, r.y);
        r.y = __fma_rn(c.x, d.y, r.y); r.y = __fma_rn(c.y, d.x, r.y);
        return r;
    }
};

// ------------------------------------------------------------ FP32 pairs ----
struct fpair { float h, l; };
struct zpair { fpair x, y; };   // complex: real pair, imaginary pair

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// a + b, leading part exact, error part not renormalised
__device__ __forceinline__ fpair p_add(fpair a, fpair b) {
    fpair r;
    float e;
    two_sum(a.h, b.h, r.h, e);
    r.l = e + (a.l + b.l);
    return r;
}
__device__ __forceinline__ fpair p_sub(fpair a, fpair b) {
    fpair r;
    float e;
    two_sum(a.h, -b.h, r.h, e);
    r.l = e + (a.l - b.l);
    return r;
}

// Accumulates a sum of products of pairs: leading parts exactly (two_sum),
// error parts in plain FP32.
struct pacc {
    float s, lo;
    __device__ __forceinline__ void first(float ah, float al, float bh, float bl) {
        s = ah * bh;
        lo = fmaf(ah, bh, -s);
        lo = fmaf(ah, bl, lo);
        lo = fmaf(al, bh, lo);
    }
    __device__ __forceinline__ void prod(float ah, float al, float bh, float bl) {
        const float p = ah * bh;
        float e = fmaf(ah, bh, -p);
        e = fmaf(ah, bl, e);
        e = fmaf(al, bh, e);
        float t;
        two_sum(s, p, s, t);
        lo += t + e;
    }
    __device__ __forceinline__ void term(fpair v) {
        float t;
        two_sum(s, v.h, s, t);
        lo += t + v.l;
    }
    __device__ __forceinline__ fpair result() const {   // renormalised
        fpair r;
        r.h = s + lo;
        r.l = lo - (r.h - s);
        return r;
    }
};

__device__ __forceinline__ fpair split_double(double d) {
    fpair r;
    r.h = __double2float_rn(d);
    r.l = __double2float_rn(d - (double)r.h);
    return r;
}

template <int IN_PAIRS, int OUT_PAIRS>
struct PairArith {
    typedef zpair Z;
    static constexpr bool pairs = true;
    static constexpr int min_blocks = 2;
    static constexpr int l1_prefetch = 2;
    __device__ static __forceinline__ Z zero() { Z z; z.x.h = z.x.l = z.y.h = z.y.l = 0.f; return z; }
    __device__ static __forceinline__ Z from_f4(float4 v) { Z z; z.x.h = v.x; z.x.l = v.y; z.y.h = v.z; z.y.l = v.w; return z; }
    __device__ static __forceinline__ Z ld_field(const void *b, size_t i) {
        if (IN_PAIRS) return from_f4(ldg_as<float4>(b, i));
        const double2 v = ldg_as<double2>(b, i);
        Z z; z.x = split_double(v.x); z.y = split_double(v.y);
        return z;
    }
    __device__ static __forceinline__ Z ld_field_hint(const void *b, size_t i, uint64_t pol) {
        if (IN_PAIRS) return from_f4(ldg_hint<float4>(b, i, pol));
        const double2 v = ldg_hint<double2>(b, i, pol);
        Z z; z.x = split_double(v.x); z.y = split_double(v.y);
        return z;
    }
    __device__ static __forceinline__ Z ld_coef(const void *b, size_t i) { return from_f4(ldg_as<float4>(b, i)); }
    __device__ static __forceinline__ void st_field(void *b, size_t i, Z v) {
        if (OUT_PAIRS) {
            stg_as<float4>(b, i, make_float4(v.x.h, v.x.l, v.y.h, v.y.l));
        } else {
            stg_as<double2>(b, i, make_double2(re(v), im(v)));
        }
    }
    __device__ static __forceinline__ Z add(Z a, Z b) { Z r; r.x = p_add(a.x, b.x); r.y = p_add(a.y, b.y); return r; }
    __device__ static __forceinline__ Z sub(Z a, Z b) { Z r; r.x = p_sub(a.x, b.x); r.y = p_sub(a.y, b.y); return r; }
    // t*x + s + c*d: real = tr xr - ti xi + cr dr - ci di (+ sr); imag = tr xi + ti xr + cr di + ci dr (+ si)
    __device__ static __forceinline__ Z upd_impl(Z x, Z t, Z c, Z d, const Z *s) {
        pacc r, q;
        r.first(t.x.h, t.x.l, x.x.h, x.x.l);
        r.prod(-t.y.h, -t.y.l, x.y.h, x.y.l);
        r.prod(c.x.h, c.x.l, d.x.h, d.x.l);
        r.prod(-c.y.h, -c.y.l, d.y.h, d.y.l);
        q.first(t.x.h, t.x.l, x.y.h, x.y.l);
        q.prod(t.y.h, t.y.l, x.x.h, x.x.l);
        q.prod(c.x.h, c.x.l, d.y.h, d.y.l);
        q.prod(c.y.h, c.y.l, d.x.h, d.x.l);
        if (s) { r.term(s->x); q.term(s->y); }
        Z z; z.x = r.result(); z.y = q.result();
        return z;
    }
    __device__ static __forceinline__ Z upd_src(Z x, Z t, Z c, Z d, Z s) { return upd_impl(x, t, c, d, &s); }
    __device__ static __forceinline__ Z upd(Z x, Z t, Z c, Z d) { return upd_impl(x, t, c, d, nullptr); }
    __device__ static __forceinline__ double re(Z a) { return (double)a.x.h + (double)a.x.l; }
    __device__ static __forceinline__ double im(Z a) { return (double)a.y.h + (double)a.y.l; }
    // residual norms: squares and sums in pair arithmetic on the FP32 pipe (the
    // per-thread sum keeps ~48 bits); converted to FP64 once per thread
    typedef pacc Acc;
    __device__ static __forceinline__ Acc acc_zero() { Acc a; a.s = 0.f; a.lo = 0.f; return a; }
    __device__ static __forceinline__ double acc_value(Acc a) { return (double)a.s + (double)a.lo; }
    __device__ static __forceinline__ void acc_sq(Acc &acc, fpair v) { acc.prod(v.h, v.l, v.h, v.l); }
    __device__ static __forceinline__ void acc_d3(Acc &acc, Z a0, Z b0, Z a1, Z b1, Z a2, Z b2) {
        acc_sq(acc, p_sub(a0.x, b0.x)); acc_sq(acc, p_sub(a0.y, b0.y));
        acc_sq(acc, p_sub(a1.x, b1.x)); acc_sq(acc, p_sub(a1.y, b1.y));
        acc_sq(acc, p_sub(a2.x, b2.x)); acc_sq(acc, p_sub(a2.y, b2.y));
    }
    __device__ static __forceinline__ void acc_n3(Acc &acc, Z a0, Z a1, Z a2) {
        acc_sq(acc, a0.x); acc_sq(acc, a0.y); acc_sq(acc, a1.x); acc_sq(acc, a1.y);
        acc_sq(acc, a2.x); acc_sq(acc, a2.y);
    }
};

}  // namespace thiim
