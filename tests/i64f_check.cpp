// Bit-for-bit check of the integer-pipe binary64 add / sub / mul
// (paper_1510_05218_gb300/csrc/thiim_i64f.cuh) against the host's IEEE 754
// double arithmetic (round to nearest even).  Built and run by
// tests/test_i64f.py.  Prints one line per case family:
//   <family> <cases> <integer-path hits> <mismatches>
// and exits 1 on any mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "thiim_i64f.cuh"

using namespace thiim::i64f;

static uint64_t g_state = 0x9E3779B97F4A7C15ull;

// splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014)
static uint64_t next() {
    uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double mk(uint64_t sign, uint64_t exp, uint64_t frac) {
    return from_bits((sign << 63) | ((exp & 0x7FF) << 52) | (frac & FRAC));
}

// NaN results compare as equal whatever their payload where the payload is
// not defined alike everywhere (two NaN operands; products, whose rare cases
// use the host's own instruction).
static bool same(double x, double y) {
    if (std::isnan(x) && std::isnan(y)) return true;
    return bits(x) == bits(y);
}

// Sums: exact bits; a NaN result only as NaN (IEEE 754 leaves the sign and
// payload of a propagated NaN open, and a - NaN keeps the operand's sign on
// the host but not after the negation the subtraction applies here).
static bool same_sum(double x, double y, double, double) {
    return same(x, y);
}

struct Tally {
    long cases = 0, hits = 0, bad = 0;
};

static void check(Tally &t, double a, double b, bool do_add, bool do_mul) {
    if (do_add) {   // the integer sum covers every operand pair: no fallback
        volatile double ref = a + b;
        const double got = from_bits(add_bits(bits(a), bits(b)));
        t.cases++;
        t.hits++;
        if (!same_sum(got, ref, a, b) || !same_sum(add(a, b), ref, a, b)) {
            if (t.bad++ < 5) printf("MISMATCH add %a + %a: got %a ref %a\n", a, b, got, (double)ref);
        }
        volatile double ref2 = a - b;
        const double got2 = from_bits(add_bits(bits(a), bits(b) ^ SIGN));
        t.cases++;
        t.hits++;
        if (!same_sum(got2, ref2, a, b) || !same_sum(sub(a, b), ref2, a, b)) {
            if (t.bad++ < 5) printf("MISMATCH sub %a - %a: got %a ref %a\n", a, b, got2, (double)ref2);
        }
    }
    if (do_mul) {
        volatile double ref = a * b;
        const Res r = mul_int(bits(a), bits(b));
        const double got = mul(a, b);
        t.cases++;
        t.hits += r.ok;
        if (!same(got, ref) || (r.ok && !same(from_bits(r.v), ref))) {
            if (t.bad++ < 5)
                printf("MISMATCH mul %a * %a: got %a ref %a (int path %d)\n", a, b, got, (double)ref, (int)r.ok);
        }
    }
}

static double special(uint64_t k) {
    switch (k % 10) {
        case 0: return 0.0;
        case 1: return -0.0;
        case 2: return INFINITY;
        case 3: return -INFINITY;
        case 4: return NAN;
        case 5: return mk(next() & 1, 0, next());          // subnormal
        case 6: return mk(next() & 1, 1, next());          // smallest normals
        case 7: return mk(next() & 1, 2046, next());       // largest normals
        case 8: return mk(next() & 1, 0, 1);               // smallest subnormal
        default: return mk(next() & 1, 1023, next());     // ordinary
    }
}

int main(int argc, char **argv) {
    const long n = argc > 1 ? atol(argv[1]) : 1000000;
    int fail = 0;
    auto report = [&](const char *name, const Tally &t) {
        printf("%s %ld %ld %ld\n", name, t.cases, t.hits, t.bad);
        if (t.bad) fail = 1;
    };
    {   // arbitrary bit patterns: every exponent, mostly far apart
        Tally t;
        for (long i = 0; i < n; ++i) check(t, from_bits(next()), from_bits(next()), true, true);
        report("random_bits", t);
    }
    {   // close exponents: alignment by 0..60 bits, carries and cancellation
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t ea = 900 + next() % 250;
            const uint64_t eb = ea - (next() % 61) + (next() % 3);
            check(t, mk(next() & 1, ea, next()), mk(next() & 1, eb, next()), true, true);
        }
        report("close_exponents", t);
    }
    {   // massive cancellation: b differs from -a in a few low bits or exponents
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t e = 1 + next() % 2046;
            const uint64_t f = next();
            const uint64_t g = (next() & 3) ? (f ^ (next() & ((1ull << (next() % 53)) - 1))) : next();
            const uint64_t e2 = (next() & 1) ? e : (e > 1 ? e - 1 : e);
            check(t, mk(0, e, f), mk(1, e2, g), true, false);
        }
        report("cancellation", t);
    }
    {   // exact ties of the sum: b is half an ulp of a (times an odd factor)
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t e = 60 + next() % 1900;
            const double a = mk(next() & 1, e, next());
            const double b = mk(next() & 1, e - 53 - (next() % 3), (next() & 1) ? 0 : (next() & 0xFF) << 44);
            check(t, a, b, true, false);
        }
        report("add_ties", t);
    }
    {   // products with short significands: exact results and ties
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t e = 700 + next() % 600;
            const uint64_t short_frac = (next() & 0xF) << 48;                // 1.xxxx
            check(t, mk(next() & 1, e, next()), mk(next() & 1, 2046 - e + (next() % 3), short_frac), false, true);
        }
        report("mul_short", t);
    }
    {   // products near the top and bottom of the normal range
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t ea = 1 + next() % 2046;
            const uint64_t eb = (3069 - ea + (next() % 5) - 2) % 2047;      // sum near 2046 (overflow edge)
            const uint64_t ec = (1023 + 1 - ea + 2046 + (next() % 5) - 2) % 2047;   // sum near 1 (underflow edge)
            check(t, mk(next() & 1, ea, next()), mk(next() & 1, eb, next()), true, true);
            check(t, mk(next() & 1, ea, next()), mk(next() & 1, ec, next()), true, true);
        }
        report("range_edges", t);
    }
    {   // sums near overflow: carries into the top exponent
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t f = FRAC - (next() & 0xFFFF);
            check(t, mk(next() & 1, 2046, f), mk(next() & 1, 2046 - next() % 60, next()), true, false);
        }
        report("add_overflow", t);
    }
    {   // specials mixed with ordinary values
        Tally t;
        for (long i = 0; i < n / 10 + 100; ++i) {
            check(t, special(next()), special(next()), true, true);
            check(t, special(next()), mk(next() & 1, 1 + next() % 2046, next()), true, true);
            check(t, mk(next() & 1, 1 + next() % 2046, next()), special(next()), true, true);
        }
        report("specials", t);
    }
    {   // the sweep's value range: O(1) fields and coefficients, exponents within +-40
        Tally t;
        for (long i = 0; i < n; ++i) {
            const uint64_t ea = 1023 - 40 + next() % 44, eb = 1023 - 40 + next() % 44;
            check(t, mk(next() & 1, ea, next()), mk(next() & 1, eb, next()), true, true);
        }
        report("sweep_range", t);
    }
    return fail;
}
