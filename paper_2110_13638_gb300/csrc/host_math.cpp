// host_math.cpp -- see host_math.h.  Compiled with -ffp-contract=off so the
// double-double algorithms (Dekker / Knuth error-free transformations) round
// the same way on every host.
#include "host_math.h"

#include <cmath>

namespace fhe {

u64 hmul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 hpow(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = hmul(r, a, q);
        a = hmul(a, a, q);
    }
    return r;
}

u64 hinv(u64 a, u64 q) { return hpow(a % q, q - 2, q); }

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

bool is_prime64(u64 n)
{
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; ++r; }
    for (u64 a : bases) {
        u64 x = hpow(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; ++i) {
            x = hmul(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

bool prime_chain(uint32_t N, const uint32_t* bits, uint32_t n_bits, std::vector<u64>& out)
{
    out.clear();
    const u64 step = 2ull * N;
    for (uint32_t i = 0; i < n_bits; ++i) {
        const uint32_t b = bits[i];
        if (b < 20 || b > 61) return false;
        // how many earlier entries share this size: take that many primes first
        uint32_t skip = 0;
        for (uint32_t k = 0; k < i; ++k) skip += (bits[k] == b);
        u64 lo = 1ull << b;
        u64 c = (lo / step) * step + 1;
        if (c <= lo) c += step;
        for (;; c += step) {
            if (c >= (1ull << 62)) return false;
            if (is_prime64(c)) {
                if (skip == 0) break;
                --skip;
            }
        }
        out.push_back(c);
    }
    return true;
}

u64 primitive_root_2n(u64 q, uint32_t N)
{
    for (u64 x = 2;; ++x) {
        u64 g = hpow(x, (q - 1) / (2ull * N), q);
        if (hpow(g, N, q) == q - 1) return g;
    }
}

uint32_t bitrev(uint32_t x, int bits)
{
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

// ---------------------------------------------------------------- double-double
static inline dd two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

static inline dd fast_two_sum(double a, double b)
{
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}

static inline dd two_prod(double a, double b)
{
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}

static inline dd dd_add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

static inline dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

static inline dd dd_mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}

static inline dd dd_div(dd a, dd b)
{
    double q1 = a.hi / b.hi;
    dd r = dd_add(a, dd_neg(dd_mul(b, {q1, 0.0})));
    double q2 = r.hi / b.hi;
    r = dd_add(r, dd_neg(dd_mul(b, {q2, 0.0})));
    double q3 = r.hi / b.hi;
    return dd_add(fast_two_sum(q1, q2), {q3, 0.0});
}

// exp(x) for |x| <= 32: Taylor series of exp(x / 2^10), then 10 squarings
static dd dd_exp(dd x)
{
    dd y = {std::ldexp(x.hi, -10), std::ldexp(x.lo, -10)};
    dd sum = {1.0, 0.0}, term = {1.0, 0.0};
    for (int n = 1; n <= 20; ++n) {
        term = dd_div(dd_mul(term, y), {(double)n, 0.0});
        sum = dd_add(sum, term);
    }
    for (int i = 0; i < 10; ++i) sum = dd_mul(sum, sum);
    return sum;
}

std::vector<u64> gauss_cdt()
{
    const int K = kGaussKmax;
    std::vector<dd> rho;
    dd S = {0.0, 0.0};
    for (int k = -K; k <= K; ++k) {
        // k^2 / (2 sigma^2) with sigma = 16/5: 25 k^2 / 512, exact in double
        dd x = {-(25.0 * k * k) / 512.0, 0.0};
        dd r = dd_exp(x);
        rho.push_back(r);
    }
    for (const dd& r : rho) S = dd_add(S, r);
    std::vector<u64> T;
    dd acc = {0.0, 0.0};
    for (int i = 0; i < 2 * K; ++i) {
        acc = dd_add(acc, rho[i]);
        dd f = dd_div(acc, S);
        dd v = {std::ldexp(f.hi, 64), std::ldexp(f.lo, 64)};
        // floor of a double-double below 2^64: hi is an integer here (ulp >= 1
        // once hi >= 2^53; smaller hi are handled by the same formula)
        double fh = std::floor(v.hi);
        double rest = (v.hi - fh) + v.lo;          // fractional remainder, |rest| < 2
        double fr = std::floor(rest);
        u64 base = (u64)fh;
        int64_t adj = (int64_t)fr;
        T.push_back(base + (u64)adj);
    }
    return T;
}

// ---------------------------------------------------------------- roots
static const dd kPi = {3.141592653589793116e+00, 1.224646799147353207e-16};

static void dd_sincos(dd t, dd* s, dd* c)
{
    // Taylor series, |t| <= pi/4
    dd t2 = dd_mul(t, t);
    dd term = t;                 // t^(2n+1)/(2n+1)!
    dd ss = t;
    for (int n = 1; n <= 15; ++n) {
        term = dd_div(dd_mul(term, t2), {(double)((2 * n) * (2 * n + 1)), 0.0});
        ss = (n & 1) ? dd_add(ss, dd_neg(term)) : dd_add(ss, term);
    }
    term = {1.0, 0.0};
    dd cc = {1.0, 0.0};
    for (int n = 1; n <= 15; ++n) {
        term = dd_div(dd_mul(term, t2), {(double)((2 * n - 1) * (2 * n)), 0.0});
        cc = (n & 1) ? dd_add(cc, dd_neg(term)) : dd_add(cc, term);
    }
    *s = ss;
    *c = cc;
}

cdd zeta_pow_dd(int64_t e, uint32_t N)
{
    const int64_t M = 2 * (int64_t)N;
    int64_t idx = e % M;
    if (idx < 0) idx += M;
    const int64_t oct = N / 4;                       // N >= 4
    const int64_t o = idx / oct, rem = idx % oct;
    // theta = pi * rem / N, theta' = pi * (oct - rem) / N, both in [0, pi/4]
    dd th = dd_mul(kPi, {(double)rem / (double)N, 0.0});
    dd thp = dd_mul(kPi, {(double)(oct - rem) / (double)N, 0.0});
    dd s, c, sp, cp;
    dd_sincos(th, &s, &c);
    dd_sincos(thp, &sp, &cp);
    cdd r;
    switch (o) {
    case 0: r.re = c; r.im = s; break;
    case 1: r.re = sp; r.im = cp; break;
    case 2: r.re = dd_neg(s); r.im = c; break;
    case 3: r.re = dd_neg(cp); r.im = sp; break;
    case 4: r.re = dd_neg(c); r.im = dd_neg(s); break;
    case 5: r.re = dd_neg(sp); r.im = dd_neg(cp); break;
    case 6: r.re = s; r.im = dd_neg(c); break;
    default: r.re = cp; r.im = dd_neg(sp); break;
    }
    return r;
}

// d 2^126 truncated toward zero, |d| <= 2
static __int128 scaled_q126(double d)
{
    if (d == 0.0) return 0;
    int e = 0;
    const double m = std::frexp(std::fabs(d), &e);         // |d| = m 2^e, m in [0.5, 1)
    const u64 M = (u64)std::ldexp(m, 53);                   // exact
    const int sh = e - 53 + 126;
    u128 v = 0;
    if (sh >= 0) v = (u128)M << sh;
    else if (sh > -64) v = (u128)(M >> -sh);
    return d < 0.0 ? -(__int128)v : (__int128)v;
}

void dd_to_q126(dd v, u64* lo, u64* hi)
{
    const __int128 t = scaled_q126(v.hi) + scaled_q126(v.lo);
    const u128 mag = t < 0 ? (u128)(-t) : (u128)t;
    *lo = (u64)mag;
    *hi = (u64)(mag >> 64) | (t < 0 ? (1ull << 63) : 0ull);
}

void parameterise(uint32_t c, uint32_t s, double p, uint32_t* N, std::vector<uint32_t>& bits)
{
    bits.assign(c + 2, s);
    bits.front() = (uint32_t)(bits.front() * p);
    bits.back() = (uint32_t)(bits.back() * p);
    uint64_t sum = 0;
    for (uint32_t b : bits) sum += b;
    uint64_t b = 27;
    while (b < sum) b *= 2;
    *N = (uint32_t)(1024 * (b / 27));
}

}  // namespace fhe
