// host_math.h -- host-side number theory and high-precision constants for the
// RNS-CKKS library: prime chains, primitive roots, Shoup quotients, the
// discrete-Gaussian table and double-double roots of unity for the encoder.
#pragma once
#include <cstdint>
#include <vector>

namespace fhe {

typedef unsigned __int128 u128;
typedef unsigned long long u64;

u64 hmul(u64 a, u64 b, u64 q);
u64 hpow(u64 a, u64 e, u64 q);
u64 hinv(u64 a, u64 q);                       // q prime
u64 shoup(u64 w, u64 q);                      // floor(w 2^64 / q)
bool is_prime64(u64 n);

// Primes q > 2^b, q = 1 (mod 2N), increasing; a repeated bit size takes the
// next prime of that size.  Returns false if a size is out of range.
bool prime_chain(uint32_t N, const uint32_t* bits, uint32_t n_bits, std::vector<u64>& out);

// primitive 2N-th root of unity mod q (the smallest base whose power works)
u64 primitive_root_2n(u64 q, uint32_t N);

uint32_t bitrev(uint32_t x, int bits);

// Discrete Gaussian table: support [-19, 19], sigma = 3.2 exactly (2 sigma^2 =
// 512/25), thresholds T_i = floor(2^64 * CDF(-19 + i)), i = 0..37, evaluated
// in double-double arithmetic.
std::vector<u64> gauss_cdt();
constexpr int kGaussKmax = 19;

// double-double number and zeta^e = exp(i pi e / N) with both parts in dd
struct dd { double hi, lo; };
struct cdd { dd re, im; };
cdd zeta_pow_dd(int64_t e, uint32_t N);

// v = hi + lo (|v| <= 2) as a sign-magnitude fixed-point number with 126
// fractional bits: magnitude = (*hi & ~2^63) 2^64 + *lo, sign = bit 63 of *hi
// (truncated toward zero, error below 2^-126)
void dd_to_q126(dd v, u64* lo, u64* hi);

// Alg. parameterise: cost c, scale power s, special-prime multiplier p
void parameterise(uint32_t c, uint32_t s, double p, uint32_t* N, std::vector<uint32_t>& bits);

}  // namespace fhe
