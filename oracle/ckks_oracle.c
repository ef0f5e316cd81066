/*
 * ckks_oracle.c -- arithmetic core of the plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant generator with
 * the CUDA library under paper_2110_13638_gb300/csrc.
 *
 * What it computes (arXiv 2110.13638 evaluates graphs through MS-SEAL's RNS-CKKS,
 * Sec. 2.1 "FHE Background" and Sec. 3; the paper prints none of the ring
 * arithmetic, so each routine below is the textbook definition):
 *   - modular arithmetic with exact 128-bit products reduced by '%';
 *   - the negacyclic NTT over Z_q[X]/(X^N+1) written as "twist by psi^i, then
 *     a radix-2 cyclic DFT with omega = psi^2", plus the O(N^2) schoolbook
 *     negacyclic product that pins it;
 *   - the counter-based SplitMix64 sampling spec (uniform mod q by rejection,
 *     ternary by rejection, discrete Gaussian by a cumulative table passed in);
 *   - the canonical-embedding encode/decode of CKKS in IEEE binary128
 *     (x86-64: __float128 + libquadmath; aarch64: long double).
 * Every loop is the plain definition; no blocking, fusion or reordering.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Modular arithmetic (exact: 128-bit product, then remainder).        */
/* ------------------------------------------------------------------ */
u64 o_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * (u128)b) % q); }
u64 o_addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + (u128)b) % q); }
u64 o_submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + (u128)q - (u128)(b % q)) % q); }

u64 o_powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = o_mulmod(r, a, q);
        a = o_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* a[i] = a[i] * c mod q */
void o_vec_mul_scalar(u64* a, size_t n, u64 c, u64 q)
{
    for (size_t i = 0; i < n; ++i) a[i] = o_mulmod(a[i], c, q);
}

/* c[i] = a[i] * b[i] mod q */
void o_vec_mul(const u64* a, const u64* b, u64* c, size_t n, u64 q)
{
    for (size_t i = 0; i < n; ++i) c[i] = o_mulmod(a[i], b[i], q);
}

/* acc[i] = (acc[i] + a[i] * c) mod q   (a multiply-accumulate by one scalar) */
void o_vec_mac_scalar(u64* acc, const u64* a, size_t n, u64 c, u64 q)
{
    for (size_t i = 0; i < n; ++i) acc[i] = (u64)(((u128)acc[i] + (u128)a[i] * c) % q);
}

/* ------------------------------------------------------------------ */
/* Negacyclic number-theoretic transform.                              */
/*   forward:  A_k = sum_i a_i psi^{(2k+1) i},  k = 0..N-1 (natural)   */
/*   inverse:  a_i = N^{-1} psi^{-i} sum_k A_k psi^{-2ik}              */
/* psi is a primitive 2N-th root of unity mod q.                       */
/* ------------------------------------------------------------------ */
static void bit_reverse(u64* a, uint32_t N)
{
    for (uint32_t i = 1, j = 0; i < N; ++i) {
        uint32_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* cyclic DFT in place: A_k = sum_i a_i w^{ik} (iterative radix-2, DIT) */
static void cyclic_dft(u64* a, uint32_t N, u64 q, u64 w)
{
    bit_reverse(a, N);
    for (uint32_t len = 2; len <= N; len <<= 1) {
        u64 wl = o_powmod(w, N / len, q);          /* primitive len-th root */
        for (uint32_t i = 0; i < N; i += len) {
            u64 x = 1;
            for (uint32_t j = 0; j < len / 2; ++j) {
                u64 u = a[i + j];
                u64 v = o_mulmod(a[i + j + len / 2], x, q);
                a[i + j] = o_addmod(u, v, q);
                a[i + j + len / 2] = o_submod(u, v, q);
                x = o_mulmod(x, wl, q);
            }
        }
    }
}

void o_ntt(u64* a, uint32_t N, u64 q, u64 psi)
{
    u64 x = 1;
    for (uint32_t i = 0; i < N; ++i) { a[i] = o_mulmod(a[i], x, q); x = o_mulmod(x, psi, q); }
    cyclic_dft(a, N, q, o_mulmod(psi, psi, q));
}

void o_intt(u64* a, uint32_t N, u64 q, u64 psi)
{
    u64 psi_inv = o_powmod(psi, q - 2, q);
    cyclic_dft(a, N, q, o_mulmod(psi_inv, psi_inv, q));
    u64 n_inv = o_powmod(N % q, q - 2, q);
    u64 x = n_inv;
    for (uint32_t i = 0; i < N; ++i) { a[i] = o_mulmod(a[i], x, q); x = o_mulmod(x, psi_inv, q); }
}

/* c = a * b in Z_q[X]/(X^N+1), through the transform (c may alias a or b) */
void o_polymul(const u64* a, const u64* b, u64* c, uint32_t N, u64 q, u64 psi)
{
    u64* fa = (u64*)malloc(sizeof(u64) * N);
    u64* fb = (u64*)malloc(sizeof(u64) * N);
    memcpy(fa, a, sizeof(u64) * N);
    memcpy(fb, b, sizeof(u64) * N);
    o_ntt(fa, N, q, psi);
    o_ntt(fb, N, q, psi);
    for (uint32_t k = 0; k < N; ++k) fa[k] = o_mulmod(fa[k], fb[k], q);
    o_intt(fa, N, q, psi);
    memcpy(c, fa, sizeof(u64) * N);
    free(fa);
    free(fb);
}

/* c = a * b in Z_q[X]/(X^N+1) by the O(N^2) definition: X^N = -1 */
void o_polymul_schoolbook(const u64* a, const u64* b, u64* c, uint32_t N, u64 q)
{
    u64* r = (u64*)calloc(N, sizeof(u64));
    for (uint32_t i = 0; i < N; ++i)
        for (uint32_t j = 0; j < N; ++j) {
            u64 p = o_mulmod(a[i], b[j], q);
            uint32_t k = i + j;
            if (k < N) r[k] = o_addmod(r[k], p, q);
            else r[k - N] = o_submod(r[k - N], p, q);
        }
    memcpy(c, r, sizeof(u64) * N);
    free(r);
}

/* ------------------------------------------------------------------ */
/* Sampling spec (the paper is silent; SEAL's defaults are assumed:    */
/* ternary secret, discrete Gaussian sigma = 3.2).                      */
/*   SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the i-th output of    */
/*   the generator started in state s is mix64(s + (i+1) * GAMMA).      */
/*   stream(seed, domain, object) = out(out(seed, domain), object)       */
/*   draw index i = coef | residue << 16 | retry << 24                   */
/* ------------------------------------------------------------------ */
#define SM_GAMMA 0x9E3779B97F4A7C15ull

static u64 mix64(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

u64 o_splitmix_out(u64 state, u64 i) { return mix64(state + (i + 1) * SM_GAMMA); }

u64 o_stream(u64 seed, u64 domain, u64 object)
{
    return o_splitmix_out(o_splitmix_out(seed, domain), object);
}

static u64 draw(u64 s0, uint32_t coef, uint32_t residue, u64 retry)
{
    return o_splitmix_out(s0, (u64)coef | ((u64)residue << 16) | (retry << 24));
}

/* uniform in [0, q): reject u >= floor(2^64 / q) * q, then reduce */
void o_sample_uniform(u64 s0, uint32_t residue, u64 q, uint32_t N, u64* out)
{
    u64 bound = (u64)((((u128)1 << 64) / q) * q);
    for (uint32_t c = 0; c < N; ++c) {
        for (u64 t = 0;; ++t) {
            u64 u = draw(s0, c, residue, t);
            if (u < bound) { out[c] = u % q; break; }
        }
    }
}

/* ternary in {-1, 0, 1}: reject u >= floor(2^64 / 3) * 3, then (u mod 3) - 1 */
void o_sample_ternary(u64 s0, uint32_t N, i64* out)
{
    u64 bound = (u64)((((u128)1 << 64) / 3) * 3);
    for (uint32_t c = 0; c < N; ++c) {
        for (u64 t = 0;; ++t) {
            u64 u = draw(s0, c, 0, t);
            if (u < bound) { out[c] = (i64)(u % 3) - 1; break; }
        }
    }
}

/* discrete Gaussian on [-kmax, kmax]: one 64-bit draw u; the value is
 * -kmax + #{i : u >= cdt[i]} over the 2*kmax cumulative thresholds cdt[]. */
void o_sample_gauss(u64 s0, uint32_t N, const u64* cdt, uint32_t kmax, i64* out)
{
    for (uint32_t c = 0; c < N; ++c) {
        u64 u = draw(s0, c, 0, 0);
        i64 e = -(i64)kmax;
        for (uint32_t i = 0; i < 2 * kmax; ++i)
            if (u >= cdt[i]) e += 1;
        out[c] = e;
    }
}

/* ------------------------------------------------------------------ */
/* CKKS canonical embedding in binary128.                              */
/* Slot j lives at zeta_j = zeta^{5^j mod 2N}, zeta = exp(i pi / N).   */
/* decode: z_j = (1/scale) * m(zeta_j) = (1/scale) sum_k m_k zeta_j^k   */
/* encode: m_k = round(scale * (1/N) * sum_{l} M_l zeta^{-(2l+1)k}),    */
/*   M_l = m(zeta^{2l+1}) with M at 5^j = z_j and at -5^j = conj(z_j). */
/* Both are an N-point complex DFT of the twisted sequence m_k zeta^k.  */
/* ------------------------------------------------------------------ */
#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 qf;
#define Q_COS cosq
#define Q_SIN sinq
#define Q_PI M_PIq
#define Q_FLOOR floorq
#define Q_FABS fabsq
#else
#include <math.h>
typedef long double qf; /* IEEE binary128 on aarch64 Linux */
#define Q_COS cosl
#define Q_SIN sinl
#define Q_PI 3.141592653589793238462643383279502884L
#define Q_FLOOR floorl
#define Q_FABS fabsl
#endif

typedef struct { qf re, im; } qc;

static qc qc_mul(qc a, qc b) { qc r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re }; return r; }
static qc qc_add(qc a, qc b) { qc r = { a.re + b.re, a.im + b.im }; return r; }
static qc qc_sub(qc a, qc b) { qc r = { a.re - b.re, a.im - b.im }; return r; }

/* zeta^e for any integer e, e taken mod 2N: exp(i pi e / N) */
static qc zeta_pow(i64 e, uint32_t N)
{
    i64 m = e % (i64)(2 * N);
    if (m < 0) m += 2 * N;
    qf ang = Q_PI * (qf)m / (qf)N;
    qc r = { Q_COS(ang), Q_SIN(ang) };
    return r;
}

/* in-place N-point DFT: A_l = sum_k a_k exp(sign * 2 pi i l k / N), radix-2 */
static void qdft(qc* a, uint32_t N, int sign)
{
    for (uint32_t i = 1, j = 0; i < N; ++i) {
        uint32_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { qc t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (uint32_t len = 2; len <= N; len <<= 1) {
        for (uint32_t j = 0; j < len / 2; ++j) {
            /* exp(sign * 2 pi i j / len) = zeta^{sign * 2N j / len} */
            qc w = zeta_pow((i64)sign * (i64)(2 * N / len) * (i64)j, N);
            for (uint32_t i = 0; i < N; i += len) {
                qc u = a[i + j];
                qc v = qc_mul(a[i + j + len / 2], w);
                a[i + j] = qc_add(u, v);
                a[i + j + len / 2] = qc_sub(u, v);
            }
        }
    }
}

/* index l with 2l+1 = e (e odd, 0 < e < 2N) */
static uint32_t odd_index(u64 e) { return (uint32_t)((e - 1) / 2); }

/* round half away from zero of a binary128 value into int64.
 * Returns 0 on success, -1 if the value does not fit. */
static int q_round_i64(qf x, i64* out)
{
    qf a = Q_FLOOR(Q_FABS(x) + (qf)0.5);
    if (a >= (qf)9.2e18) return -1;
    i64 v = (i64)a;
    *out = (x < 0) ? -v : v;
    return 0;
}

/* z: N/2 real slot values (imaginary parts zero).  m: N integer coefficients.
 * Also writes the unrounded scaled values (as double, for the exemption rule)
 * into frac_out when it is not NULL: frac_out[k] = distance of scale*m_k to the
 * nearest .5 boundary, computed in binary128. */
int o_encode(const double* z, uint32_t N, double scale, i64* m, double* frac_out)
{
    qc* M = (qc*)calloc(N, sizeof(qc));
    u64 p = 1; /* 5^j mod 2N */
    for (uint32_t j = 0; j < N / 2; ++j) {
        qc v = { (qf)z[j], 0 };
        qc vc = { (qf)z[j], 0 };
        M[odd_index(p)] = v;
        M[odd_index(2 * N - p)] = vc; /* conjugate (imag part is zero) */
        p = (p * 5) % (2 * N);
    }
    /* b_k = sum_l M_l exp(-2 pi i l k / N); then m_k = zeta^{-k} b_k / N */
    qdft(M, N, -1);
    int rc = 0;
    for (uint32_t k = 0; k < N; ++k) {
        qc t = qc_mul(M[k], zeta_pow(-(i64)k, N));
        qf val = (qf)scale * t.re / (qf)N;
        if (frac_out) {
            qf f = val - Q_FLOOR(val);           /* in [0,1) */
            qf d = f - (qf)0.5;
            frac_out[k] = (double)Q_FABS(d);
        }
        if (q_round_i64(val, &m[k])) rc = -1;
    }
    free(M);
    return rc;
}

/* m: N integer coefficients -> z: N/2 slots (real and imaginary parts) */
void o_decode(const i64* m, uint32_t N, double scale, double* z_re, double* z_im)
{
    qc* a = (qc*)calloc(N, sizeof(qc));
    for (uint32_t k = 0; k < N; ++k) {
        qc mk = { (qf)m[k], 0 };
        a[k] = qc_mul(mk, zeta_pow((i64)k, N));
    }
    /* M_l = sum_k (m_k zeta^k) exp(+2 pi i l k / N) = m(zeta^{2l+1}) */
    qdft(a, N, +1);
    u64 p = 1;
    for (uint32_t j = 0; j < N / 2; ++j) {
        qc v = a[odd_index(p)];
        z_re[j] = (double)(v.re / (qf)scale);
        z_im[j] = (double)(v.im / (qf)scale);
        p = (p * 5) % (2 * N);
    }
    free(a);
}
