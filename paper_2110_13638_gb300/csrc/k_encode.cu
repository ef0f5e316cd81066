// k_encode.cu -- canonical-embedding encode (128-bit fixed point) and decode (FP64).
#include "launch.cuh"

namespace fhe {

// ---------------------------------------------------------------- encode
// The encoder's inverse DFT runs in 128-bit fixed point on the integer pipes:
// a value is a two's-complement integer X with value X / 2^64 (63 integer
// bits, 64 fractional bits); a root of unity is a sign-magnitude integer with
// 126 fractional bits.  Inputs (slot * scale / M, formed as an exact product
// of two doubles) enter exactly to 2^-64, each product drops less than
// 6 2^-64, so the rounded coefficients carry an absolute error below 2^-40,
// far inside the 1e-6 band around .5 where encodings may differ.
// Range: |slot| * scale must stay below 2^61 (intermediate sums stay below
// 2^62); larger inputs cannot be encoded against a 60-bit first prime anyway.
struct fx { u64 lo, hi; };

__device__ __forceinline__ fx fx_add(fx a, fx b)
{
    fx r;
    asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;" : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
    return r;
}
__device__ __forceinline__ fx fx_sub(fx a, fx b)
{
    fx r;
    asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;" : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
    return r;
}
__device__ __forceinline__ fx fx_neg(fx a) { return fx_sub({0ull, 0ull}, a); }
__device__ __forceinline__ fx fx_cneg(fx a, bool neg) { return neg ? fx_neg(a) : a; }
__device__ __forceinline__ bool fx_isneg(fx a) { return (i64)a.hi < 0; }

// exact double -> fixed point (bits below 2^-64 truncated toward zero)
__device__ __forceinline__ fx fx_from_double(double d)
{
    const u64 b = (u64)__double_as_longlong(d);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return {0ull, 0ull};                    // zero or below 2^-1022
    const u64 m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = ex - 1011;                             // |d| 2^64 = m 2^sh
    fx r;
    if (sh >= 64) r = {0ull, m << (sh - 64)};
    else if (sh > 0) r = {m << sh, m >> (64 - sh)};
    else if (sh > -64) r = {m >> (-sh), 0ull};
    else r = {0ull, 0ull};
    return fx_cneg(r, (b >> 63) != 0);
}

// x * y as fixed point, x * y = p + e exactly (two-product)
__device__ __forceinline__ fx fx_product(double x, double y)
{
    const double p = __dmul_rn(x, y);
    const double e = __fma_rn(x, y, -p);
    return fx_add(fx_from_double(p), fx_from_double(e));
}

// (|a| |w|) / 2^126 for magnitudes a < 2^126 (value scale 2^64) and w <= 2^127
// (scale 2^126); the a_lo w_lo partial product (below 4 units) is dropped
__device__ __forceinline__ fx umul_q126(u64 alo, u64 ahi, u64 wlo, u64 whi)
{
    const u64 lo1 = ahi * whi, hi1 = __umul64hi(ahi, whi);
    const u64 t2l = ahi * wlo, t2h = __umul64hi(ahi, wlo);
    const u64 t3l = alo * whi, t3h = __umul64hi(alo, whi);
    u64 ml, mh, mc;
    asm("add.cc.u64 %0, %3, %5;\n\taddc.cc.u64 %1, %4, %6;\n\taddc.u64 %2, %7, %7;"
        : "=l"(ml), "=l"(mh), "=l"(mc)
        : "l"(t2l), "l"(t2h), "l"(t3l), "l"(t3h), "l"(0ull));
    const fx top = {lo1 << 2, (hi1 << 2) | (lo1 >> 62)};
    const fx mid = {(mh << 2) | (ml >> 62), (mc << 2) | (mh >> 62)};
    return fx_add(top, mid);
}

struct cfx { fx re, im; };
__device__ __forceinline__ cfx cfx_add(cfx a, cfx b) { return {fx_add(a.re, b.re), fx_add(a.im, b.im)}; }
__device__ __forceinline__ cfx cfx_sub(cfx a, cfx b) { return {fx_sub(a.re, b.re), fx_sub(a.im, b.im)}; }

// a * w for a root w = (re, im) in sign-magnitude Q126 form
__device__ __forceinline__ cfx cfx_mul_root(cfx a, ulonglong2 wr, ulonglong2 wi)
{
    const bool sar = fx_isneg(a.re), sai = fx_isneg(a.im);
    const fx ar = fx_cneg(a.re, sar), ai = fx_cneg(a.im, sai);
    const bool sbr = (wr.y >> 63) != 0, sbi = (wi.y >> 63) != 0;
    const u64 brh = wr.y & ~(1ull << 63), bih = wi.y & ~(1ull << 63);
    const fx p1 = umul_q126(ar.lo, ar.hi, wr.x, brh);     // re re
    const fx p2 = umul_q126(ai.lo, ai.hi, wi.x, bih);     // im im
    const fx p3 = umul_q126(ar.lo, ar.hi, wi.x, bih);     // re im
    const fx p4 = umul_q126(ai.lo, ai.hi, wr.x, brh);     // im re
    return {fx_add(fx_cneg(p1, sar != sbr), fx_cneg(p2, sai == sbi)),
            fx_add(fx_cneg(p3, sar != sbi), fx_cneg(p4, sai != sbr))};
}

// a (real) * w
__device__ __forceinline__ cfx fx_mul_root(fx a, ulonglong2 wr, ulonglong2 wi)
{
    const bool sa = fx_isneg(a);
    const fx aa = fx_cneg(a, sa);
    const fx pr = umul_q126(aa.lo, aa.hi, wr.x, wr.y & ~(1ull << 63));
    const fx pi = umul_q126(aa.lo, aa.hi, wi.x, wi.y & ~(1ull << 63));
    return {fx_cneg(pr, sa != ((wr.y >> 63) != 0)), fx_cneg(pi, sa != ((wi.y >> 63) != 0))};
}

// round half away from zero
__device__ __forceinline__ i64 fx_round(fx v)
{
    const bool neg = fx_isneg(v);
    const fx a = fx_cneg(v, neg);
    const i64 r = (i64)(a.hi + (a.lo >> 63));
    return neg ? -r : r;
}

// A ciphertext's N/2-point inverse DFT (slots placed at l(j) = (5^j mod 2N -
// 1)/4, pre-multiplied by scale / M) is split by its first a decimation-in-
// frequency levels into A = 2^a blocks of H = M / A <= 4096 points: block r
// forms y_r[n] = sum_s x[n + s H] W^((n + s H) r) (W = e^{-2 pi i / M}) and runs
// the H-point DIF of y_r in shared memory (real and imaginary parts in
// separate arrays); its outputs are the frequencies k = A p' + r.
// Output: m_k = round(Re c_k), m_{k+N/2} = round(Im c_k), c_k = zeta^{-k} X_k.
__global__ void __launch_bounds__(512) k_encode_kernel(const double* __restrict__ slots, const uint32_t* __restrict__ slot_of,
                                                        const ulonglong2* __restrict__ tw, const ulonglong2* __restrict__ twist,
                                                        double scale_over_M, int N, int logA, i64* __restrict__ m)
{
    extern __shared__ ulonglong2 S[];    // [H] real parts, then [H] imaginary parts
    const int M = N / 2, A = 1 << logA, H = M >> logA;
    ulonglong2* Sr = S;
    ulonglong2* Si = S + H;
    const int ct = blockIdx.x >> logA, r = blockIdx.x & (A - 1);
    const double* z = slots + (size_t)ct * M;
    auto put = [&](int i, const cfx& v) {
        Sr[i] = make_ulonglong2(v.re.lo, v.re.hi);
        Si[i] = make_ulonglong2(v.im.lo, v.im.hi);
    };
    auto get = [&](int i) {
        const ulonglong2 a = Sr[i], b = Si[i];
        return cfx{{a.x, a.y}, {b.x, b.y}};
    };
    for (int n = threadIdx.x; n < H; n += blockDim.x) {
        cfx y = {{0ull, 0ull}, {0ull, 0ull}};
        for (int s = 0; s < A; ++s) {
            const int i = n + s * H;
            const fx x = fx_product(z[slot_of[i]], scale_over_M);
            if (r == 0) {
                y.re = fx_add(y.re, x);
            } else {
                int e = (int)(((unsigned)i * (unsigned)r) & (unsigned)(M - 1));
                const bool neg = e >= M / 2;               // W^(M/2) = -1
                if (neg) e -= M / 2;
                const cfx t = fx_mul_root(x, __ldg(&tw[2 * e]), __ldg(&tw[2 * e + 1]));
                y = neg ? cfx_sub(y, t) : cfx_add(y, t);
            }
        }
        put(n, y);
    }
    __syncthreads();
    // H-point DIF, twiddle for offset o at half-size hs: W^{o * M / (2 hs)}
    for (int hs = H / 2; hs >= 1; hs >>= 1) {
        for (int b = threadIdx.x; b < H / 2; b += blockDim.x) {
            const int blk = b / hs, o = b % hs;
            const int i0 = blk * 2 * hs + o, i1 = i0 + hs;
            const cfx x = get(i0), y = get(i1);
            const int e = o * (M / (2 * hs));
            put(i0, cfx_add(x, y));
            put(i1, cfx_mul_root(cfx_sub(x, y), __ldg(&tw[2 * e]), __ldg(&tw[2 * e + 1])));
        }
        __syncthreads();
    }
    int lg = 0;
    while ((1 << lg) < H) ++lg;
    for (int p = threadIdx.x; p < H; p += blockDim.x) {
        const int kp = lg ? (int)(__brev((unsigned)p) >> (32 - lg)) : 0;
        const int k = (kp << logA) + r;                 // frequency index in [0, M)
        const cfx c = cfx_mul_root(get(p), __ldg(&twist[2 * k]), __ldg(&twist[2 * k + 1]));
        m[(size_t)ct * N + k] = fx_round(c.re);
        m[(size_t)ct * N + k + M] = fx_round(c.im);
    }
}

// blocks per ciphertext (log2) so that one block holds at most hmax points
static int split_log(int M, int hmax)
{
    int a = 1;
    while ((M >> a) > hmax) ++a;
    return a;
}

struct OpSignedRows {
    static const char* family() { return "encode_ntt"; }
    const i64* m;       // [n][N]
    u64* out;           // [n][L][N]
    int n, L, N;
    __host__ __device__ int count() const { return n * L; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& P) const { return from_signed(m[(size_t)(p / L) * N + j], P); }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { out[(size_t)p * N + j] = v; }
};

size_t encode_scratch_bytes(const fhe_ctx* c, uint32_t n_ct) { return (size_t)n_ct * c->N * sizeof(i64); }

void encode_coefficients(const fhe_ctx* c, const double* slots, uint32_t n_ct, double scale, i64* m, cudaStream_t st)
{
    const int N = (int)c->N;
    const int logA = split_log(N / 2, 4096);
    const int H = (N / 2) >> logA;
    const size_t smem = (size_t)H * 2 * sizeof(ulonglong2);
    ensure_smem((const void*)k_encode_kernel, smem);
    int thr = H / 2;
    thr = thr < 32 ? 32 : (thr > 512 ? 512 : thr);
    {
    LaunchScope ls(c, "encode_fft", st);
    k_encode_kernel<<<n_ct << logA, thr, smem, st>>>(slots, c->d_slot_of, c->d_enc_tw_q, c->d_enc_twist_q,
                                                      scale / (double)(N / 2), N, logA, m);
    }
}

void k_encode(const fhe_ctx* c, const double* slots, uint32_t n_ct, uint32_t L, double scale, u64* pt, void* scratch,
              cudaStream_t st)
{
    if (n_ct == 0) return;
    i64* m = (i64*)scratch;
    encode_coefficients(c, slots, n_ct, scale, m, st);
    OpSignedRows op{m, pt, (int)n_ct, (int)L, (int)c->N};
    launch_ntt<false>(c, op, st);
}

// ---------------------------------------------------------------- decode
// z_j = Re Z_{l(j)} / scale, Z = DFT_{N/2}(v), v_k = c_k zeta^k with
// conj(W) = e^{+2 pi i / M}, c_k = m_k + i m_{k+N/2}; FP64.  Split like the
// encoder: block r of A = 2^a forms y_r[n] = sum_s v[n + s H] conj(W)^((n + s H) r)
// and runs the H-point DIF (H <= 8192); its outputs are Z_{A p' + r}.
__global__ void __launch_bounds__(512) k_decode_kernel(const i64* __restrict__ m, const uint32_t* __restrict__ slot_of,
                                                        const double4* __restrict__ tw, const double4* __restrict__ twist,
                                                        double inv_scale, int N, int logA, double* __restrict__ slots)
{
    extern __shared__ double2 B[];       // H complex doubles
    const int M = N / 2, A = 1 << logA, H = M >> logA;
    const int ct = blockIdx.x >> logA, r = blockIdx.x & (A - 1);
    const i64* mc = m + (size_t)ct * N;
    for (int n = threadIdx.x; n < H; n += blockDim.x) {
        double yr = 0.0, yi = 0.0;
        for (int s = 0; s < A; ++s) {
            const int k = n + s * H;
            const double a = (double)mc[k], b = (double)mc[k + M];
            const double4 t = twist[k];                 // zeta^{-k}: use its conjugate
            double vr = a * t.x + b * t.z, vi = -a * t.z + b * t.x;
            if (r != 0) {
                int e = (int)(((unsigned)k * (unsigned)r) & (unsigned)(M - 1));
                const bool neg = e >= M / 2;
                if (neg) e -= M / 2;
                const double4 w4 = tw[e];
                const double wr = neg ? -w4.x : w4.x, wi = neg ? w4.z : -w4.z;   // conj(W^e)
                const double ur = vr * wr - vi * wi, ui = vr * wi + vi * wr;
                vr = ur;
                vi = ui;
            }
            yr += vr;
            yi += vi;
        }
        B[n] = make_double2(yr, yi);
    }
    __syncthreads();
    for (int hs = H / 2; hs >= 1; hs >>= 1) {
        for (int b = threadIdx.x; b < H / 2; b += blockDim.x) {
            const int blk = b / hs, o = b % hs;
            const int i0 = blk * 2 * hs + o, i1 = i0 + hs;
            const double2 x = B[i0], y = B[i1];
            const double4 w4 = tw[o * (M / (2 * hs))];  // W^e, W = e^{-2 pi i / M}: conjugate
            const double wr = w4.x, wi = -w4.z;
            const double dr = x.x - y.x, di = x.y - y.y;
            B[i0] = make_double2(x.x + y.x, x.y + y.y);
            B[i1] = make_double2(dr * wr - di * wi, dr * wi + di * wr);
        }
        __syncthreads();
    }
    int lg = 0;
    while ((1 << lg) < H) ++lg;
    for (int p = threadIdx.x; p < H; p += blockDim.x) {
        const int tp = lg ? (int)(__brev((unsigned)p) >> (32 - lg)) : 0;
        const int t = (tp << logA) + r;                 // DFT index in [0, M)
        slots[(size_t)ct * M + slot_of[t]] = B[p].x * inv_scale;
    }
}

void k_decode(const fhe_ctx* c, const i64* m, uint32_t n_ct, double scale, double* slots, cudaStream_t st)
{
    if (n_ct == 0) return;
    const int N = (int)c->N;
    int logA = 0;
    while (((N / 2) >> logA) > 8192) ++logA;
    const int H = (N / 2) >> logA;
    const size_t smem = (size_t)H * sizeof(double2);
    ensure_smem((const void*)k_decode_kernel, smem);
    int thr = H / 2;
    thr = thr < 32 ? 32 : (thr > 512 ? 512 : thr);
    LaunchScope ls(c, "decode_fft", st);
    k_decode_kernel<<<n_ct << logA, thr, smem, st>>>(m, c->d_slot_of, c->d_enc_tw, c->d_enc_twist, 1.0 / scale, N,
                                                      logA, slots);
}


}  // namespace fhe
