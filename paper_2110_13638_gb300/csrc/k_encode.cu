// k_encode.cu -- canonical-embedding encode (double-double) and decode (FP64).
#include "launch.cuh"

namespace fhe {

// ---------------------------------------------------------------- encode
// double-double helpers (explicit _rn intrinsics: never contracted)
struct ddv { double hi, lo; };
__device__ __forceinline__ ddv two_sum(double a, double b)
{
    double s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ddv fast_two_sum(double a, double b)
{
    double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
// double-double sum with one error-free transformation on the high parts
// (relative error ~2^-100 of the operands: the encoder needs ~2^-70)
__device__ __forceinline__ ddv dadd(ddv a, ddv b)
{
    ddv s = two_sum(a.hi, b.hi);
    s.lo = __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ddv dneg(ddv a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ddv dmul(ddv a, ddv b)
{
    double p = __dmul_rn(a.hi, b.hi);
    double e = __fma_rn(a.hi, b.hi, -p);
    e = __dadd_rn(e, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi)));
    return fast_two_sum(p, e);
}
struct cddv { ddv re, im; };
__device__ __forceinline__ cddv cadd(cddv a, cddv b) { return {dadd(a.re, b.re), dadd(a.im, b.im)}; }
__device__ __forceinline__ cddv csub(cddv a, cddv b) { return {dadd(a.re, dneg(b.re)), dadd(a.im, dneg(b.im))}; }
__device__ __forceinline__ cddv cmul(cddv a, cddv b)
{
    return {dadd(dmul(a.re, b.re), dneg(dmul(a.im, b.im))), dadd(dmul(a.re, b.im), dmul(a.im, b.re))};
}
__device__ __forceinline__ cddv ld4(const double4& v) { return {{v.x, v.y}, {v.z, v.w}}; }

// round half away from zero of a double-double to int64
__device__ __forceinline__ i64 dd_round(ddv v)
{
    bool neg = v.hi < 0.0 || (v.hi == 0.0 && v.lo < 0.0);
    if (neg) v = dneg(v);
    double f = floor(v.hi);
    double frac = __dadd_rn(__dsub_rn(v.hi, f), v.lo);
    double add = floor(__dadd_rn(frac, 0.5));
    i64 r = (i64)f + (i64)add;
    return neg ? -r : r;
}

// One block per (ct, half h): the N/2-point inverse DFT of the slots (placed
// at l(j) = (5^j mod 2N - 1)/4) is split by its first decimation-in-frequency
// stage; half h runs the N/4-point DFT of its half in shared memory.
// Output: m_k = round(scale * Re c_k), m_{k+N/2} = round(scale * Im c_k),
// c_k = (2/N) zeta^{-k} X_k.
__global__ void __launch_bounds__(512) k_encode_kernel(const double* __restrict__ slots, const uint32_t* __restrict__ slot_of,
                                                        const double4* __restrict__ tw, const double4* __restrict__ twist,
                                                        double scale_over_M, int N, i64* __restrict__ m)
{
    extern __shared__ double4 A[];       // N/4 complex dd values
    const int M = N / 2, H = M / 2;
    const int ct = blockIdx.x >> 1, h = blockIdx.x & 1;
    const double* z = slots + (size_t)ct * M;
    for (int l = threadIdx.x; l < H; l += blockDim.x) {
        const double x0 = z[slot_of[l]], x1 = z[slot_of[l + H]];
        cddv v;
        if (h == 0) {
            v.re = two_sum(x0, x1);
            v.im = {0.0, 0.0};
        } else {
            ddv d = two_sum(x0, -x1);
            const cddv w = ld4(tw[l]);                 // W^l, W = e^{-2 pi i / M}
            v.re = dmul(d, w.re);
            v.im = dmul(d, w.im);
        }
        A[l] = make_double4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
    }
    __syncthreads();
    // H-point DIF, twiddle for offset o at half-size hs: W^{o * M / (2 hs)}
    for (int hs = H / 2; hs >= 1; hs >>= 1) {
        for (int b = threadIdx.x; b < H / 2; b += blockDim.x) {
            const int blk = b / hs, o = b % hs;
            const int i0 = blk * 2 * hs + o, i1 = i0 + hs;
            const cddv x = ld4(A[i0]), y = ld4(A[i1]);
            const cddv s = cadd(x, y);
            const cddv d = cmul(csub(x, y), ld4(tw[o * (M / (2 * hs))]));
            A[i0] = make_double4(s.re.hi, s.re.lo, s.im.hi, s.im.lo);
            A[i1] = make_double4(d.re.hi, d.re.lo, d.im.hi, d.im.lo);
        }
        __syncthreads();
    }
    int lg = 0;
    while ((1 << lg) < H) ++lg;
    for (int p = threadIdx.x; p < H; p += blockDim.x) {
        const int kp = (int)(__brev((unsigned)p) >> (32 - lg));
        const int k = 2 * kp + h;                       // frequency index in [0, M)
        const cddv X = ld4(A[p]);
        cddv c = cmul(X, ld4(twist[k]));
        const ddv s = {scale_over_M, 0.0};
        m[(size_t)ct * N + k] = dd_round(dmul(c.re, s));
        m[(size_t)ct * N + k + M] = dd_round(dmul(c.im, s));
    }
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
    const size_t smem = (size_t)(N / 4) * sizeof(double4);
    static size_t configured = 0;
    if (configured < smem) {
        cudaFuncSetAttribute(k_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    int thr = N / 8;
    thr = thr < 32 ? 32 : (thr > 512 ? 512 : thr);
    {
    LaunchScope ls(c, "encode_fft", st);
    k_encode_kernel<<<2 * n_ct, thr, smem, st>>>(slots, c->d_slot_of, c->d_enc_tw, c->d_enc_twist,
                                                 scale / (double)(N / 2), N, m);
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
// z_j = Re Z_{l(j)} / scale, Z = DFT_{N/2}(c_k zeta^k) with e^{+2 pi i / M},
// c_k = m_k + i m_{k+N/2}; FP64, one block per ciphertext.
__global__ void __launch_bounds__(512) k_decode_kernel(const i64* __restrict__ m, const uint32_t* __restrict__ slot_of,
                                                        const double4* __restrict__ tw, const double4* __restrict__ twist,
                                                        double inv_scale, int N, double* __restrict__ slots)
{
    extern __shared__ double2 B[];       // N/2 complex doubles
    const int M = N / 2;
    const int ct = blockIdx.x;
    const i64* mc = m + (size_t)ct * N;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const double a = (double)mc[k], b = (double)mc[k + M];
        const double4 t = twist[k];                     // zeta^{-k}: use its conjugate
        const double wr = t.x, wi = -t.z;
        B[k] = make_double2(a * wr - b * wi, a * wi + b * wr);
    }
    __syncthreads();
    for (int hs = M / 2; hs >= 1; hs >>= 1) {
        for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
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
    while ((1 << lg) < M) ++lg;
    for (int l = threadIdx.x; l < M; l += blockDim.x) {
        const int p = (int)(__brev((unsigned)l) >> (32 - lg));
        slots[(size_t)ct * M + slot_of[l]] = B[p].x * inv_scale;
    }
}

void k_decode(const fhe_ctx* c, const i64* m, uint32_t n_ct, double scale, double* slots, cudaStream_t st)
{
    if (n_ct == 0) return;
    const int N = (int)c->N;
    const size_t smem = (size_t)(N / 2) * sizeof(double2);
    static size_t configured = 0;
    if (configured < smem) {
        cudaFuncSetAttribute(k_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = smem;
    }
    int thr = N / 4;
    thr = thr < 32 ? 32 : (thr > 512 ? 512 : thr);
    LaunchScope ls(c, "decode_fft", st);
    k_decode_kernel<<<n_ct, thr, smem, st>>>(m, c->d_slot_of, c->d_enc_tw, c->d_enc_twist, 1.0 / scale, N, slots);
}


}  // namespace fhe
