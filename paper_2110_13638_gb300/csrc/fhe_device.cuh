// fhe_device.cuh -- device-side modular arithmetic and the shared-memory
// negacyclic NTT used by every kernel of the RNS-CKKS path.
//
// Arithmetic: residues are u64 below primes q < 2^62.  Products by a constant
// use Shoup's precomputed quotient (w' = floor(w 2^64 / q)); general products
// use the 128-bit product reduced through 2^64 mod q; Barrett reduction of a
// 64-bit word uses mu = floor(2^64 / q).
//
// NTT: forward = Cooley-Tukey with psi powers in bit-reversed order (natural
// input, bit-reversed output); inverse = Gentleman-Sande (bit-reversed input,
// natural output) followed by N^{-1}.  Butterflies are Harvey's lazy forms
// (values in [0, 4q) forward, [0, 2q) inverse), which needs q < 2^62.
// One thread block transforms one residue polynomial held in shared memory;
// stages are grouped into passes of up to 2^LOGR-point sub-transforms kept in
// registers, so shared memory is touched once per pass instead of once per
// stage.  Shared-memory index j is padded to j + j/16 (conflict-free 64-bit
// accesses for every pass stride).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned long long u64;
typedef long long i64;

struct PrimeC {
    u64 q;       // the prime
    u64 q2;      // 2q
    u64 mu;      // floor(2^64 / q)
    u64 r64;     // 2^64 mod q
    u64 r64s;    // Shoup quotient of r64
    u64 ninv;    // N^{-1} mod q
    u64 ninvs;   // Shoup quotient of ninv
    u64 half;    // (q - 1) / 2
    u64 ub;      // floor(2^64 / q) * q (rejection bound of the uniform sampler)
};

// ---------------------------------------------------------------- scalar ops
__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 ws, u64 q)
{
    u64 t = __umul64hi(a, ws);
    return a * w - t * q;              // in [0, 2q) for any a < 2^64
}

__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 ws, u64 q)
{
    u64 r = mul_shoup_lazy(a, w, ws, q);
    return r >= q ? r - q : r;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q)
{
    u64 r = a + b;
    return r >= q ? r - q : r;
}

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q)
{
    return a >= b ? a - b : a + q - b;
}

// x mod q for any 64-bit x
__device__ __forceinline__ u64 reduce64(u64 x, const PrimeC& P)
{
    u64 t = __umul64hi(x, P.mu);
    u64 r = x - t * P.q;               // in [0, 2q)
    return r >= P.q ? r - P.q : r;
}

// (hi 2^64 + lo) mod q
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const PrimeC& P)
{
    u64 h = reduce64(hi, P);
    u64 t = mul_shoup(h, P.r64, P.r64s, P.q);
    return add_mod(t, reduce64(lo, P), P.q);
}

// a * b mod q for a, b < 2^64 (b need not be a precomputed constant)
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeC& P)
{
    return reduce128(__umul64hi(a, b), a * b, P);
}

// signed 64-bit integer -> residue mod q
__device__ __forceinline__ u64 from_signed(i64 v, const PrimeC& P)
{
    if (v >= 0) return reduce64((u64)v, P);
    u64 r = reduce64((u64)(-(v + 1)) + 1ull, P);   // |v| mod q, no overflow at INT64_MIN
    return r == 0 ? 0 : P.q - r;
}

// residue v mod p (p odd, centred in (-p/2, p/2)) -> residue mod q
__device__ __forceinline__ u64 centred_to(u64 v, u64 p, u64 p_half, u64 p_mod_q, const PrimeC& Q)
{
    u64 r = reduce64(v, Q);
    if (v > p_half) r = sub_mod(r, p_mod_q, Q.q);
    return r;
}

// ---------------------------------------------------------------- NTT core
__device__ __forceinline__ int spad(int j) { return j + (j >> 4); }

__host__ __device__ constexpr int ntt_smem_words(int N) { return N + (N >> 4); }

// forward Cooley-Tukey pass over stages s0 .. s0+K-1 (distances N>>(s+1)).
// A group is the 2^K elements j0 + i 2^ltb; at stage l its pairs (i, i+h),
// h = 2^(K-1-l), with i = m 2h + t share the twiddle psi_rev[2^st + g 2^l + m],
// so each group loads 2^K - 1 twiddles per pass.
template <int K>
__device__ __forceinline__ void ntt_fwd_pass(u64* sm, int logN, int s0, const ulonglong2* __restrict__ tw,
                                             u64 q, u64 q2, int tid, int nthr)
{
    constexpr int R = 1 << K;
    const int N = 1 << logN;
    const int ltb = logN - s0 - K;               // log2 of the smallest distance
    const int ngroups = N >> K;
    for (int gi = tid; gi < ngroups; gi += nthr) {
        const int g = gi >> ltb;
        const int r = gi & ((1 << ltb) - 1);
        const int j0 = (g << (ltb + K)) + r;
        u64 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = sm[spad(j0 + (i << ltb))];
#pragma unroll
        for (int l = 0; l < K; ++l) {
            const int h = R >> (l + 1);
            const ulonglong2* twl = tw + (1 << (s0 + l)) + (g << l);
#pragma unroll
            for (int m = 0; m < (1 << l); ++m) {
                const ulonglong2 w = __ldg(&twl[m]);
#pragma unroll
                for (int t = 0; t < h; ++t) {
                    const int i = m * 2 * h + t;
                    u64 X = x[i];
                    X = X >= q2 ? X - q2 : X;
                    const u64 T = mul_shoup_lazy(x[i + h], w.x, w.y, q);
                    x[i] = X + T;
                    x[i + h] = X + q2 - T;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) sm[spad(j0 + (i << ltb))] = x[i];
    }
}

// inverse Gentleman-Sande pass over distances 2^lt0 .. 2^(lt0+K-1); at stage l
// (distance 2^(lt0+l), h = 2^l) the pairs i = m 2h + t share the twiddle
// psi_inv_rev[N / 2^(lt0+l+1) + g 2^(K-l-1) + m].
template <int K>
__device__ __forceinline__ void ntt_inv_pass(u64* sm, int logN, int lt0, const ulonglong2* __restrict__ tw,
                                             u64 q, u64 q2, int tid, int nthr)
{
    constexpr int R = 1 << K;
    const int N = 1 << logN;
    const int ngroups = N >> K;
    for (int gi = tid; gi < ngroups; gi += nthr) {
        const int g = gi >> lt0;
        const int r = gi & ((1 << lt0) - 1);
        const int j0 = (g << (lt0 + K)) + r;
        u64 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = sm[spad(j0 + (i << lt0))];
#pragma unroll
        for (int l = 0; l < K; ++l) {
            const int h = 1 << l;
            const ulonglong2* twl = tw + (N >> (lt0 + l + 1)) + (g << (K - l - 1));
#pragma unroll
            for (int m = 0; m < (R >> (l + 1)); ++m) {
                const ulonglong2 w = __ldg(&twl[m]);
#pragma unroll
                for (int t = 0; t < h; ++t) {
                    const int i = m * 2 * h + t;
                    const u64 X = x[i], Y = x[i + h];
                    u64 S = X + Y;
                    S = S >= q2 ? S - q2 : S;
                    x[i] = S;
                    x[i + h] = mul_shoup_lazy(X + q2 - Y, w.x, w.y, q);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) sm[spad(j0 + (i << lt0))] = x[i];
    }
}

template <int LOGR>
__device__ __forceinline__ void ntt_fwd_smem(u64* sm, int logN, const ulonglong2* __restrict__ tw, u64 q, int tid, int nthr)
{
    const u64 q2 = 2 * q;
    int s = 0;
    while (s < logN) {
        const int k = (logN - s) < LOGR ? (logN - s) : LOGR;
        switch (k) {
        case 4: ntt_fwd_pass<4>(sm, logN, s, tw, q, q2, tid, nthr); break;
        case 3: ntt_fwd_pass<3>(sm, logN, s, tw, q, q2, tid, nthr); break;
        case 2: ntt_fwd_pass<2>(sm, logN, s, tw, q, q2, tid, nthr); break;
        default: ntt_fwd_pass<1>(sm, logN, s, tw, q, q2, tid, nthr); break;
        }
        __syncthreads();
        s += k;
    }
}

template <int LOGR>
__device__ __forceinline__ void ntt_inv_smem(u64* sm, int logN, const ulonglong2* __restrict__ tw, u64 q, int tid, int nthr)
{
    const u64 q2 = 2 * q;
    int lt = 0;
    while (lt < logN) {
        const int k = (logN - lt) < LOGR ? (logN - lt) : LOGR;
        switch (k) {
        case 4: ntt_inv_pass<4>(sm, logN, lt, tw, q, q2, tid, nthr); break;
        case 3: ntt_inv_pass<3>(sm, logN, lt, tw, q, q2, tid, nthr); break;
        case 2: ntt_inv_pass<2>(sm, logN, lt, tw, q, q2, tid, nthr); break;
        default: ntt_inv_pass<1>(sm, logN, lt, tw, q, q2, tid, nthr); break;
        }
        __syncthreads();
        lt += k;
    }
}

// final reductions of the lazy ranges
__device__ __forceinline__ u64 fwd_final(u64 x, u64 q)
{
    const u64 q2 = 2 * q;
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

__device__ __forceinline__ u64 inv_final(u64 x, const PrimeC& P)
{
    return mul_shoup(x, P.ninv, P.ninvs, P.q);       // x in [0, 2q) times N^{-1}
}

// ---------------------------------------------------------------- tables
struct NttTables {
    const ulonglong2* tw_fwd;   // [nprimes][N] (w, w') psi^{bitrev(i)}
    const ulonglong2* tw_inv;   // [nprimes][N] (w, w') psi^{-bitrev(i)}
    const PrimeC* pc;           // [nprimes]
    int logN;
};

// ---------------------------------------------------------------- kernel
// Generic batched transform with a fused prologue and epilogue.  Op supplies
//   static const char* family()             -- name for the measurement hook
//   int  count() const                      -- number of transform units
//   int  nsub(int p) const                  -- transforms in unit p (run in order)
//   int  prime(int p, int u) const          -- key-prime index of transform u
//   bool direct(int p, int u) const         -- skip the transform (store reads input itself)
//   u64  load(int p, int u, int j, const PrimeC&) const   -- input value in [0, q)
//   Pre  pre(int p, int u, int j) const     -- global words the epilogue needs (issued
//                                              for several j before any store)
//   void store(int p, int u, int j, u64 v, const Pre&, const PrimeC&) const -- v in [0, q)
// Grid-stride over units so one launch may cover any batch.  Prologue loads
// and epilogue pre-loads are issued kUnroll at a time per thread.
constexpr int kUnroll = 4;

template <bool INV, int LOGR, int MAXT, class Op>
__global__ void __launch_bounds__(MAXT, 1) k_ntt_op(Op op, NttTables T)
{
    extern __shared__ u64 sm[];
    const int logN = T.logN;
    const int N = 1 << logN;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int p = blockIdx.x; p < op.count(); p += gridDim.x) {
        const int ns = op.nsub(p);
        for (int u = 0; u < ns; ++u) {
            const int pi = op.prime(p, u);
            const PrimeC P = T.pc[pi];
            const bool dir = op.direct(p, u);
            if (!dir) {
                for (int j0 = tid; j0 < N; j0 += nthr * kUnroll) {
                    u64 v[kUnroll];
#pragma unroll
                    for (int k = 0; k < kUnroll; ++k) {
                        const int j = j0 + k * nthr;
                        v[k] = j < N ? op.load(p, u, j, P) : 0;
                    }
#pragma unroll
                    for (int k = 0; k < kUnroll; ++k) {
                        const int j = j0 + k * nthr;
                        if (j < N) sm[spad(j)] = v[k];
                    }
                }
                __syncthreads();
                if (INV) ntt_inv_smem<LOGR>(sm, logN, T.tw_inv + (size_t)pi * N, P.q, tid, nthr);
                else ntt_fwd_smem<LOGR>(sm, logN, T.tw_fwd + (size_t)pi * N, P.q, tid, nthr);
            }
            for (int j0 = tid; j0 < N; j0 += nthr * kUnroll) {
                typename Op::Pre pr[kUnroll];
                u64 v[kUnroll];
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    const int j = j0 + k * nthr;
                    if (j < N) {
                        pr[k] = op.pre(p, u, j);
                        const u64 x = dir ? 0 : sm[spad(j)];
                        v[k] = dir ? 0 : (INV ? inv_final(x, P) : fwd_final(x, P.q));
                    }
                }
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    const int j = j0 + k * nthr;
                    if (j < N) op.store(p, u, j, v[k], pr[k], P);
                }
            }
            __syncthreads();
        }
    }
}
