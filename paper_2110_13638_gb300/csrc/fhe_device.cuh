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
#include <type_traits>
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
    u64 p21[4];  // 2^21, 2^42, 2^63, 2^84 mod q (limb positions of the MAC)
    u64 p21s[4]; // their Shoup quotients
    u64 bmu;     // Barrett constant floor(2^(2b) / q) << (63 - b), b = bit length of q
    u64 bsh;     // b - 1
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

// a * b mod q for REDUCED a, b < q < 2^62 (Barrett): with x = a b < 2^(2b),
// t = floor(floor(x / 2^(b-1)) floor(2^(2b) / q) / 2^(b+1)) lies within 2 of
// floor(x / q), so x - t q is in [0, 3q) and two conditional subtractions
// finish it; two 64-bit products and two high products instead of mul_mod's
// four high products
__device__ __forceinline__ u64 mul_mod_r(u64 a, u64 b, const PrimeC& P)
{
    const u64 lo = a * b, hi = __umul64hi(a, b);
    const u64 xh = (hi << (64 - P.bsh)) | (lo >> P.bsh);
    const u64 t = __umul64hi(xh, P.bmu);
    u64 r = lo - t * P.q;
    r = r >= P.q ? r - P.q : r;
    return r >= P.q ? r - P.q : r;
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

// An Op whose store accepts forward-transform outputs in the lazy range
// [0, 4q) declares  static constexpr bool kLazyStore = true;
template <class Op, class = void>
struct lazy_store : std::false_type {};
template <class Op>
struct lazy_store<Op, std::void_t<decltype(Op::kLazyStore)>> : std::integral_constant<bool, Op::kLazyStore> {};

// An Op that runs once per context (key generation) declares
//   static constexpr bool kColdPath = true;
// and gets only the reduced butterflies of the fused-I/O kernel (half the code).
template <class Op, class = void>
struct cold_path : std::false_type {};
template <class Op>
struct cold_path<Op, std::void_t<decltype(Op::kColdPath)>> : std::integral_constant<bool, Op::kColdPath> {};

template <class Op>
__device__ __forceinline__ u64 fwd_out(u64 x, u64 q)
{
    if constexpr (lazy_store<Op>::value) return x;
    else return fwd_final(x, q);
}

// ---------------------------------------------------------------- tables
struct NttTables {
    const ulonglong2* tw_fwd;   // [nprimes][N] (w, w') psi^{bitrev(i)}
    const ulonglong2* tw_inv;   // [nprimes][N] (w, w') psi^{-bitrev(i)}
    // the same tables with the five stages whose twiddles vary per lane in
    // the warp-local transform (forward: the last five, inverse: the first
    // five) transposed so that the 32 lanes of a warp read 32 consecutive
    // entries (wl_perm); the other stages as in tw_fwd / tw_inv.  Null when
    // the ring is outside the warp-local schedule's range
    const ulonglong2* tw_fwd_wl;
    const ulonglong2* tw_inv_wl;
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
//                                              (forward transforms accept [0, 4q))
//   Pre  pre(int p, int u, int j) const     -- global words the epilogue needs (issued
//                                              for several j before any store)
//   void store(int p, int u, int j, u64 v, const Pre&, const PrimeC&) const -- v in [0, q)
//                                              ([0, 4q) after a forward transform if
//                                              the Op declares kLazyStore; below 36 q
//                                              in the fused-I/O kernel's unreduced form)
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
                        v[k] = dir ? 0 : (INV ? inv_final(x, P) : fwd_out<Op>(x, P.q));
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

// ---------------------------------------------------------------- two-pass NTT
// The ring degree N = N1 N2 (N1 = 2^k1 rows, N2 = 2^k2 columns, element
// j = N2 i + c).  Forward: the first k1 stages (distances N/2 .. N2) act on
// each column as an N1-point transform whose twiddles are the first N1 entries
// of the psi table; the last k2 stages act on each row with the row's own
// twiddles.  Inverse: rows first (distances 1 .. N2/2), then columns
// (N1-point transforms on the prefix of the inverse table).  Each pass is a
// kernel over small tiles (16 columns or 16 rows), so many blocks share an SM
// and their load, compute and store phases overlap; the intermediate goes
// through a scratch buffer S[unit][sub][N].
constexpr int kTile2 = 16;      // columns (or rows) per block
constexpr int kThr2 = 128;      // threads per block

// column pass: N1-point transforms on the kTile2 columns held as sm[i * cs + cc]
template <bool INV, int K>
__device__ __forceinline__ void col_pass(u64* sm, int cs, int k1, int s0, const ulonglong2* __restrict__ tw, u64 q,
                                         u64 q2, int tid, int nthr)
{
    constexpr int R = 1 << K;
    const int tpc = nthr / cs;                 // threads per column
    const int cc = tid % cs, gt = tid / cs;
    const int ngroups = (1 << k1) >> K;
    // forward: ltb = k1 - s0 - K (smallest distance); inverse: s0 is lt0 (smallest distance)
    const int lsh = INV ? s0 : (k1 - s0 - K);
    for (int gi = gt; gi < ngroups; gi += tpc) {
        const int g = gi >> lsh;
        const int r = gi & ((1 << lsh) - 1);
        const int i0 = (g << (lsh + K)) + r;
        u64 x[R];
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = sm[(i0 + (m << lsh)) * cs + cc];
        if (!INV) {
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
        } else {
#pragma unroll
            for (int l = 0; l < K; ++l) {
                const int h = 1 << l;
                const ulonglong2* twl = tw + ((1 << k1) >> (s0 + l + 1)) + (g << (K - l - 1));
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
        }
#pragma unroll
        for (int m = 0; m < R; ++m) sm[(i0 + (m << lsh)) * cs + cc] = x[m];
    }
}

// row pass: N2-point segments of the full transform on the rows held as
// sm[ri * pitch + spad(c)], row ri being global row rbase + ri
template <bool INV, int K>
__device__ __forceinline__ void row_pass(u64* sm, int rs, int pitch, int k1, int k2, int s0, int rbase,
                                         const ulonglong2* __restrict__ tw, u64 q, u64 q2, int tid, int nthr)
{
    constexpr int R = 1 << K;
    const int tpr = nthr / rs;                 // threads per row
    const int ri = tid / tpr, gt = tid % tpr;
    const int i = rbase + ri;
    const int N = 1 << (k1 + k2);
    const int ngroups = (1 << k2) >> K;
    const int lsh = INV ? s0 : (k2 - s0 - K);
    u64* row = sm + ri * pitch;
    for (int gi = gt; gi < ngroups; gi += tpr) {
        const int g = gi >> lsh;
        const int r = gi & ((1 << lsh) - 1);
        const int c0 = (g << (lsh + K)) + r;
        u64 x[R];
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = row[spad(c0 + (m << lsh))];
        if (!INV) {
            const int gf = (i << s0) + g;                 // group index in the full transform
#pragma unroll
            for (int l = 0; l < K; ++l) {
                const int h = R >> (l + 1);
                const ulonglong2* twl = tw + (1 << (k1 + s0 + l)) + ((size_t)gf << l);
#pragma unroll
                for (int m = 0; m < (1 << l); ++m) {
                    const ulonglong2 w = __ldg(&twl[m]);
#pragma unroll
                    for (int t = 0; t < h; ++t) {
                        const int ii = m * 2 * h + t;
                        u64 X = x[ii];
                        X = X >= q2 ? X - q2 : X;
                        const u64 T = mul_shoup_lazy(x[ii + h], w.x, w.y, q);
                        x[ii] = X + T;
                        x[ii + h] = X + q2 - T;
                    }
                }
            }
        } else {
            const int gf = (i << (k2 - s0 - K)) + g;
#pragma unroll
            for (int l = 0; l < K; ++l) {
                const int h = 1 << l;
                const ulonglong2* twl = tw + (N >> (s0 + l + 1)) + ((size_t)gf << (K - l - 1));
#pragma unroll
                for (int m = 0; m < (R >> (l + 1)); ++m) {
                    const ulonglong2 w = __ldg(&twl[m]);
#pragma unroll
                    for (int t = 0; t < h; ++t) {
                        const int ii = m * 2 * h + t;
                        const u64 X = x[ii], Y = x[ii + h];
                        u64 S = X + Y;
                        S = S >= q2 ? S - q2 : S;
                        x[ii] = S;
                        x[ii + h] = mul_shoup_lazy(X + q2 - Y, w.x, w.y, q);
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < R; ++m) row[spad(c0 + (m << lsh))] = x[m];
    }
}

template <bool INV, int LOGR>
__device__ __forceinline__ void col_passes(u64* sm, int cs, int k1, const ulonglong2* tw, u64 q, int tid, int nthr)
{
    const u64 q2 = 2 * q;
    for (int s = 0; s < k1;) {
        const int k = (k1 - s) < LOGR ? (k1 - s) : LOGR;
        switch (k) {
        case 4: col_pass<INV, 4>(sm, cs, k1, s, tw, q, q2, tid, nthr); break;
        case 3: col_pass<INV, 3>(sm, cs, k1, s, tw, q, q2, tid, nthr); break;
        case 2: col_pass<INV, 2>(sm, cs, k1, s, tw, q, q2, tid, nthr); break;
        default: col_pass<INV, 1>(sm, cs, k1, s, tw, q, q2, tid, nthr); break;
        }
        __syncthreads();
        s += k;
    }
}

template <bool INV, int LOGR>
__device__ __forceinline__ void row_passes(u64* sm, int rs, int pitch, int k1, int k2, int rbase, const ulonglong2* tw,
                                           u64 q, int tid, int nthr)
{
    const u64 q2 = 2 * q;
    for (int s = 0; s < k2;) {
        const int k = (k2 - s) < LOGR ? (k2 - s) : LOGR;
        switch (k) {
        case 4: row_pass<INV, 4>(sm, rs, pitch, k1, k2, s, rbase, tw, q, q2, tid, nthr); break;
        case 3: row_pass<INV, 3>(sm, rs, pitch, k1, k2, s, rbase, tw, q, q2, tid, nthr); break;
        case 2: row_pass<INV, 2>(sm, rs, pitch, k1, k2, s, rbase, tw, q, q2, tid, nthr); break;
        default: row_pass<INV, 1>(sm, rs, pitch, k1, k2, s, rbase, tw, q, q2, tid, nthr); break;
        }
        __syncthreads();
        s += k;
    }
}

struct Split2 {
    int k1, k2;          // N1 = 2^k1 rows, N2 = 2^k2 columns
    int cs, rs;          // columns / rows per block
    int p0, nunits;      // unit range of this chunk
};

// First pass: prologue (op.load) + column passes (forward) or row passes
// (inverse); writes the partial transform to S[(pp * ns + u) * N + j].
// Blocks: (pp, u, tile) with tile = column slab (forward) or row slab (inverse).
template <bool INV, int LOGR, class Op>
__global__ void __launch_bounds__(kThr2) k_ntt2_first(Op op, NttTables T, Split2 sp, u64* __restrict__ S)
{
    extern __shared__ u64 sm[];
    const int k1 = sp.k1, k2 = sp.k2, N1 = 1 << k1, N2 = 1 << k2, N = N1 * N2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ns = op.nsub(sp.p0);
    const int tiles = INV ? N1 / sp.rs : N2 / sp.cs;
    const int tile = blockIdx.x % tiles;
    const int pu = blockIdx.x / tiles;
    const int u = pu % ns, pp = pu / ns, p = sp.p0 + pp;
    if (pp >= sp.nunits || op.direct(p, u)) return;
    const int pi = op.prime(p, u);
    const PrimeC P = T.pc[pi];
    u64* out = S + (size_t)pu * N;
    if (!INV) {
        const int cs = sp.cs, cb = tile * cs, tot = N1 * cs;
        for (int e0 = tid; e0 < tot; e0 += nthr * kUnroll) {
            u64 v[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int e = e0 + k * nthr;
                v[k] = e < tot ? op.load(p, u, (e / cs) * N2 + cb + (e % cs), P) : 0;
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k)
                if (e0 + k * nthr < tot) sm[e0 + k * nthr] = v[k];
        }
        __syncthreads();
        col_passes<false, LOGR>(sm, cs, k1, T.tw_fwd + (size_t)pi * N, P.q, tid, nthr);
        for (int e = tid; e < tot; e += nthr) out[(e / cs) * N2 + cb + (e % cs)] = sm[e];
    } else {
        const int rs = sp.rs, rb = tile * rs, pitch = ntt_smem_words(N2), tot = rs * N2;
        for (int e0 = tid; e0 < tot; e0 += nthr * kUnroll) {
            u64 v[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int e = e0 + k * nthr;
                v[k] = e < tot ? op.load(p, u, rb * N2 + e, P) : 0;
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const int e = e0 + k * nthr;
                if (e < tot) sm[(e / N2) * pitch + spad(e % N2)] = v[k];
            }
        }
        __syncthreads();
        row_passes<true, LOGR>(sm, rs, pitch, k1, k2, rb, T.tw_inv + (size_t)pi * N, P.q, tid, nthr);
        for (int e = tid; e < tot; e += nthr) out[rb * N2 + e] = sm[(e / N2) * pitch + spad(e % N2)];
    }
}

// Second pass: for every sub u of the unit in order, read its partial
// transform (unless direct), finish it (row passes forward, column passes
// inverse) and run the epilogue (op.pre / op.store) on this block's tile.
template <bool INV, int LOGR, class Op>
__global__ void __launch_bounds__(kThr2) k_ntt2_second(Op op, NttTables T, Split2 sp, const u64* __restrict__ S)
{
    extern __shared__ u64 sm[];
    const int k1 = sp.k1, k2 = sp.k2, N1 = 1 << k1, N2 = 1 << k2, N = N1 * N2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tiles = INV ? N2 / sp.cs : N1 / sp.rs;
    const int tile = blockIdx.x % tiles;
    const int pp = blockIdx.x / tiles;
    if (pp >= sp.nunits) return;
    const int p = sp.p0 + pp;
    const int ns = op.nsub(p);
    for (int u = 0; u < ns; ++u) {
        const int pi = op.prime(p, u);
        const PrimeC P = T.pc[pi];
        const bool dir = op.direct(p, u);
        const u64* in = S + ((size_t)pp * ns + u) * N;
        if (!INV) {
            const int rs = sp.rs, rb = tile * rs, pitch = ntt_smem_words(N2), tot = rs * N2;
            if (!dir) {
                for (int e = tid; e < tot; e += nthr) sm[(e / N2) * pitch + spad(e % N2)] = in[rb * N2 + e];
                __syncthreads();
                row_passes<false, LOGR>(sm, rs, pitch, k1, k2, rb, T.tw_fwd + (size_t)pi * N, P.q, tid, nthr);
            }
            for (int e0 = tid; e0 < tot; e0 += nthr * kUnroll) {
                typename Op::Pre pr[kUnroll];
                u64 v[kUnroll];
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    const int e = e0 + k * nthr;
                    if (e < tot) {
                        pr[k] = op.pre(p, u, rb * N2 + e);
                        v[k] = dir ? 0 : fwd_out<Op>(sm[(e / N2) * pitch + spad(e % N2)], P.q);
                    }
                }
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    const int e = e0 + k * nthr;
                    if (e < tot) op.store(p, u, rb * N2 + e, v[k], pr[k], P);
                }
            }
        } else {
            const int cs = sp.cs, cb = tile * cs, tot = N1 * cs;
            if (!dir) {
                for (int e = tid; e < tot; e += nthr) sm[e] = in[(e / cs) * N2 + cb + (e % cs)];
                __syncthreads();
                col_passes<true, LOGR>(sm, cs, k1, T.tw_inv + (size_t)pi * N, P.q, tid, nthr);
            }
            for (int e0 = tid; e0 < tot; e0 += nthr * kUnroll) {
                typename Op::Pre pr[kUnroll];
                u64 v[kUnroll];
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    const int e = e0 + k * nthr;
                    if (e < tot) {
                        const int j = (e / cs) * N2 + cb + (e % cs);
                        pr[k] = op.pre(p, u, j);
                        v[k] = dir ? 0 : inv_final(sm[e], P);
                    }
                }
#pragma unroll
                for (int k = 0; k < kUnroll; ++k) {
                    const int e = e0 + k * nthr;
                    if (e < tot) op.store(p, u, (e / cs) * N2 + cb + (e % cs), v[k], pr[k], P);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- fused-I/O transform
// Same transform, but the first register pass reads its group straight from
// the prologue (op.load: the group's 2^K global loads issued together) and
// the last register pass hands its group straight to the epilogue
// (op.pre / op.store), so shared memory is only used between passes.
//
// Butterflies come in two forms.  RED: Harvey's, values brought back below
// 2q before each butterfly (forward: X; inverse: the sum).  Unreduced, for
// small primes: the Shoup product stays in [0, 2q) for any 64-bit
// multiplicand, so nothing else needs reducing while the values fit 64 bits.
//  - forward (q < kFwdNoRedBound): X is used as it is and both outputs grow
//    by at most 2q per stage, so inputs in [0, 4q) end below
//    (4 + 2 logN) q <= 36 q < 2^64 for logN <= 16; the epilogue reduces once;
//  - inverse (q < kInvNoRedBound): the sum X + Y is kept as it is, so after
//    global stage s every value is below 2^s 2q; the difference is taken as
//    X + 2^s 2q - Y >= 0.  After logN <= 16 stages values are below
//    2^17 q < 2^64 and the final product by N^{-1} (a Shoup product, valid
//    for any 64-bit input) reduces them.
constexpr u64 kFwdNoRedBound = 1ull << 58;
constexpr u64 kInvNoRedBound = 1ull << 46;

//
// fetch(R, j0, lsh) runs before a group's values are read: the epilogue uses
// it to issue the first batch of its global loads, whose latency then hides
// behind the group's loads and butterflies; put(R, j0, lsh, x, fetched).
struct NoFetch {};

// The butterflies of one group: the 2^K values x[i] = a[j0 + i 2^lsh] of a
// pass starting at global stage s0, g being the group's index at that stage
// (forward: j >> (logN - s0); inverse: j >> (s0 + K)).
//  - forward, stage s0 + l: pairs (i, i + h), h = 2^(K-1-l), i = m 2h + t,
//    twiddle psi_rev[2^(s0+l) + g 2^l + m];
//  - inverse, stage s0 + l: pairs (i, i + h), h = 2^l, i = m 2h + t,
//    twiddle psi_rev^-1[N / 2^(s0+l+1) + g 2^(K-1-l) + m].
// Each stage is its own instantiation (bfly_*_from<K, RED, l>), so every loop
// has a constant trip count and x stays in registers (with the stage index a
// loop variable the inverse kept x in local memory).
template <int K, bool RED, int l>
__device__ __forceinline__ void bfly_fwd_from(u64* x, const ulonglong2* __restrict__ tw, int s0, int g, u64 q, u64 q2)
{
    if constexpr (l < K) {
        constexpr int R = 1 << K, h = R >> (l + 1);
        const ulonglong2* twl = tw + (1 << (s0 + l)) + (g << l);
#pragma unroll
        for (int m = 0; m < (1 << l); ++m) {
            const ulonglong2 w = __ldg(&twl[m]);
#pragma unroll
            for (int t = 0; t < h; ++t) {
                const int i = m * 2 * h + t;
                u64 X = x[i];
                if (RED) X = X >= q2 ? X - q2 : X;
                const u64 T = mul_shoup_lazy(x[i + h], w.x, w.y, q);
                x[i] = X + T;
                x[i + h] = X + q2 - T;
            }
        }
        bfly_fwd_from<K, RED, l + 1>(x, tw, s0, g, q, q2);
    }
}

template <int K, bool RED>
__device__ __forceinline__ void bfly_fwd(u64* x, const ulonglong2* __restrict__ tw, int s0, int g, u64 q, u64 q2)
{
    bfly_fwd_from<K, RED, 0>(x, tw, s0, g, q, q2);
}

template <int K, bool RED, int l>
__device__ __forceinline__ void bfly_inv_from(u64* x, const ulonglong2* __restrict__ tw, int N, int s0, int g, u64 q,
                                              u64 q2)
{
    if constexpr (l < K) {
        constexpr int R = 1 << K, h = 1 << l;
        const ulonglong2* twl = tw + (N >> (s0 + l + 1)) + (g << (K - l - 1));
        const u64 c = RED ? q2 : (q2 << (s0 + l));       // bound of Y at this stage
#pragma unroll
        for (int m = 0; m < (R >> (l + 1)); ++m) {
            const ulonglong2 w = __ldg(&twl[m]);
#pragma unroll
            for (int t = 0; t < h; ++t) {
                const int i = m * 2 * h + t;
                const u64 X = x[i], Y = x[i + h];
                u64 S = X + Y;
                if (RED) S = S >= q2 ? S - q2 : S;
                x[i] = S;
                x[i + h] = mul_shoup_lazy(X + c - Y, w.x, w.y, q);
            }
        }
        bfly_inv_from<K, RED, l + 1>(x, tw, N, s0, g, q, q2);
    }
}

template <int K, bool RED>
__device__ __forceinline__ void bfly_inv(u64* x, const ulonglong2* __restrict__ tw, int logN, int s0, int g, u64 q,
                                         u64 q2)
{
    bfly_inv_from<K, RED, 0>(x, tw, 1 << logN, s0, g, q, q2);
}

// Five stages on 32 values as one stage over all of them and two independent
// 16-value groups (forward; the inverse in the opposite order), so fewer
// twiddles are live at once than in one 32-value group (less spilling).
template <bool RED>
__device__ __forceinline__ void bfly_fwd32(u64* x, const ulonglong2* __restrict__ tw, int s0, int g, u64 q, u64 q2)
{
    {
        const ulonglong2 w = __ldg(&tw[(1 << s0) + g]);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            u64 X = x[i];
            if (RED) X = X >= q2 ? X - q2 : X;
            const u64 T = mul_shoup_lazy(x[i + 16], w.x, w.y, q);
            x[i] = X + T;
            x[i + 16] = X + q2 - T;
        }
    }
    bfly_fwd<4, RED>(x, tw, s0 + 1, 2 * g, q, q2);
    bfly_fwd<4, RED>(x + 16, tw, s0 + 1, 2 * g + 1, q, q2);
}

template <bool RED>
__device__ __forceinline__ void bfly_inv32(u64* x, const ulonglong2* __restrict__ tw, int logN, int s0, int g, u64 q,
                                           u64 q2)
{
    bfly_inv<4, RED>(x, tw, logN, s0, 2 * g, q, q2);
    bfly_inv<4, RED>(x + 16, tw, logN, s0, 2 * g + 1, q, q2);
    const ulonglong2 w = __ldg(&tw[((1 << logN) >> (s0 + 5)) + g]);
    const u64 c = RED ? q2 : (q2 << (s0 + 4));
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const u64 X = x[i], Y = x[i + 16];
        u64 S = X + Y;
        if (RED) S = S >= q2 ? S - q2 : S;
        x[i] = S;
        x[i + 16] = mul_shoup_lazy(X + c - Y, w.x, w.y, q);
    }
}

// sh, goff (forward only): the pass works on one half of a larger transform
// (k_ntt_half_io): its local stage s is global stage s + sh, and its local
// group g is global group g + goff at the pass's first stage.
// tail: the last pass of the warp-local tail of a 16384-point forward
// transform (4096 groups of 4): with per = 4096 / (2 nthr) groups per lane in
// each half, warp w takes the groups of [32 per 4 w + 8192 h, + 32 per 4),
// h = 0, 1: the elements it wrote in the pass before (see ntt_io_unit).
template <bool INV, int K, bool RED, class Get, class Put, class Fetch>
__device__ __forceinline__ void pass_io(int logN, int s0, const ulonglong2* __restrict__ tw, u64 q, u64 q2, int tid,
                                        int nthr, Get& get, Put& put, Fetch& fetch, int sh = 0, int goff = 0,
                                        bool tail = false)
{
    constexpr int R = 1 << K;
    const int N = 1 << logN;
    const int lsh = INV ? s0 : (logN - s0 - K);
    const int ngroups = N >> K;
    auto group = [&](int gi) {
        const int g = gi >> lsh;
        const int r = gi & ((1 << lsh) - 1);
        const int j0 = (g << (lsh + K)) + r;
        auto fetched = fetch(std::integral_constant<int, R>{}, j0, lsh);
        u64 x[R];
        get(std::integral_constant<int, R>{}, j0, lsh, x);
        if (!INV) bfly_fwd<K, RED>(x, tw, s0 + sh, g + goff, q, q2);
        else bfly_inv<K, RED>(x, tw, logN, s0, g, q, q2);
        put(std::integral_constant<int, R>{}, j0, lsh, x, fetched);
    };
    if (tail) {
        const int per = ngroups / (2 * nthr);
        const int base = (tid >> 5) * 32 * per + (tid & 31);
        for (int h = 0; h < 2; ++h)
            for (int k = 0; k < per; ++k) group(h * (ngroups >> 1) + base + k * 32);
    } else {
        for (int gi = tid; gi < ngroups; gi += nthr) group(gi);
    }
}

template <bool INV, int KMAX, bool RED, class Get, class Put, class Fetch>
__device__ __forceinline__ void pass_io_k(int k, int logN, int s0, const ulonglong2* tw, u64 q, u64 q2, int tid, int nthr,
                                          Get& get, Put& put, Fetch& fetch, int sh = 0, int goff = 0, bool tail = false)
{
    if constexpr (KMAX >= 1) {
        if (k == KMAX) {
            pass_io<INV, KMAX, RED>(logN, s0, tw, q, q2, tid, nthr, get, put, fetch, sh, goff, tail);
            return;
        }
        pass_io_k<INV, KMAX - 1, RED>(k, logN, s0, tw, q, q2, tid, nthr, get, put, fetch, sh, goff, tail);
    }
}

template <class Pre, int B>
struct PreBatch {
    Pre v[B];
};

// forward outputs of the unreduced form, below 36 q: a lazy-store Op takes
// them as they are, any other Op gets them reduced into [0, q)
template <class Op>
__device__ __forceinline__ u64 fwd_out_wide(u64 x, const PrimeC& P)
{
    if constexpr (lazy_store<Op>::value) return x;
    else return reduce64(x, P);
}

// epilogue pre-loads issued together: two at 64 registers per thread (more
// spill), up to eight with the 128 registers of the 512-thread schedules
// (measured on the key-switching step: 8 and 16 beat 4 and 2)
constexpr int kEpiBatch = 2;
constexpr int kEpiBatchWide = 8;
// epilogue loads issued before the last pass's butterflies: four with the
// 128 registers of the 512-thread schedules, none at 64 (they would spill)
template <int MAXT>
constexpr int kEpiPrefetch = MAXT <= 512 ? 4 : 0;

// one unit p of a fused-I/O transform step (all its sub-transforms, in
// order) by the calling block; shared memory sm holds ntt_smem_words(N) words
template <bool INV, int LOGR, int MAXT, class Op>
__device__ __forceinline__ void ntt_io_unit(const Op& op, const NttTables& T, int p, u64* sm)
{
    const int logN = T.logN;
    const int N = 1 << logN;
    const int tid = threadIdx.x, nthr = blockDim.x;
    {
        const int ns = op.nsub(p);
        for (int u = 0; u < ns; ++u) {
            const int pi = op.prime(p, u);
            const PrimeC P = T.pc[pi];
            if (op.direct(p, u)) {
                for (int j = tid; j < N; j += nthr) op.store(p, u, j, 0, op.pre(p, u, j), P);
                __syncthreads();
                continue;
            }
            const u64 q = P.q, q2 = 2 * P.q;
            const bool wide = !cold_path<Op>::value && q < (INV ? kInvNoRedBound : kFwdNoRedBound);  // block-uniform
            const ulonglong2* tw = (INV ? T.tw_inv : T.tw_fwd) + (size_t)pi * N;
            // 16384 points, radix 8 on 1024 threads or radix 16 on 512: the
            // inverse passes at stages 0 and 3 (radix 8) or 4 (radix 16), and
            // with radix 8 the forward passes at stages 6, 9 and 12 (the last
            // with its groups assigned to match, pass_io's tail), stay within
            // blocks of 256 or 512 elements that one warp writes and reads, so
            // those passes are separated by warp barriers only (a radix-16
            // forward tail would add a second copy of the last pass and its
            // epilogue, which doubled the spills of the persistent kernel's
            // forward units)
            const bool warp_tail = logN == 14 && ((LOGR == 3 && MAXT == 1024 && nthr == 1024) ||
                                                  (LOGR == 4 && MAXT == 512 && nthr == 512));
            int s = 0;
            bool first = true;
            while (s < logN) {
                // the remainder pass comes last: a small-radix last pass keeps the
                // epilogue's registers free (the remainder first measured 37% slower
                // on the key-switching step)
                const int k = (logN - s) < LOGR ? (logN - s) : LOGR;
                const bool last = s + k >= logN;
                auto gload = [&](auto Rc, int j0, int lsh, u64* x) {
                    constexpr int R = decltype(Rc)::value;
#pragma unroll
                    for (int i = 0; i < R; ++i) x[i] = op.load(p, u, j0 + (i << lsh), P);
                };
                auto gsm = [&](auto Rc, int j0, int lsh, u64* x) {
                    constexpr int R = decltype(Rc)::value;
#pragma unroll
                    for (int i = 0; i < R; ++i) x[i] = sm[spad(j0 + (i << lsh))];
                };
                auto psm = [&](auto Rc, int j0, int lsh, u64* x, NoFetch) {
                    constexpr int R = decltype(Rc)::value;
#pragma unroll
                    for (int i = 0; i < R; ++i) sm[spad(j0 + (i << lsh))] = x[i];
                };
                constexpr int EB = MAXT <= 512 ? kEpiBatchWide : kEpiBatch;
                auto nofetch = [&](auto, int, int) { return NoFetch{}; };
                // the first PF elements' loads are issued before the
                // butterflies, the rest in batches of EB after them
                auto efetch = [&](auto Rc, int j0, int lsh) {
                    constexpr int R = decltype(Rc)::value;
                    constexpr int PF = R < kEpiPrefetch<MAXT> ? R : kEpiPrefetch<MAXT>;
                    if constexpr (PF == 0) {
                        return NoFetch{};
                    } else {
                        PreBatch<typename Op::Pre, PF> f;
#pragma unroll
                        for (int i = 0; i < PF; ++i) f.v[i] = op.pre(p, u, j0 + (i << lsh));
                        return f;
                    }
                };
                auto pepi = [&](auto Rc, int j0, int lsh, u64* x, const auto& f) {
                    constexpr int R = decltype(Rc)::value;
                    constexpr int PF = R < kEpiPrefetch<MAXT> ? R : kEpiPrefetch<MAXT>;
                    constexpr int B = R < EB ? R : EB;
                    auto out = [&](int i, const typename Op::Pre& pr) {
                        op.store(p, u, j0 + (i << lsh),
                                 INV    ? inv_final(x[i], P)
                                 : wide ? fwd_out_wide<Op>(x[i], P)
                                        : fwd_out<Op>(x[i], q),
                                 pr, P);
                    };
                    if constexpr (PF > 0) {
#pragma unroll
                        for (int i = 0; i < PF; ++i) out(i, f.v[i]);
                    }
#pragma unroll
                    for (int i0 = PF; i0 < R; i0 += B) {
                        typename Op::Pre pr[B];
#pragma unroll
                        for (int i = 0; i < B; ++i)
                            if (i0 + i < R) pr[i] = op.pre(p, u, j0 + ((i0 + i) << lsh));
#pragma unroll
                        for (int i = 0; i < B; ++i)
                            if (i0 + i < R) out(i0 + i, pr[i]);
                    }
                };
                const bool tail = !INV && LOGR == 3 && warp_tail && last;
                auto run = [&](auto redc, auto& get, auto& put, auto& fetch) {
                    pass_io_k<INV, LOGR, decltype(redc)::value>(k, logN, s, tw, q, q2, tid, nthr, get, put, fetch, 0, 0,
                                                                tail);
                };
                auto run_rw = [&](auto& get, auto& put, auto& fetch) {
                    if constexpr (cold_path<Op>::value) {
                        run(std::true_type{}, get, put, fetch);
                    } else {
                        if (wide) run(std::false_type{}, get, put, fetch);
                        else run(std::true_type{}, get, put, fetch);
                    }
                };
                if (first && last) run_rw(gload, pepi, efetch);
                else if (first) run_rw(gload, psm, nofetch);
                else if (last) run_rw(gsm, pepi, efetch);
                else run_rw(gsm, psm, nofetch);
                // the next pass reads only what this warp wrote: forward after
                // stages 6 and 9 (radix 8) or 8 (radix 16), inverse after stage 0
                const bool wsync = INV ? s == 0 : (LOGR == 3 && (s == 6 || s == 9));
                if (warp_tail && !last && wsync) __syncwarp();
                else __syncthreads();
                first = false;
                s += k;
            }
        }
    }
}

template <bool INV, int LOGR, int MAXT, class Op>
__global__ void __launch_bounds__(MAXT, 1) k_ntt_io(Op op, NttTables T)
{
    extern __shared__ u64 sm[];
    for (int p = blockIdx.x; p < op.count(); p += gridDim.x) ntt_io_unit<INV, LOGR, MAXT>(op, T, p, sm);
}

// ---------------------------------------------------------------- warp-local transforms
// One block of N/32 threads per residue polynomial, 1024 <= N <= 16384 (a
// larger block works too: its extra warps take part in the block stages and
// barriers only).
// After the first logN - 10 stages (distances N/2 .. 1024, forward) the
// array falls apart into N/1024 independent 1024-point problems on
// contiguous blocks; warp w owns block [1024 w, 1024 w + 1024), 32 values
// per lane, and runs its ten stages with warp-level synchronisation only:
//   five stages with lane l holding elements 1024 w + l + 32 i (i = 0..31:
//   the pairs at distances 512 .. 32 are in one lane), then, after a
//   transpose through shared memory, five with lane l holding 1024 w + 32 l
//   + i (distances 16 .. 1).
// So a forward transform takes one block-wide barrier (after the first
// logN - 10 stages, done by the whole block on groups of 2^(logN-10) values
// at stride 1024) instead of one per register pass, and every global access
// (the prologue's loads, the epilogue's loads and stores, which go through
// shared memory once more) is coalesced.  The inverse runs the same steps in
// the opposite order (warp stages 0..9, barrier, block stages 10..logN-1).
// The five stages whose twiddles differ per lane (forward: the last five,
// inverse: the first five) read them from tables transposed by wl_perm, so
// the lanes of a warp read consecutive entries.
// Shared-memory word j sits at j + j/32: conflict-free for lanes reading
// consecutive words and for lanes reading words 32 apart.
__device__ __forceinline__ int wpad(int j) { return j + (j >> 5); }

__host__ __device__ constexpr int ntt_wl_smem_words(int N) { return N + (N >> 5); }

constexpr int kWlEpiBatch = 8;

// the block stages of a forward transform (0 .. KA-1, KA = logN - 10):
// group gi in [0, 1024) is the 2^KA values gi + 1024 i, read by the prologue
template <int KA, bool RED, class Op>
__device__ __forceinline__ void wl_fwd_block(const Op& op, int p, int u, const PrimeC& P,
                                             const ulonglong2* __restrict__ tw, u64* sm, int tid, int nthr)
{
    constexpr int R = 1 << KA;
#pragma unroll 1
    for (int gi = tid; gi < 1024; gi += nthr) {
        u64 x[R];
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = op.load(p, u, gi + (i << 10), P);
        bfly_fwd<KA, RED>(x, tw, 0, 0, P.q, P.q2);
        u64* const g = sm + wpad(gi);         // element gi + 1024 i at g[1056 i]
#pragma unroll
        for (int i = 0; i < R; ++i) g[1056 * i] = x[i];
    }
}

// the block stages of an inverse transform (10 .. logN-1) from shared memory,
// each group's outputs (times N^-1) handed to the epilogue
template <int KA, bool RED, class Op>
__device__ __forceinline__ void wl_inv_block(const Op& op, int p, int u, const PrimeC& P,
                                             const ulonglong2* __restrict__ tw, const u64* sm, int logN, int tid,
                                             int nthr)
{
    constexpr int R = 1 << KA;
    constexpr int B = R < kWlEpiBatch ? R : kWlEpiBatch;
#pragma unroll 1
    for (int gi = tid; gi < 1024; gi += nthr) {
        u64 x[R];
        const u64* const g = sm + wpad(gi);   // element gi + 1024 i at g[1056 i]
#pragma unroll
        for (int i = 0; i < R; ++i) x[i] = g[1056 * i];
        bfly_inv<KA, RED>(x, tw, logN, 10, 0, P.q, P.q2);
#pragma unroll
        for (int i0 = 0; i0 < R; i0 += B) {
            typename Op::Pre pr[B];
#pragma unroll
            for (int i = 0; i < B; ++i) pr[i] = op.pre(p, u, gi + ((i0 + i) << 10));
#pragma unroll
            for (int i = 0; i < B; ++i) op.store(p, u, gi + ((i0 + i) << 10), inv_final(x[i0 + i], P), pr[i], P);
        }
    }
}

// Position, within a stage's block of a warp-local twiddle table, of the
// entry at natural offset k, for a stage at which each lane of a warp needs
// 2^u consecutive entries: k = (w 32 + lane) 2^u + m (m < 2^u) is stored at
// (w 2^u + m) 32 + lane, so lanes read consecutive entries for each m.
__host__ __device__ constexpr uint32_t wl_perm(uint32_t k, int u)
{
    return ((k >> (u + 5)) << (u + 5)) | ((k & ((1u << u) - 1)) << 5) | ((k >> u) & 31u);
}

// The five lane-varying stages of the warp-local forward transform (global
// stages sb .. sb+4, sb = log2 N - 5) on lane `lane` of warp w, its 32 values
// x[i] = a[1024 w + 32 lane + i], twiddles from the transposed table: one
// stage over all 32 values, then two independent 16-value halves h.
template <int K, bool RED, int l>
__device__ __forceinline__ void bfly_fwd_lanes_from(u64* x, const ulonglong2* __restrict__ tw, int sb, int w, int lane,
                                                    int h, u64 q, u64 q2)
{
    if constexpr (l < K) {
        constexpr int R = 1 << K, hh = R >> (l + 1), t = l + 1;   // global stage sb + t
        const ulonglong2* twl = tw + (1 << (sb + t)) + ((((w << t) + (h << l))) << 5) + lane;
#pragma unroll
        for (int m = 0; m < (1 << l); ++m) {
            const ulonglong2 wv = __ldg(&twl[m << 5]);
#pragma unroll
            for (int tt = 0; tt < hh; ++tt) {
                const int i = m * 2 * hh + tt;
                u64 X = x[i];
                if (RED) X = X >= q2 ? X - q2 : X;
                const u64 T = mul_shoup_lazy(x[i + hh], wv.x, wv.y, q);
                x[i] = X + T;
                x[i + hh] = X + q2 - T;
            }
        }
        bfly_fwd_lanes_from<K, RED, l + 1>(x, tw, sb, w, lane, h, q, q2);
    }
}

template <bool RED>
__device__ __forceinline__ void bfly_fwd32_lanes(u64* x, const ulonglong2* __restrict__ tw, int sb, int w, int lane,
                                                 u64 q, u64 q2)
{
    {
        const ulonglong2 wv = __ldg(&tw[(1 << sb) + (w << 5) + lane]);    // 2^0 entries per lane: natural order
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            u64 X = x[i];
            if (RED) X = X >= q2 ? X - q2 : X;
            const u64 T = mul_shoup_lazy(x[i + 16], wv.x, wv.y, q);
            x[i] = X + T;
            x[i + 16] = X + q2 - T;
        }
    }
    bfly_fwd_lanes_from<4, RED, 0>(x, tw, sb, w, lane, 0, q, q2);
    bfly_fwd_lanes_from<4, RED, 0>(x + 16, tw, sb, w, lane, 1, q, q2);
}

// The five lane-varying stages of the warp-local inverse transform (global
// stages 0 .. 4) in the same layout: two independent 16-value halves h
// (stages 0 .. 3, 2^(4-s) entries per lane at stage s), then one stage over
// all 32 values.
template <int K, bool RED, int l>
__device__ __forceinline__ void bfly_inv_lanes_from(u64* x, const ulonglong2* __restrict__ tw, int N, int w, int lane,
                                                    int h, u64 q, u64 q2)
{
    if constexpr (l < K) {
        constexpr int R = 1 << K, hh = 1 << l, u = K - l;            // global stage l
        const ulonglong2* twl = tw + (N >> (l + 1)) + ((((w << u) + (h << (K - l - 1)))) << 5) + lane;
        const u64 c = RED ? q2 : (q2 << l);
#pragma unroll
        for (int m = 0; m < (R >> (l + 1)); ++m) {
            const ulonglong2 wv = __ldg(&twl[m << 5]);
#pragma unroll
            for (int tt = 0; tt < hh; ++tt) {
                const int i = m * 2 * hh + tt;
                const u64 X = x[i], Y = x[i + hh];
                u64 S = X + Y;
                if (RED) S = S >= q2 ? S - q2 : S;
                x[i] = S;
                x[i + hh] = mul_shoup_lazy(X + c - Y, wv.x, wv.y, q);
            }
        }
        bfly_inv_lanes_from<K, RED, l + 1>(x, tw, N, w, lane, h, q, q2);
    }
}

template <bool RED>
__device__ __forceinline__ void bfly_inv32_lanes(u64* x, const ulonglong2* __restrict__ tw, int logN, int w, int lane,
                                                 u64 q, u64 q2)
{
    const int N = 1 << logN;
    bfly_inv_lanes_from<4, RED, 0>(x, tw, N, w, lane, 0, q, q2);
    bfly_inv_lanes_from<4, RED, 0>(x + 16, tw, N, w, lane, 1, q, q2);
    const ulonglong2 wv = __ldg(&tw[(N >> 5) + (w << 5) + lane]);         // natural order
    const u64 c = RED ? q2 : (q2 << 4);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const u64 X = x[i], Y = x[i + 16];
        u64 S = X + Y;
        if (RED) S = S >= q2 ? S - q2 : S;
        x[i] = S;
        x[i + 16] = mul_shoup_lazy(X + c - Y, wv.x, wv.y, q);
    }
}

// sub-transform u of unit p; warps beyond the N/1024 that own a
// sub-transform (a block larger than N/32 threads) only take part in the
// block stages and barriers
template <bool INV, bool RED, class Op>
__device__ __forceinline__ void wl_transform(const Op& op, int p, int u, const PrimeC& P,
                                             const ulonglong2* __restrict__ tw, u64* sm, int logN)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int w = tid >> 5, l = tid & 31, b = w << 10;
    const int KA = logN - 10;
    const bool owner = w < (1 << KA);
    const u64 q = P.q, q2 = P.q2;
    // the warp's two layouts in shared memory (index j + j/32, l < 32):
    // element b + l + 32 i at smA[33 i], element b + 32 l + i at smB[i]
    u64* const smA = sm + wpad(b + l);
    u64* const smB = sm + wpad(b + 32 * l);
    u64 x[32];
    if (!INV) {
        if (KA > 0) {
            switch (KA) {
            case 1: wl_fwd_block<1, RED>(op, p, u, P, tw, sm, tid, nthr); break;
            case 2: wl_fwd_block<2, RED>(op, p, u, P, tw, sm, tid, nthr); break;
            case 3: wl_fwd_block<3, RED>(op, p, u, P, tw, sm, tid, nthr); break;
            default: wl_fwd_block<4, RED>(op, p, u, P, tw, sm, tid, nthr); break;
            }
            __syncthreads();
        }
        if (!owner) return;
        if (KA == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = op.load(p, u, l + 32 * i, P);
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = smA[33 * i];
        }
        // stages KA .. KA+4 (distances 512 .. 32 within the block of warp w)
        bfly_fwd32<RED>(x, tw, KA, w, q, q2);
#pragma unroll
        for (int i = 0; i < 32; ++i) smA[33 * i] = x[i];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = smB[i];
        // stages KA+5 .. logN-1 (distances 16 .. 1), twiddles per lane
        bfly_fwd32_lanes<RED>(x, tw, KA + 5, w, l, q, q2);
#pragma unroll
        for (int i = 0; i < 32; ++i) smB[i] = x[i];
        __syncwarp();
        // epilogue, coalesced: element b + l + 32 i
#pragma unroll 1
        for (int i0 = 0; i0 < 32; i0 += kWlEpiBatch) {
            typename Op::Pre pr[kWlEpiBatch];
#pragma unroll
            for (int i = 0; i < kWlEpiBatch; ++i) pr[i] = op.pre(p, u, b + l + 32 * (i0 + i));
#pragma unroll
            for (int i = 0; i < kWlEpiBatch; ++i) {
                const int j = b + l + 32 * (i0 + i);
                const u64 v = smA[33 * (i0 + i)];
                op.store(p, u, j, RED ? fwd_out<Op>(v, q) : fwd_out_wide<Op>(v, P), pr[i], P);
            }
        }
    } else {
        if (owner) {
            // coalesced loads, transposed through shared memory
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = op.load(p, u, b + l + 32 * i, P);
#pragma unroll
            for (int i = 0; i < 32; ++i) smA[33 * i] = x[i];
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = smB[i];
            // stages 0 .. 4 (distances 1 .. 16), twiddles per lane
            bfly_inv32_lanes<RED>(x, tw, logN, w, l, q, q2);
#pragma unroll
            for (int i = 0; i < 32; ++i) smB[i] = x[i];
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = smA[33 * i];
            // stages 5 .. 9 (distances 32 .. 512)
            bfly_inv32<RED>(x, tw, logN, 5, w, q, q2);
            if (KA == 0) {
#pragma unroll
                for (int i0 = 0; i0 < 32; i0 += kWlEpiBatch) {
                    typename Op::Pre pr[kWlEpiBatch];
#pragma unroll
                    for (int i = 0; i < kWlEpiBatch; ++i) pr[i] = op.pre(p, u, l + 32 * (i0 + i));
#pragma unroll
                    for (int i = 0; i < kWlEpiBatch; ++i)
                        op.store(p, u, l + 32 * (i0 + i), inv_final(x[i0 + i], P), pr[i], P);
                }
                return;
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) smA[33 * i] = x[i];
        }
        if (KA > 0) {
            __syncthreads();
            switch (KA) {
            case 1: wl_inv_block<1, RED>(op, p, u, P, tw, sm, logN, tid, nthr); break;
            case 2: wl_inv_block<2, RED>(op, p, u, P, tw, sm, logN, tid, nthr); break;
            case 3: wl_inv_block<3, RED>(op, p, u, P, tw, sm, logN, tid, nthr); break;
            default: wl_inv_block<4, RED>(op, p, u, P, tw, sm, logN, tid, nthr); break;
            }
        }
    }
}

// one unit p (all its sub-transforms) by the calling block of at least N/32
// threads (a multiple of 32); shared memory sm holds ntt_wl_smem_words(N) words
template <bool INV, class Op>
__device__ __forceinline__ void ntt_wl_unit(const Op& op, const NttTables& T, int p, u64* sm)
{
    const int logN = T.logN;
    const int N = 1 << logN;
    const int ns = op.nsub(p);
    for (int u = 0; u < ns; ++u) {
        const int pi = op.prime(p, u);
        const PrimeC& P = T.pc[pi];
        if (op.direct(p, u)) {
            for (int j = threadIdx.x; j < N; j += blockDim.x) op.store(p, u, j, 0, op.pre(p, u, j), P);
        } else {
            const ulonglong2* tw = (INV ? T.tw_inv_wl : T.tw_fwd_wl) + (size_t)pi * N;
            const bool wide = !cold_path<Op>::value && P.q < (INV ? kInvNoRedBound : kFwdNoRedBound);  // block-uniform
            if constexpr (cold_path<Op>::value) {
                wl_transform<INV, true>(op, p, u, P, tw, sm, logN);
            } else {
                if (wide) wl_transform<INV, false>(op, p, u, P, tw, sm, logN);
                else wl_transform<INV, true>(op, p, u, P, tw, sm, logN);
            }
        }
        // the next sub-transform rewrites shared memory
        __syncthreads();
    }
}

template <bool INV, class Op>
__global__ void __launch_bounds__(512, 1) k_ntt_wl(Op op, NttTables T)
{
    extern __shared__ u64 sm[];
    for (int p = blockIdx.x; p < op.count(); p += gridDim.x) ntt_wl_unit<INV>(op, T, p, sm);
}

// ---------------------------------------------------------------- half transforms
// A forward transform split over two blocks, one per half of the output.  The
// first stage pairs j with j + N/2; after it the halves [0, N/2) and
// [N/2, N) are independent N/2-point problems that keep the full transform's
// twiddles (local stage s is global stage s + 1, local group g of half h is
// global group g + h 2^s).  Each block reads both halves of the input for
// that first stage and keeps only its own outputs (the stage's twiddle
// product is made by both blocks: 1/(2 log2 N) more multiplies), so a block
// holds N/2 words of shared memory and two blocks share an SM: one block's
// loads and epilogue overlap the other's butterflies.  The epilogue of each
// half is independent (the key-switching digit transforms).
// LOGR: radix of the register passes; MINB: blocks per SM the registers are
// budgeted for
template <int MAXT, int LOGR, int MINB, class Op>
__global__ void __launch_bounds__(MAXT, MINB) k_ntt_half_io(Op op, NttTables T)
{
    extern __shared__ u64 sm[];
    const int logN = T.logN;
    const int N = 1 << logN, logNh = logN - 1, Nh = N >> 1;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int b = blockIdx.x; b < 2 * op.count(); b += gridDim.x) {
        const int p = b >> 1, hh = b & 1;
        const int jb = hh * Nh;                      // this half's first coefficient
        const int ns = op.nsub(p);
        for (int u = 0; u < ns; ++u) {
            const int pi = op.prime(p, u);
            const PrimeC P = T.pc[pi];
            if (op.direct(p, u)) {
                for (int j = tid; j < Nh; j += nthr) op.store(p, u, jb + j, 0, op.pre(p, u, jb + j), P);
                __syncthreads();
                continue;
            }
            const u64 q = P.q, q2 = 2 * q;
            const bool wide = !cold_path<Op>::value && q < kFwdNoRedBound;  // block-uniform
            const ulonglong2* tw = T.tw_fwd + (size_t)pi * N;
            const ulonglong2 w1 = __ldg(&tw[1]);    // the first stage's twiddle
            int s = 0;
            bool first = true;
            while (s < logNh) {
                // radix-2^LOGR passes, but never a last pass of one stage
                // (its epilogue would wait for its loads two elements at a time)
                const int rem = logNh - s;
                const int k = rem <= LOGR ? rem : (rem - LOGR == 1 ? LOGR - 1 : LOGR);
                const bool last = s + k >= logNh;
                const int goff = hh << s;
                // first pass: global stage 0 for this half's outputs from both input halves
                auto gload = [&](auto Rc, int j0, int lsh, u64* x) {
                    constexpr int R = decltype(Rc)::value;
                    u64 top[R], bot[R];
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        top[i] = op.load(p, u, j0 + (i << lsh), P);
                        bot[i] = op.load(p, u, Nh + j0 + (i << lsh), P);
                    }
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        u64 X = top[i];
                        if (!wide) X = X >= q2 ? X - q2 : X;
                        const u64 Tv = mul_shoup_lazy(bot[i], w1.x, w1.y, q);
                        x[i] = hh ? X + q2 - Tv : X + Tv;
                    }
                };
                auto gsm = [&](auto Rc, int j0, int lsh, u64* x) {
                    constexpr int R = decltype(Rc)::value;
#pragma unroll
                    for (int i = 0; i < R; ++i) x[i] = sm[spad(j0 + (i << lsh))];
                };
                auto psm = [&](auto Rc, int j0, int lsh, u64* x, NoFetch) {
                    constexpr int R = decltype(Rc)::value;
#pragma unroll
                    for (int i = 0; i < R; ++i) sm[spad(j0 + (i << lsh))] = x[i];
                };
                constexpr int EB = MAXT <= 512 ? kEpiBatchWide : kEpiBatch;
                auto nofetch = [&](auto, int, int) { return NoFetch{}; };
                auto efetch = [&](auto Rc, int j0, int lsh) {
                    constexpr int R = decltype(Rc)::value;
                    constexpr int PF = R < kEpiPrefetch<MAXT> ? R : kEpiPrefetch<MAXT>;
                    if constexpr (PF == 0) {
                        return NoFetch{};
                    } else {
                        PreBatch<typename Op::Pre, PF> f;
#pragma unroll
                        for (int i = 0; i < PF; ++i) f.v[i] = op.pre(p, u, jb + j0 + (i << lsh));
                        return f;
                    }
                };
                auto pepi = [&](auto Rc, int j0, int lsh, u64* x, const auto& f) {
                    constexpr int R = decltype(Rc)::value;
                    constexpr int PF = R < kEpiPrefetch<MAXT> ? R : kEpiPrefetch<MAXT>;
                    constexpr int B = R < EB ? R : EB;
                    auto out = [&](int i, const typename Op::Pre& pr) {
                        op.store(p, u, jb + j0 + (i << lsh), wide ? fwd_out_wide<Op>(x[i], P) : fwd_out<Op>(x[i], q),
                                 pr, P);
                    };
                    if constexpr (PF > 0) {
#pragma unroll
                        for (int i = 0; i < PF; ++i) out(i, f.v[i]);
                    }
#pragma unroll
                    for (int i0 = PF; i0 < R; i0 += B) {
                        typename Op::Pre pr[B];
#pragma unroll
                        for (int i = 0; i < B; ++i)
                            if (i0 + i < R) pr[i] = op.pre(p, u, jb + j0 + ((i0 + i) << lsh));
#pragma unroll
                        for (int i = 0; i < B; ++i)
                            if (i0 + i < R) out(i0 + i, pr[i]);
                    }
                };
                auto run = [&](auto redc, auto& get, auto& put, auto& fetch) {
                    pass_io_k<false, LOGR, decltype(redc)::value>(k, logNh, s, tw, q, q2, tid, nthr, get, put, fetch, 1,
                                                                  goff);
                };
                auto run_rw = [&](auto& get, auto& put, auto& fetch) {
                    if (wide) run(std::false_type{}, get, put, fetch);
                    else run(std::true_type{}, get, put, fetch);
                };
                if (first && last) run_rw(gload, pepi, efetch);
                else if (first) run_rw(gload, psm, nofetch);
                else if (last) run_rw(gsm, pepi, efetch);
                else run_rw(gsm, psm, nofetch);
                __syncthreads();
                first = false;
                s += k;
            }
        }
    }
}
