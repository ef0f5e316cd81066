// launch.cuh -- shared device helpers of the kernel translation units: the
// counter-based sampler, the launch wrappers of the fused transform kernels
// (schedule dispatch, multi-batch wrapper) and element-wise grid sizing.
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "ctx.h"
#include "host_math.h"

namespace fhe {

enum { DOM_SECRET = 1, DOM_PK_A = 2, DOM_PK_E = 3, DOM_KSK_A = 4, DOM_KSK_E = 5,
       DOM_ENC_U = 6, DOM_ENC_E0 = 7, DOM_ENC_E1 = 8, DOM_GAL_A = 9, DOM_GAL_E = 10 };

static constexpr u64 kGamma = 0x9E3779B97F4A7C15ull;

// ---------------------------------------------------------------- PRNG
// SplitMix64 (Steele, Lea, Flood 2014): output i of the generator started in
// state s is mix(s + (i + 1) * gamma).  Draw index = coef | residue << 16 | retry << 24.
__host__ __device__ __forceinline__ u64 mix64(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ u64 sm_out(u64 s, u64 i) { return mix64(s + (i + 1) * kGamma); }

inline uint64_t stream_key(uint64_t seed, uint64_t domain, uint64_t object)
{
    return sm_out(sm_out(seed, domain), object);
}

__device__ __forceinline__ i64 draw_ternary(u64 s0, int j)
{
    const u64 bound = 0xFFFFFFFFFFFFFFFFull;     // 3 * floor(2^64 / 3) = 2^64 - 1
    for (u64 t = 0;; ++t) {
        u64 u = sm_out(s0, (u64)j | (t << 24));
        if (u < bound) return (i64)(u % 3ull) - 1;
    }
}

__device__ __forceinline__ i64 draw_gauss(u64 s0, int j, const u64* __restrict__ cdt)
{
    u64 u = sm_out(s0, (u64)j);
    i64 e = -19;
#pragma unroll
    for (int i = 0; i < 38; ++i) e += (u >= __ldg(&cdt[i])) ? 1 : 0;
    return e;
}

__device__ __forceinline__ u64 draw_uniform(u64 s0, int j, int r, const PrimeC& P)
{
    for (u64 t = 0;; ++t) {
        u64 u = sm_out(s0, (u64)j | ((u64)r << 16) | (t << 24));
        if (u < P.ub) return reduce64(u, P);
    }
}

inline int ew_grid(size_t total)
{
    size_t g = (total + 255) / 256;
    return (int)std::min<size_t>(g, 152 * 32);
}

// ---------------------------------------------------------------- launch
// NTT schedule variants (radix of the register passes, threads per block);
// the context's autotuner picks one per ring degree.
template <bool INV, int LOGR, int MAXT, class Op, bool IO = false>
static void launch_ntt_v(const fhe_ctx* c, const Op& op, int count, cudaStream_t st)
{
    const int N = (int)c->N;
    int thr = N >> LOGR;
    thr = thr < 32 ? 32 : (thr > MAXT ? MAXT : thr);
    const size_t smem = (size_t)ntt_smem_words(N) * sizeof(u64);
    if constexpr (IO) {
        auto fn = k_ntt_io<INV, LOGR, MAXT, Op>;
        ensure_smem((const void*)fn, smem);
        LaunchScope ls(c, Op::family(), st);
        fn<<<count, thr, smem, st>>>(op, c->tabs());
    } else {
        auto fn = k_ntt_op<INV, LOGR, MAXT, Op>;
        ensure_smem((const void*)fn, smem);
        LaunchScope ls(c, Op::family(), st);
        fn<<<count, thr, smem, st>>>(op, c->tabs());
    }
}

// Several batches of one transform step, each with its own level, in ONE
// launch: unit p is located in the group table by prefix sums.
constexpr int kMaxGroups = 8;

// Ops that declare  static constexpr bool kKeySwitchMac = true  (the digit
// transforms with the key inner product in their epilogue) run with the
// schedule the autotuner picked for them, the rest with the general one.
template <class Op, class = void>
struct keyswitch_mac : std::false_type {};
template <class Op>
struct keyswitch_mac<Op, std::void_t<decltype(Op::kKeySwitchMac)>> : std::integral_constant<bool, Op::kKeySwitchMac> {};

// Ops that declare  static constexpr bool kTransformBound = true  (prologue
// and epilogue light on HBM: encryption's samples, the digit inverses) also
// run with the key-switching pick, whose probe is transform-bound too.
template <class Op, class = void>
struct transform_bound : std::false_type {};
template <class Op>
struct transform_bound<Op, std::void_t<decltype(Op::kTransformBound)>>
    : std::integral_constant<bool, Op::kTransformBound> {};

template <class Op>
struct MultiOp {
    static const char* family() { return Op::family(); }
    static constexpr bool kLazyStore = lazy_store<Op>::value;
    static constexpr bool kKeySwitchMac = keyswitch_mac<Op>::value;
    static constexpr bool kTransformBound = transform_bound<Op>::value;
    typedef typename Op::Pre Pre;
    Op ops[kMaxGroups];
    int pre_[kMaxGroups + 1];
    int ng;
    __host__ __device__ int count() const { return pre_[ng]; }
    __host__ __device__ int locate(int p, int& q) const
    {
        int g = 0;
        while (g + 1 < ng && p >= pre_[g + 1]) ++g;
        q = p - pre_[g];
        return g;
    }
    __host__ __device__ int nsub(int p) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].nsub(q);
    }
    __device__ int prime(int p, int u) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].prime(q, u);
    }
    __device__ bool direct(int p, int u) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].direct(q, u);
    }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].load(q, u, j, P);
    }
    __device__ Pre pre(int p, int u, int j) const
    {
        int q;
        const int g = locate(p, q);
        return ops[g].pre(q, u, j);
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        int q;
        const int g = locate(p, q);
        ops[g].store(q, u, j, v, pr, P);
    }
};

// forward transforms split over two blocks per residue polynomial (schedule
// 6, key-switching digit transforms): radix 16 with two blocks per SM
template <class Op, int LOGR = 4, int MINB = 2>
static void launch_ntt_half(const fhe_ctx* c, const Op& op, int count, cudaStream_t st)
{
    const int N = (int)c->N;
    const int thr = std::min(256, std::max(32, (N / 2) >> LOGR));
    const size_t smem = (size_t)ntt_smem_words(N / 2) * sizeof(u64);
    auto fn = k_ntt_half_io<256, LOGR, MINB, Op>;
    ensure_smem((const void*)fn, smem);
    LaunchScope ls(c, Op::family(), st);
    fn<<<2 * count, thr, smem, st>>>(op, c->tabs());
}

// warp-local transforms (schedule 8): one block of N/32 threads per unit
template <bool INV, class Op>
static void launch_ntt_wl(const fhe_ctx* c, const Op& op, int count, cudaStream_t st)
{
    const int N = (int)c->N;
    const size_t smem = (size_t)ntt_wl_smem_words(N) * sizeof(u64);
    auto fn = k_ntt_wl<INV, Op>;
    ensure_smem((const void*)fn, smem);
    LaunchScope ls(c, Op::family(), st);
    fn<<<count, N / 32, smem, st>>>(op, c->tabs());
}

template <class Op> struct uniform_subs { static constexpr bool value = true; };
template <class Op> struct uniform_subs<MultiOp<Op>> { static constexpr bool value = false; };

// two-pass schedule: column / row tiles, intermediate in the context's
// scratch, units processed in chunks that fit it
template <bool INV, int LOGR, class Op>
static void launch_ntt_2pass(const fhe_ctx* c, const Op& op, int count, cudaStream_t st)
{
    Split2 sp;
    sp.k1 = (int)c->logN / 2;
    sp.k2 = (int)c->logN - sp.k1;
    const int N1 = 1 << sp.k1, N2 = 1 << sp.k2, N = (int)c->N;
    sp.cs = N2 < kTile2 ? N2 : kTile2;
    sp.rs = N1 < kTile2 ? N1 : kTile2;
    const int ns = op.nsub(0);
    const size_t words = (size_t)(N1 * sp.cs > sp.rs * ntt_smem_words(N2) ? N1 * sp.cs : sp.rs * ntt_smem_words(N2));
    const size_t smem = words * sizeof(u64);
    int chunk = (int)(c->ntt2_words / ((size_t)ns * N));
    if (chunk < 1) chunk = 1;
    const int t1 = INV ? N1 / sp.rs : N2 / sp.cs;      // tiles of the first pass
    const int t2 = INV ? N2 / sp.cs : N1 / sp.rs;      // tiles of the second pass
    for (int p0 = 0; p0 < count; p0 += chunk) {
        sp.p0 = p0;
        sp.nunits = count - p0 < chunk ? count - p0 : chunk;
        {
            LaunchScope ls(c, Op::family(), st);
            k_ntt2_first<INV, LOGR, Op><<<sp.nunits * ns * t1, kThr2, smem, st>>>(op, c->tabs(), sp, c->d_ntt2);
        }
        {
            LaunchScope ls(c, Op::family(), st);
            k_ntt2_second<INV, LOGR, Op><<<sp.nunits * t2, kThr2, smem, st>>>(op, c->tabs(), sp, c->d_ntt2);
        }
    }
}

// single_pass: the caller's scratch must be the only memory the transform
// touches besides its operands, so the two-pass schedules (whose intermediate
// is the context's scratch) are replaced by their one-block-per-transform form
template <bool INV, class Op>
static void launch_ntt(const fhe_ctx* c, const Op& op, cudaStream_t st, bool single_pass = false)
{
    const int count = op.count();
    if (count <= 0) return;
    // the two-pass schedule needs the same number of transforms in every unit
    // (callers refuse single-pass-only work above kMaxSinglePassN)
    const bool single = single_pass || !uniform_subs<Op>::value;
    const int base = keyswitch_mac<Op>::value || transform_bound<Op>::value ? c->ntt_variant_ks : c->ntt_variant;
    int v = single && (base == 2 || base == 3) ? 1 : base;
    // fewer units than SMs: each unit's latency sets the launch's time, and a
    // 1024-thread block (schedule 4) works on a unit with twice the warps of
    // a warp-local one (schedules fixed by FHE_NTT_VARIANT are kept as given)
    if (v == 8 && !c->ntt_forced && count < c->sms) v = 4;
    switch (v) {
    case 1: launch_ntt_v<INV, 3, 1024>(c, op, count, st); break;
    case 2: launch_ntt_2pass<INV, 4>(c, op, count, st); break;
    case 3: launch_ntt_2pass<INV, 3>(c, op, count, st); break;
    case 4: launch_ntt_v<INV, 3, 1024, Op, true>(c, op, count, st); break;
    case 5: launch_ntt_v<INV, 4, 512, Op, true>(c, op, count, st); break;
    case 6:
    case 7:
        // half transforms: forward key-switching digit transforms only; the
        // rest run as schedule 5 (schedule 7, the ModUp cluster kernel, is
        // launched by launch_modup; other key-switching ops take 6 under it)
        if constexpr (!INV && keyswitch_mac<Op>::value) {
            if (c->N >= 64) {
                launch_ntt_half<Op, 4, 2>(c, op, count, st);
                break;
            }
        }
        launch_ntt_v<INV, 4, 512, Op, true>(c, op, count, st);
        break;
    case 8:
        if (ntt_wl_fits(c->logN)) launch_ntt_wl<INV>(c, op, count, st);
        else launch_ntt_v<INV, 4, 512, Op, true>(c, op, count, st);
        break;
    default: launch_ntt_v<INV, 4, 512>(c, op, count, st); break;
    }
}


}  // namespace fhe
