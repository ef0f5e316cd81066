// k_peak.cu -- integer-pipe ceilings of this GPU, measured: register-resident
// streams of the multiply forms the transforms and key products are built
// from, each with many independent chains per thread so that issue, not
// latency, sets the rate.  They are the denominators of the ALU roofline
// (measurement only; the paper has no counterpart).
//
//   kind 0  IMAD       32-bit multiply-add, a = a m + c        (1 op per chain step)
//   kind 1  IMAD.WIDE  32 x 32 -> 64-bit multiply-add          (1 op)
//   kind 2  mul.hi.u64 high half of a 64 x 64-bit product       (1 op)
//   kind 3  Shoup butterfly, unreduced form (primes below 2^58): T = a w - floor(a w' / 2^64) q,
//           (X, Y) -> (X + T, X + 2q - T); exactly the butterfly of the fused
//           transforms for the 40-bit primes                    (1 op = 1 butterfly)
//   kind 4  Shoup butterfly, Harvey form (X reduced below 2q first)
//
// Each thread runs `iters` steps of 32 operations (kinds 3/4: one radix-16
// pass of 4 stages x 8 butterflies over 16 chained values) and writes one
// word to sink[thread], so nothing is dead code.
#include "../../include/fhe.h"
#include "launch.cuh"

namespace fhe {

namespace {

__global__ void k_peak_imad(uint32_t iters, uint32_t m, uint32_t c0, u64* sink)
{
    uint32_t a[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = threadIdx.x * 33u + (uint32_t)i;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 32; ++i) a[i] = a[i] * m + (c0 ^ (uint32_t)i);
    }
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) r ^= a[i];
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = r;
}

__global__ void k_peak_imad_wide(uint32_t iters, uint32_t m, uint32_t c0, u64* sink)
{
    u64 a[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = threadIdx.x * 33u + (uint32_t)i;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            u64 r;
            asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"((uint32_t)a[i]), "r"(m + c0), "l"(a[i]));
            a[i] = r;
        }
    }
    u64 r = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) r ^= a[i];
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = r;
}

__global__ void k_peak_mulhi64(uint32_t iters, u64 m, u64 c0, u64* sink)
{
    u64 a[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = (u64)threadIdx.x * 0x9E3779B97F4A7C15ull + (u64)i;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 32; ++i) a[i] = __umul64hi(a[i], m) ^ (c0 + (u64)i);
    }
    u64 r = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) r ^= a[i];
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = r;
}

template <bool RED>
__global__ void k_peak_butterfly(uint32_t iters, u64 q, ulonglong2 w0, ulonglong2 w1, ulonglong2 w2, ulonglong2 w3,
                                 u64* sink)
{
    const u64 q2 = 2 * q;
    const ulonglong2 w[4] = {w0, w1, w2, w3};
    u64 x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = ((u64)threadIdx.x * 16 + (u64)i) % q;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int h = 8 >> l;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i & h) continue;
                u64 X = x[i];
                if (RED) X = X >= q2 ? X - q2 : X;
                const u64 T = mul_shoup_lazy(x[i + h], w[l].x, w[l].y, q);
                x[i] = X + T;
                x[i + h] = X + q2 - T;
            }
        }
    }
    u64 r = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) r ^= x[i];
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = r;
}

}  // namespace

}  // namespace fhe

using namespace fhe;

extern "C" int fhe_peak_launch(uint32_t kind, uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t* d_sink,
                               void* stream)
{
    if (kind > 4) return fail(FHE_EINVAL, "unknown peak kind (0..4)");
    if (blocks == 0 || threads == 0 || threads > 1024 || threads % 32 != 0)
        return fail(FHE_EINVAL, "blocks >= 1 and threads a multiple of 32 up to 1024");
    if (!d_sink) return fail(FHE_EINVAL, "null sink");
    cudaStream_t st = (cudaStream_t)stream;
    u64* sink = (u64*)d_sink;
    // a 40-bit NTT prime of the CNN's chain and twiddle-like constants with their Shoup quotients
    const u64 q = 0x10000048001ull;
    auto tw = [&](u64 v) {
        v %= q;
        return make_ulonglong2(v, (u64)(((unsigned __int128)v << 64) / q));
    };
    const ulonglong2 a = tw(0x123456789ull), b = tw(0x2468ace0135ull), c = tw(0x0fedcba987ull), d = tw(0x55aa55aa55ull);
    switch (kind) {
    case 0: k_peak_imad<<<blocks, threads, 0, st>>>(iters, 0x9E3779B1u, 0x7F4A7C15u, sink); break;
    case 1: k_peak_imad_wide<<<blocks, threads, 0, st>>>(iters, 0x9E3779B1u, 0x7F4A7C15u, sink); break;
    case 2: k_peak_mulhi64<<<blocks, threads, 0, st>>>(iters, 0xBF58476D1CE4E5B9ull, 0x94D049BB133111EBull, sink); break;
    case 3: k_peak_butterfly<false><<<blocks, threads, 0, st>>>(iters, q, a, b, c, d, sink); break;
    default: k_peak_butterfly<true><<<blocks, threads, 0, st>>>(iters, q, a, b, c, d, sink); break;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FHE_OK : cuda_check(e, "peak launch");
}
