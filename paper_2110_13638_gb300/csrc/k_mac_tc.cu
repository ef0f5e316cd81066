// k_mac_tc.cu -- dense layer multiply-accumulate on the 5th-generation tensor
// cores (tcgen05 MMA, accumulators in tensor memory): exact modular products
// from bf16 limb GEMMs.
//
// Per residue r a dense layer is Y_r = W_r X_r mod q_r, a [rows x terms] by
// [terms x 2N] contraction.  For primes q < 2^41 every residue x (and weight
// w) is centred to |x| < 2^40 and written in balanced base 256:
//     x = sum_{a<4} x_a 256^a + x_4 2^32,  x_a in [-128, 127],  |x_4| <= 256,
// all exact in bf16.  Then sum_i w_i x_i = sum_s 2^{8s} C_s with the
// shift-class sums C_s = sum_{a+b=s} sum_i w_{b,i} x_{a,i}, s = 0..8.  Each
// limb product is an exact integer (|.| <= 2^16 with a top limb, <= 2^14
// otherwise) and at most five limb pairs share a class, so over a chunk of
// 32 terms |C_s| < 2^22: the tensor core's fp32 accumulators hold C_s
// exactly.  After every chunk the epilogue reads the nine class sums out of
// tensor memory, turns them into integers and adds them, shifted, into two
// 64-bit sums per output:
//     lo = sum_{s<=4} C_s 2^{8s},   hi = sum_{s>=5} C_s 2^{8(s-5)},
// so the dot product is lo + hi 2^40 and y = (lo + hi 2^40) mod q_r.
//
// Tile: 128 coefficients (MMA M, the tensor-memory lanes) x 48 output rows
// (MMA N); the nine class accumulators take 9 x 48 = 432 of the 512
// tensor-memory columns the block allocates.  Operands sit in shared memory
// K-major without swizzle: core matrices of 8 rows x 16 bytes (8 bf16 terms),
// adjacent along K 128 bytes apart, 8-row groups 512 bytes apart.  The input
// limbs are split by the block's threads from the u64 residues (coalesced
// along the coefficients); the weight limbs come pre-split and pre-laid-out
// from the host.  One thread issues the 50 MMAs of a chunk and commits them
// to an mbarrier; every wait on it is bounded and a wait that gives up sets
// g_mac_tc_fault, skips the rest of the block's work and frees its tensor
// memory.
#include "../../include/fhe.h"
#include "launch.cuh"

namespace fhe {

namespace {
constexpr int kTcM = 128;                      // coefficients per tile
constexpr int kTcN = kMacTcRows;               // output rows per tile (48)
constexpr int kTcK = kMacTcChunk;              // terms per chunk (32)
constexpr int kTcLimbs = 5;
constexpr int kTcThreads = 256;
constexpr uint32_t kTmemCols = 512;
constexpr int kALimb = kTcM * kTcK * 2;        // bytes of one input limb plane (8 KB)
constexpr int kBLimb = kTcN * kTcK * 2;        // bytes of one weight limb plane (3 KB)
constexpr int kOffB = kTcLimbs * kALimb;
constexpr int kOffBar = kOffB + kTcLimbs * kBLimb;
constexpr int kWChunkU4 = kTcLimbs * kBLimb / 16;   // uint4 per (residue, tile, chunk) of weights
// more than half of the SM's shared memory: one block per SM, so the
// tensor-memory allocation never waits on a neighbouring block
constexpr int kTcSmem = 120 * 1024;
constexpr uint32_t kSpinLimit = 1u << 22;      // polls of ~64 ns: well under a second
// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N, M
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);
static_assert(kOffBar + 16 <= kTcSmem, "shared memory layout");
static_assert(9 * kTcN <= (int)kTmemCols, "tensor memory columns");
}  // namespace

__device__ unsigned int g_mac_tc_fault;

struct MacTcArgs {
    const u64* X;
    const uint32_t* col;
    const uint4* Wl;
    const uint32_t* rows;
    u64* Y;
    const PrimeC* pc;
    uint32_t K, n_tiles, n_chunks;
    uint32_t lbo, sbo; // descriptor byte offsets along K and along M/N
    int L, N;
    uint8_t zkr[64];   // grid z -> component-residue row k L + r
    uint8_t zri[64];   // grid z -> index of r among the tensor-core residues
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: start, leading (K) and stride
// (M/N) byte offsets in 16-byte units, fixed field 0b001 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 16) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

// bf16 bits of the five balanced base-256 limbs of a centred residue |xc| < 2^40:
// u = xc + 0x80808080 puts 128 on each low digit, so limb a < 4 is byte a of u
// minus 128 and the top limb is u >> 32 (arithmetic).  The float of a small
// integer is formed exactly through the 1.5 2^23 magic constant; its upper
// half is the bf16 (at most 9 significant bits).
__device__ __forceinline__ void limbs_f32(i64 xc, float (&f)[5])
{
    const i64 u = xc + 0x80808080ll;
    const uint32_t lo = (uint32_t)u;
    const int32_t top = (int32_t)(u >> 32);
    f[0] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7650)) - 12583040.0f;
    f[1] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7651)) - 12583040.0f;
    f[2] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7652)) - 12583040.0f;
    f[3] = __uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7653)) - 12583040.0f;
    f[4] = __int_as_float(0x4B400000 + top) - 12582912.0f;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mac_tc_kernel(const MacTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint32_t* tbase_s = reinterpret_cast<uint32_t*>(sm + kOffBar + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t t = blockIdx.x;
    const int j0 = blockIdx.y * kTcM;
    const int kr = a.zkr[blockIdx.z], ri = a.zri[blockIdx.z];
    const int r = kr % a.L;
    const PrimeC P = a.pc[r];
    const int N = a.N;
    const size_t ct_stride = (size_t)2 * a.L * N;
    const uint32_t bar_a = smem_u32(bar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tbase_s)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tbase_s;

    // producer role: coefficient m, k-groups kh and kh + 2 of each chunk
    const int m = tid & (kTcM - 1), kh = tid >> 7;
    const u64* Xm = a.X + (size_t)kr * N + j0 + m;
    u64 xr[16];
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t term = (uint32_t)((kh + 2 * g) * 8 + e);
            xr[g * 8 + e] = term < a.K ? Xm[(size_t)__ldg(&a.col[term]) * ct_stride] : 0ull;
        }

    // epilogue role: lanes 32 (warp % 4) .. +31, outputs 24 (warp / 4) .. +23
    const int q4 = warp & 3, h = warp >> 2;
    const uint32_t trow = tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(h * 24);
    i64 lo[24], hi[24];
#pragma unroll
    for (int o = 0; o < 24; ++o) lo[o] = hi[o] = 0;

    bool failed = false;
    for (uint32_t c = 0; c < a.n_chunks; ++c) {
        // stage the chunk: input limbs (split here) and weight limbs (copied)
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            uint32_t w[kTcLimbs][4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                float f0[5], f1[5];
                const u64 x0 = xr[g * 8 + 2 * e2], x1 = xr[g * 8 + 2 * e2 + 1];
                limbs_f32(x0 > P.half ? (i64)(x0 - P.q) : (i64)x0, f0);
                limbs_f32(x1 > P.half ? (i64)(x1 - P.q) : (i64)x1, f1);
#pragma unroll
                for (int l = 0; l < kTcLimbs; ++l)
                    w[l][e2] = __byte_perm(__float_as_uint(f0[l]), __float_as_uint(f1[l]), 0x7632);
            }
            const int kg = kh + 2 * g;
            const int off = ((m >> 3) * (kTcK / 8) + kg) * 128 + (m & 7) * 16;
#pragma unroll
            for (int l = 0; l < kTcLimbs; ++l)
                *reinterpret_cast<uint4*>(sm + l * kALimb + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
        }
        {
            const uint4* wsrc = a.Wl + ((size_t)(ri * a.n_tiles + t) * a.n_chunks + c) * kWChunkU4;
            uint4* wdst = reinterpret_cast<uint4*>(sm + kOffB);
            for (int i = tid; i < kWChunkU4; i += kTcThreads) wdst[i] = __ldg(&wsrc[i]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();

        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sm), b0 = smem_u32(sm + kOffB);
            uint32_t seen = 0;
#pragma unroll
            for (int ks = 0; ks < kTcK / 16; ++ks)
#pragma unroll
                for (int ai = 0; ai < kTcLimbs; ++ai)
#pragma unroll
                    for (int bi = 0; bi < kTcLimbs; ++bi) {
                        const int s = ai + bi;
                        const uint64_t da = smem_desc(a0 + ai * kALimb + ks * 256, a.lbo, a.sbo);
                        const uint64_t db = smem_desc(b0 + bi * kBLimb + ks * 256, a.lbo, a.sbo);
                        mma_bf16(tbase + (uint32_t)(s * kTcN), da, db, (seen >> s) & 1u);
                        seen |= 1u << s;
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                         : "memory");
        }

        // prefetch the next chunk's inputs while the tensor core works
        if (c + 1 < a.n_chunks) {
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t term = (c + 1) * kTcK + (uint32_t)((kh + 2 * g) * 8 + e);
                    xr[g * 8 + e] = term < a.K ? Xm[(size_t)__ldg(&a.col[term]) * ct_stride] : 0ull;
                }
        }

        const bool ok = mbar_wait(bar_a, c & 1u);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(&g_mac_tc_fault, 1u);
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            uint32_t v[3][8];
#pragma unroll
            for (int p = 0; p < 3; ++p) tmem_ld8(trow + (uint32_t)(s * kTcN + 8 * p), v[p]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int o = 0; o < 24; ++o) {
                // exact: |C_s| < 2^22, so C_s + 1.5 2^23 has unit spacing
                const int32_t cs =
                    (int32_t)(__float_as_uint(__uint_as_float(v[o >> 3][o & 7]) + 12582912.0f) - 0x4B400000u);
                if (s <= 4)
                    lo[o] += (i64)cs << (8 * s);
                else
                    hi[o] += (i64)cs << (8 * (s - 5));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }

    if (!failed) {
        const u64 p40 = reduce64(1ull << 40, P);
        const size_t off = (size_t)kr * N + j0 + 32 * q4 + lane;
#pragma unroll
        for (int o = 0; o < 24; ++o) {
            const uint32_t row = __ldg(&a.rows[t * kTcN + h * 24 + o]);
            if (row != 0xFFFFFFFFu)
                a.Y[(size_t)row * ct_stride + off] =
                    add_mod(from_signed(lo[o], P), mul_mod(from_signed(hi[o], P), p40, P), P.q);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

int k_linear_mac_tc(const fhe_ctx* c, const u64* X, const uint32_t* col, uint32_t K, const uint16_t* Wl,
                    const uint32_t* rows, uint32_t n_tiles, uint64_t tc_mask, uint32_t L, u64* Y, cudaStream_t st)
{
    if (n_tiles == 0 || K == 0 || tc_mask == 0) return 0;
    const int N = (int)c->N;
    if (N % kTcM != 0 || 2 * L > 64) return fail(FHE_EINVAL, "tensor-core MAC: ring or level out of range");
    MacTcArgs a{};
    a.X = X;
    a.col = col;
    a.Wl = reinterpret_cast<const uint4*>(Wl);
    a.rows = rows;
    a.Y = Y;
    a.pc = c->d_pc;
    a.K = K;
    a.n_tiles = n_tiles;
    a.n_chunks = (K + kTcK - 1) / kTcK;
    a.L = (int)L;
    a.N = N;
    a.lbo = 128;                 // core matrices adjacent along K
    a.sbo = (kTcK / 8) * 128;    // 8-row groups
    int nz = 0;
    for (uint32_t kr = 0; kr < 2 * L; ++kr) {
        const uint32_t r = kr % L;
        if ((tc_mask >> r) & 1u) {
            a.zkr[nz] = (uint8_t)kr;
            a.zri[nz] = (uint8_t)__builtin_popcountll(tc_mask & ((1ull << r) - 1));
            ++nz;
        }
    }
    ensure_smem((const void*)k_mac_tc_kernel, kTcSmem);
    dim3 grid(n_tiles, N / kTcM, nz);
    LaunchScope ls(c, "mac_tc", st);
    k_mac_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(a);
    return 0;
}

uint32_t mac_tc_fault_take()
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_mac_tc_fault, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
    if (v) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_mac_tc_fault, &z, sizeof(z));
    }
    return v;
}

}  // namespace fhe
