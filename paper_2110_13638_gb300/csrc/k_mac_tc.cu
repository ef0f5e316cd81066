// k_mac_tc.cu -- dense layer multiply-accumulate on the 5th-generation tensor
// cores (tcgen05 MMA, accumulators in tensor memory): exact modular products
// from bf16 limb GEMMs.
//
// Per residue r a dense layer is Y_r = W_r X_r mod q_r, a [rows x terms] by
// [terms x 2N] contraction.  Every residue x (and weight w) is centred,
// |x| < q/2, and written in balanced base 256 with n limbs:
//     x = sum_{a<n-1} x_a 256^a + x_{n-1} 256^{n-1},  x_a in [-128, 127],
// the top limb taking what is left.  Five limbs cover primes below 2^41
// (|top| <= 256), eight limbs primes below 2^61 (|top| <= 16); all limbs are
// exact in bf16.  Then sum_i w_i x_i = sum_s 2^{8s} C_s with the shift-class
// sums C_s = sum_{a+b=s} sum_i w_{b,i} x_{a,i}, s = 0..2n-2.  Each limb
// product is an exact integer (|.| <= 2^16 with a top limb, <= 2^14
// otherwise) and no class holds more than 2^16 + 3 2^14 per term, so over a
// chunk of 32 terms |C_s| < 2^22: the tensor core's fp32 accumulators hold
// C_s exactly.  After every chunk the epilogue reads the class sums out of
// tensor memory, turns them into integers and adds them, shifted, into one
// 64-bit sum per five classes:
//     A_i = sum_{p<5} C_{5i+p} 2^{8p},   dot product = sum_i A_i 2^{40 i},
// and at the end y = sum_i (A_i mod q) (2^{40 i} mod q) mod q.
//
// Tile: 128 coefficients (MMA M, the tensor-memory lanes) x NT output rows
// (MMA N): NT = 48 with five limbs (9 classes x 48 = 432 of the 512
// tensor-memory columns the block allocates), NT = 32 with eight (15 x 32 =
// 480).  Operands sit in shared memory K-major without swizzle: core matrices
// of 8 rows x 16 bytes (8 bf16 terms), adjacent along K 128 bytes apart, 8-row
// groups 512 bytes apart.  The block's 16 warps split the input limbs from
// the u64 residues (coalesced along the coefficients) into one of two staging
// buffers while the tensor core works on the other, and read the class sums
// back (warp w: lanes 32 (w % 4) .. +31, a quarter of the tile's rows); the
// weight limbs come pre-split and pre-laid-out from the host.  Up to 8192
// terms keep the 64-bit sums exact.  One thread issues the MMAs of a
// chunk and commits them to an mbarrier; every wait on it is bounded.  A wait
// that gives up makes the block skip the rest of its work: it waits once more
// (bounded) for the products already committed, so that tensor memory is not
// released under a running MMA, then sets g_mac_tc_fault and the context's
// status word (the host reports FHE_ETIMEOUT) and frees its tensor memory.
#include "../../include/fhe.h"
#include "launch.cuh"

namespace fhe {

namespace {
constexpr int kTcM = 128;                      // coefficients per tile
constexpr int kTcK = kMacTcChunk;              // terms per chunk (32)
constexpr int kTcThreads = 512;             // 16 warps: 4 lane quarters x 4 column quarters
constexpr uint32_t kTmemCols = 512;
constexpr int kALimb = kTcM * kTcK * 2;        // bytes of one input limb plane (8 KB)
constexpr uint32_t kSpinLimit = 1u << 22;      // polls of ~64 ns: well under a second

// shapes of the two limb counts
template <int LIMBS>
struct TcShape {
    static constexpr int NT = LIMBS == 5 ? kMacTcRows : kMacTcRows8;   // output rows per tile
    static constexpr int kClasses = 2 * LIMBS - 1;
    static constexpr int kAcc = (kClasses + 4) / 5;                    // 64-bit sums per output
    static constexpr int kBLimb = NT * kTcK * 2;                       // bytes of one weight limb plane
    static constexpr int kOffB = LIMBS * kALimb;                       // weights after the input limbs
    static constexpr int kStage = ((kOffB + LIMBS * kBLimb) + 1023) / 1024 * 1024;
    static constexpr int kOffBar = 2 * kStage;                         // two staging buffers
    // more than half of the SM's shared memory: one block per SM, so the
    // tensor-memory allocation never waits on a neighbouring block
    static constexpr int kSmem = kOffBar + 1024 > 120 * 1024 ? kOffBar + 1024 : 120 * 1024;
    static constexpr int kWChunkU4 = LIMBS * kBLimb / 16;              // uint4 per (residue, tile, chunk)
    // instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, N >> 3, M >> 4
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                       ((uint32_t)(kTcM >> 4) << 24);
    static_assert(kClasses * NT <= (int)kTmemCols, "tensor memory columns");
    static_assert(kSmem <= 227 * 1024, "shared memory");
    static_assert(NT % 16 == 0 && (NT / 4) % 4 == 0, "MMA N and epilogue split");
};
}  // namespace

__device__ unsigned int g_mac_tc_fault;

struct MacTcArgs {
    const u64* X;
    const uint32_t* col;
    const uint4* Wl;
    const uint32_t* rows;
    u64* Y;
    const PrimeC* pc;
    unsigned int* status;  // the context's status word (host-mapped), set when a wait gives up
    uint32_t spin_limit;   // polls per mbarrier wait
    uint32_t withhold;     // test hook: issue no MMA, so every wait runs out with nothing in flight
    uint32_t K, n_tiles, n_chunks;
    int L, N;
    uint8_t zkr[64];   // grid z -> component-residue row k L + r
    uint8_t zri[64];   // grid z -> index of r among this launch's residues
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: start address, leading (K:
// 128 bytes between core matrices) and stride (M/N: 512 bytes between 8-row
// groups) offsets in 16-byte units, fixed field 0b001 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    constexpr uint32_t lbo = 128, sbo = (kTcK / 8) * 128;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
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

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* v)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr)
                 : "memory");
}

// wait for this thread's tensor-memory loads; the loaded registers pass
// through the statement, so no use of them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait4(uint32_t* v)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3])
                 :
                 : "memory");
}

// the float of (byte of word) - 128, exactly, through the 1.5 2^23 magic constant
__device__ __forceinline__ float byte_less_128(uint32_t word, uint32_t sel)
{
    return __uint_as_float(__byte_perm(word, 0x4B400000u, sel)) - 12583040.0f;
}

// balanced base-256 limbs of a centred residue: u = xc + 128 (256^0 + ... +
// 256^{n-2}) puts 128 on each low digit, so limb a < n - 1 is byte a of u
// minus 128 and the top limb is u >> 8(n-1) (arithmetic).  Each float has at
// most 9 significant bits, so its upper half is the exact bf16.
template <int LIMBS>
__device__ __forceinline__ void limbs_f32(i64 xc, float (&f)[LIMBS])
{
    if constexpr (LIMBS == 5) {
        const i64 u = xc + 0x80808080ll;
        const uint32_t lo = (uint32_t)u;
        f[0] = byte_less_128(lo, 0x7650);
        f[1] = byte_less_128(lo, 0x7651);
        f[2] = byte_less_128(lo, 0x7652);
        f[3] = byte_less_128(lo, 0x7653);
        f[4] = __int_as_float(0x4B400000 + (int32_t)(u >> 32)) - 12582912.0f;
    } else {
        const i64 u = xc + 0x80808080808080ll;
        const uint32_t lo = (uint32_t)u, mid = (uint32_t)((u64)u >> 32);
        f[0] = byte_less_128(lo, 0x7650);
        f[1] = byte_less_128(lo, 0x7651);
        f[2] = byte_less_128(lo, 0x7652);
        f[3] = byte_less_128(lo, 0x7653);
        f[4] = byte_less_128(mid, 0x7650);
        f[5] = byte_less_128(mid, 0x7651);
        f[6] = byte_less_128(mid, 0x7652);
        f[7] = __int_as_float(0x4B400000 + (int32_t)(u >> 56)) - 12582912.0f;
    }
}

template <int LIMBS>
__global__ void __launch_bounds__(kTcThreads, 1) k_mac_tc_kernel(const MacTcArgs a)
{
    using S = TcShape<LIMBS>;
    constexpr int NT = S::NT, NQ = NT / 4;     // outputs per epilogue thread
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + S::kOffBar);
    uint32_t* tbase_s = reinterpret_cast<uint32_t*>(sm + S::kOffBar + 8);
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

    // producer role: coefficient m, k-group kg (8 terms) of each chunk;
    // xr holds the inputs of the next chunk to stage
    const int m = tid & (kTcM - 1), kg = tid >> 7;
    const u64* Xm = a.X + (size_t)kr * N + j0 + m;
    u64 xr[8];
    auto fetch = [&](uint32_t c) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t term = c * kTcK + (uint32_t)(kg * 8 + e);
            xr[e] = term < a.K ? Xm[(size_t)__ldg(&a.col[term]) * ct_stride] : 0ull;
        }
    };
    // input limbs of xr and the chunk's weight limbs into staging buffer sb
    auto stage = [&](uint32_t c, unsigned char* sb) {
        {
            uint32_t w[LIMBS][4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                float f0[LIMBS], f1[LIMBS];
                const u64 x0 = xr[2 * e2], x1 = xr[2 * e2 + 1];
                limbs_f32<LIMBS>(x0 > P.half ? (i64)(x0 - P.q) : (i64)x0, f0);
                limbs_f32<LIMBS>(x1 > P.half ? (i64)(x1 - P.q) : (i64)x1, f1);
#pragma unroll
                for (int l = 0; l < LIMBS; ++l)
                    w[l][e2] = __byte_perm(__float_as_uint(f0[l]), __float_as_uint(f1[l]), 0x7632);
            }
            const int off = ((m >> 3) * (kTcK / 8) + kg) * 128 + (m & 7) * 16;
#pragma unroll
            for (int l = 0; l < LIMBS; ++l)
                *reinterpret_cast<uint4*>(sb + l * kALimb + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
        }
        const uint4* wsrc = a.Wl + ((size_t)(ri * a.n_tiles + t) * a.n_chunks + c) * S::kWChunkU4;
        uint4* wdst = reinterpret_cast<uint4*>(sb + S::kOffB);
        for (int i = tid; i < S::kWChunkU4; i += kTcThreads) wdst[i] = __ldg(&wsrc[i]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };

    // epilogue role: lanes 32 (warp % 4) .. +31, outputs NQ (warp / 4) .. +NQ-1
    const int q4 = warp & 3, h = warp >> 2;
    const uint32_t trow = tbase + ((uint32_t)(32 * q4) << 16) + (uint32_t)(h * NQ);
    i64 acc[S::kAcc][NQ];
#pragma unroll
    for (int i = 0; i < S::kAcc; ++i)
#pragma unroll
        for (int o = 0; o < NQ; ++o) acc[i][o] = 0;

    fetch(0);
    stage(0, sm);
    if (a.n_chunks > 1) fetch(1);
    __syncthreads();

    bool failed = false;
    for (uint32_t c = 0; c < a.n_chunks; ++c) {
        if (tid == 0 && !a.withhold) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sb = smem_u32(sm + (c & 1u) * S::kStage);
            uint32_t seen = 0;
#pragma unroll
            for (int ks = 0; ks < kTcK / 16; ++ks)
#pragma unroll
                for (int ai = 0; ai < LIMBS; ++ai)
#pragma unroll
                    for (int bi = 0; bi < LIMBS; ++bi) {
                        const int s = ai + bi;
                        const uint64_t da = smem_desc(sb + ai * kALimb + ks * 256);
                        const uint64_t db = smem_desc(sb + S::kOffB + bi * S::kBLimb + ks * 256);
                        mma_bf16(tbase + (uint32_t)(s * NT), da, db, S::kIdesc, (seen >> s) & 1u);
                        seen |= 1u << s;
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                         : "memory");
        }
        // while the tensor core works: stage the next chunk into the other
        // buffer (its last reader, chunk c - 1, has completed) and fetch the one after
        if (c + 1 < a.n_chunks) {
            stage(c + 1, sm + ((c + 1) & 1u) * S::kStage);
            if (c + 2 < a.n_chunks) fetch(c + 2);
        }

        const bool ok = mbar_wait(bar_a, c & 1u, a.spin_limit);
        if (__syncthreads_or(!ok)) {
            // products committed to this phase may still be running: give them
            // one more bounded wait before tensor memory is released below
            mbar_wait(bar_a, c & 1u, a.spin_limit);
            if (tid == 0) {
                atomicOr(&g_mac_tc_fault, 1u);
                if (a.status) *(volatile unsigned int*)a.status = 1u;
            }
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // class sums -> integers (exact: |C_s| < 2^22, so C_s + 1.5 2^23 has
        // unit spacing and its bits minus 0x4B400000 are C_s); within each
        // 64-bit sum the classes are paired in 32 bits first
        // (|C_s + 256 C_{s+1}| < 2^31):  A_i += (C_5i + 256 C_5i+1)
        //   + (C_5i+2 + 256 C_5i+3) 2^16 + C_5i+4 2^32
#pragma unroll
        for (int i = 0; i < S::kAcc; ++i)
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const int s0 = 5 * i + 2 * part;
                if (s0 >= S::kClasses) continue;
                const bool pair = part < 2 && s0 + 1 < S::kClasses;
                uint32_t v0[NQ], v1[NQ];
#pragma unroll
                for (int p = 0; p < NQ / 4; ++p) tmem_ld4(trow + (uint32_t)(s0 * NT + 4 * p), v0 + 4 * p);
                if (pair) {
#pragma unroll
                    for (int p = 0; p < NQ / 4; ++p) tmem_ld4(trow + (uint32_t)((s0 + 1) * NT + 4 * p), v1 + 4 * p);
                }
#pragma unroll
                for (int p = 0; p < NQ / 4; ++p) tmem_wait4(v0 + 4 * p);
                if (pair) {
#pragma unroll
                    for (int p = 0; p < NQ / 4; ++p) tmem_wait4(v1 + 4 * p);
                }
#pragma unroll
                for (int o = 0; o < NQ; ++o) {
                    const uint32_t b0 = __float_as_uint(__uint_as_float(v0[o]) + 12582912.0f);
                    if (!pair) {
                        acc[i][o] += (i64)(int32_t)(b0 - 0x4B400000u) << (16 * part);
                        continue;
                    }
                    const uint32_t b1 = __float_as_uint(__uint_as_float(v1[o]) + 12582912.0f);
                    const int32_t pr = (int32_t)(b0 + (b1 << 8) - 0x4B400000u * 257u);
                    acc[i][o] += (i64)pr << (16 * part);
                }
            }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }

    if (!failed) {
        u64 pw[S::kAcc];                      // 2^{40 i} mod q
        pw[0] = 1;
#pragma unroll
        for (int i = 1; i < S::kAcc; ++i) pw[i] = mul_mod(pw[i - 1], reduce64(1ull << 40, P), P);
        const size_t off = (size_t)kr * N + j0 + 32 * q4 + lane;
#pragma unroll
        for (int o = 0; o < NQ; ++o) {
            const uint32_t row = __ldg(&a.rows[t * NT + h * NQ + o]);
            if (row == 0xFFFFFFFFu) continue;
            u64 y = from_signed(acc[0][o], P);
#pragma unroll
            for (int i = 1; i < S::kAcc; ++i) y = add_mod(y, mul_mod(from_signed(acc[i][o], P), pw[i], P), P.q);
            a.Y[(size_t)row * ct_stride + off] = y;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

template <int LIMBS>
static int launch_mac_tc(const fhe_ctx* c, const MacTcArgs& a, int nz, cudaStream_t st)
{
    using S = TcShape<LIMBS>;
    auto fn = k_mac_tc_kernel<LIMBS>;
    ensure_smem((const void*)fn, S::kSmem);
    dim3 grid(a.n_tiles, a.N / kTcM, nz);
    LaunchScope ls(c, "mac_tc", st);
    fn<<<grid, kTcThreads, S::kSmem, st>>>(a);
    return FHE_OK;
}

int k_linear_mac_tc(const fhe_ctx* c, int limbs, const u64* X, const uint32_t* col, uint32_t K, const uint16_t* Wl,
                    const uint32_t* rows, uint32_t n_tiles, uint64_t mask, uint32_t L, u64* Y, cudaStream_t st)
{
    if (n_tiles == 0 || K == 0 || mask == 0) return FHE_OK;
    const int N = (int)c->N;
    if (N % kTcM != 0 || 2 * L > 64 || (limbs != 5 && limbs != 8) || K > 8192)
        return fail(FHE_EINVAL, "tensor-core MAC: ring, level, limb count or term count out of range");
    MacTcArgs a{};
    a.X = X;
    a.col = col;
    a.Wl = reinterpret_cast<const uint4*>(Wl);
    a.rows = rows;
    a.Y = Y;
    a.pc = c->d_pc;
    a.status = c->d_status;
    a.spin_limit = kSpinLimit;
    if (c->inject == FHE_INJECT_MAC_TC_WITHHOLD) {   // test hook, consumed by this launch
        c->inject = 0;
        a.withhold = 1;
        a.spin_limit = 1024;
    }
    a.K = K;
    a.n_tiles = n_tiles;
    a.n_chunks = (K + kTcK - 1) / kTcK;
    a.L = (int)L;
    a.N = N;
    int nz = 0;
    for (uint32_t kr = 0; kr < 2 * L; ++kr) {
        const uint32_t r = kr % L;
        if ((mask >> r) & 1u) {
            a.zkr[nz] = (uint8_t)kr;
            a.zri[nz] = (uint8_t)__builtin_popcountll(mask & ((1ull << r) - 1));
            ++nz;
        }
    }
    return limbs == 5 ? launch_mac_tc<5>(c, a, nz, st) : launch_mac_tc<8>(c, a, nz, st);
}

uint32_t mac_tc_fault_take()
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_mac_tc_fault, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
    if (v) {
        const unsigned int z = 0;
        if (cudaMemcpyToSymbol(g_mac_tc_fault, &z, sizeof(z)) != cudaSuccess) return 0xFFFFFFFFu;
    }
    return v;
}

}  // namespace fhe
