// k_persist.cu -- ct-mult + relinearise + rescale for ciphertexts at uneven
// levels in ONE persistent launch.
//
// One block per SM (512 threads, one residue polynomial in shared memory)
// takes units from a device work queue until it is empty.  A unit is one
// transform step of one ciphertext, in five phases:
//   1  digit inverse transforms, per (ct, digit u): INTT(a1_u b1_u)
//   2  ModUp + key inner products, per (ct, target t in q_0..q_{L-1}, P)
//   3  inverse transforms of P's residues, per (ct, component)
//   4  ModDown merged with the rescale: row L-1, per (ct, component)
//   5  the merged forward transforms, per (ct, component, i < L-1)
// (the steps of k_relin_rescale).  The tensor product is never stored: each
// step recomputes the components it needs from the factors a, b.  The queue
// is phase-major, so a unit only waits for units queued before it: its
// ciphertext's previous phase (a per-ciphertext completion counter, raised
// with release semantics by the block that finished a unit and read with
// acquire semantics).  Units queued earlier were taken by blocks that are
// running, so every wait ends; each is also bounded (about a second), after
// which the block raises the abort flag and the context's status word, and
// every block skips its remaining units.
#include "../../include/fhe.h"
#include "ops.cuh"

namespace fhe {

namespace {

constexpr int kPhases = 5;
constexpr int kPersistThreads = 512;
constexpr uint32_t kWaitPolls = 1u << 22;      // polls of >= 256 ns: about a second

struct PersistGroup {
    OpDigitsInvT<true> p1;
    OpModUpMacT<true> p2;
    OpAccPInv p3;
    OpKsRowInvT<true> p4;
    OpKsDivFwdT<true> p5;
    unsigned int* cnt;          // [n][4]: finished units of phases 1..4 per ciphertext
    int n, L;
};

struct PersistArgs {
    PersistGroup g[kMaxGroups];
    int ng;
    int start[kPhases][kMaxGroups + 1];     // per phase: unit prefix sums over the groups
    int phase0[kPhases + 1];                // queue index of each phase's first unit
    unsigned int* queue;                    // [0]: next unit, [1]: abort flag
    unsigned int* status;                   // the context's status word (host-mapped)
    uint32_t wait_polls;
    uint32_t stall;                         // test hook: phase 1 never reports its units
};

// units of phase ph for one ciphertext at level L, and the count its next
// phase waits for
__host__ __device__ __forceinline__ int phase_units(int ph, int L)
{
    switch (ph) {
    case 0: return L;
    case 1: return L + 1;
    case 2: return 2;
    case 3: return 2;
    default: return 2 * (L - 1);
    }
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// thread 0 only: true once *c >= need; false if the wait runs out or another
// block aborted
__device__ bool wait_count(const unsigned int* c, unsigned int need, const unsigned int* abort, uint32_t polls)
{
    for (uint32_t i = 0; i < polls; ++i) {
        if (ld_acquire(c) >= need) return true;
        if (*(const volatile unsigned int*)abort) return false;
        __nanosleep(256);
    }
    return false;
}

// each phase's transform in a function of its own, so that each gets the
// register allocation it has as a kernel of its own
template <bool INV, class Op>
__device__ __noinline__ void run_unit(const Op& op, NttTables T, int q, u64* sm)
{
    ntt_io_unit<INV, 4, kPersistThreads>(op, T, q, sm);
}

__global__ void __launch_bounds__(kPersistThreads, 1) k_persist_kernel(const __grid_constant__ PersistArgs A,
                                                                         NttTables T)
{
    extern __shared__ u64 sm[];
    __shared__ int s_unit, s_go;
    const int total = A.phase0[kPhases];
    unsigned int* abort = A.queue + 1;
    for (;;) {
        if (threadIdx.x == 0) s_unit = (int)atomicAdd(A.queue, 1u);
        __syncthreads();
        const int unit = s_unit;
        if (unit >= total) break;
        int ph = 0;
        while (unit >= A.phase0[ph + 1]) ++ph;
        const int w = unit - A.phase0[ph];
        int g = 0;
        while (g + 1 < A.ng && w >= A.start[ph][g + 1]) ++g;
        const int q = w - A.start[ph][g];
        const PersistGroup& G = A.g[g];
        const int ct = ph == 1 ? G.p2.ct_of(q) : q / phase_units(ph, G.L);
        if (threadIdx.x == 0) {
            bool go = true;
            if (ph > 0) {
                go = wait_count(G.cnt + (size_t)ct * 4 + (ph - 1), (unsigned int)phase_units(ph - 1, G.L), abort,
                                A.wait_polls);
                if (!go) {
                    atomicExch(abort, 1u);
                    if (A.status) *(volatile unsigned int*)A.status = 1u;
                }
            }
            if (*(volatile unsigned int*)abort) go = false;
            __threadfence();        // the acquire above orders this block's reads after the producers' writes
            s_go = go;
        }
        __syncthreads();
        if (!s_go) continue;
        switch (ph) {
        case 0: run_unit<true>(G.p1, T, q, sm); break;
        case 1: run_unit<false>(G.p2, T, q, sm); break;
        case 2: run_unit<true>(G.p3, T, q, sm); break;
        case 3: run_unit<true>(G.p4, T, q, sm); break;
        default: run_unit<false>(G.p5, T, q, sm); break;
        }
        // the unit ends with a barrier after every thread's stores: publish it
        if (ph < 4 && threadIdx.x == 0 && !(A.stall && ph == 0)) {
            __threadfence();
            atomicAdd(G.cnt + (size_t)ct * 4 + ph, 1u);
        }
    }
}

int g_sms[64] = {0};

}  // namespace

size_t persist_scratch_bytes(const fhe_ctx* c, const LevelBatch* g, int ng)
{
    const size_t N = c->N;
    size_t words = 2;                       // queue and abort flag
    for (int k = 0; k < ng; ++k) words += (size_t)g[k].n * 4;
    size_t s = arena_need({words * 4});
    for (int k = 0; k < ng; ++k) {
        const size_t n = g[k].n, L = g[k].L;
        s += arena_need({n * L * N * 8, n * 2 * (L + 1) * N * 8, n * 2 * N * 8, n * 2 * N * 8});
    }
    return s;
}

int k_mul_relin_rescale_persistent(const fhe_ctx* c, const LevelBatch* g, int ng, void* scratch, cudaStream_t st)
{
    const size_t N = c->N;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = persist_scratch_bytes(c, g, ng);
    size_t words = 2;
    for (int k = 0; k < ng; ++k) words += (size_t)g[k].n * 4;
    unsigned int* ctl = (unsigned int*)ar.take(words * 4);
    PersistArgs A{};
    A.ng = ng;
    A.queue = ctl;
    A.status = c->d_status;
    A.wait_polls = kWaitPolls;
    if (c->inject == FHE_INJECT_PERSIST_STALL) {        // test hook, consumed by this launch
        c->inject = 0;
        A.stall = 1;
        A.wait_polls = 1024;
    }
    unsigned int* cnt = ctl + 2;
    const KsExtra none{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    for (int ph = 0; ph < kPhases; ++ph) A.start[ph][0] = 0;
    for (int k = 0; k < ng; ++k) {
        const int n = (int)g[k].n, L = (int)g[k].L;
        u64* D = (u64*)ar.take((size_t)n * L * N * 8);
        u64* acc = (u64*)ar.take((size_t)n * 2 * (L + 1) * N * 8);
        u64* Vp = (u64*)ar.take((size_t)n * 2 * N * 8);
        u64* V = (u64*)ar.take((size_t)n * 2 * N * 8);
        const D3Src<true> src(g[k].a, g[k].b);
        PersistGroup& G = A.g[k];
        G.n = n;
        G.L = L;
        G.cnt = cnt;
        cnt += (size_t)n * 4;
        G.p1 = OpDigitsInvT<true>{src, D, n, L, (int)N};
        G.p2 = OpModUpMacT<true>{src, D, c->d_ksk, acc, n, L, (int)N, (int)c->L_top, modup_red_mask(c, (uint32_t)L),
                               modup_lazy_mask(c, (uint32_t)L)};
        G.p3 = OpAccPInv{acc, Vp, n, L, (int)N, (int)c->L_top};
        const OpKsRowInv r = make_ks_row_inv(c, nullptr, acc, Vp, V, n, L, none);
        OpKsRowInvT<true>& p4 = G.p4;
        p4.d3 = src;
        p4.acc = r.acc;
        p4.Vp = r.Vp;
        p4.V = r.V;
        p4.n = n;
        p4.L = L;
        p4.N = (int)N;
        p4.ex = none;
        p4.p = r.p;
        p4.p_half = r.p_half;
        p4.pmod = r.pmod;
        p4.pinv = r.pinv;
        p4.pinvs = r.pinvs;
        const OpKsDivFwd f = make_ks_div_fwd(c, nullptr, acc, Vp, V, g[k].out, n, L, none, nullptr, 0);
        OpKsDivFwdT<true>& p5 = G.p5;
        p5.d3 = src;
        p5.acc = f.acc;
        p5.Vp = f.Vp;
        p5.V = f.V;
        p5.out = f.out;
        p5.addc = nullptr;
        p5.n = n;
        p5.L = L;
        p5.N = (int)N;
        p5.addc_stride = 0;
        p5.ex = none;
        p5.dp = f.dp;
        p5.dq = f.dq;
        p5.small_mask = f.small_mask;
        for (int ph = 0; ph < kPhases; ++ph) A.start[ph][k + 1] = A.start[ph][k] + n * phase_units(ph, L);
    }
    A.phase0[0] = 0;
    for (int ph = 0; ph < kPhases; ++ph) A.phase0[ph + 1] = A.phase0[ph] + A.start[ph][ng];
    cudaError_t e = cudaMemsetAsync(ctl, 0, words * 4, st);
    if (e != cudaSuccess) return cuda_check(e, "persistent queue reset");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return fail(FHE_EUNSUPPORTED, "device ordinal beyond 63");
    if (!g_sms[dev]) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_check(e, "SM count");
        g_sms[dev] = sms;
    }
    const size_t smem = (size_t)ntt_smem_words((int)N) * sizeof(u64);
    ensure_smem((const void*)k_persist_kernel, smem);
    LaunchScope ls(c, "persistent", st);
    k_persist_kernel<<<g_sms[dev], kPersistThreads, smem, st>>>(A, c->tabs());
    return FHE_OK;
}

}  // namespace fhe
