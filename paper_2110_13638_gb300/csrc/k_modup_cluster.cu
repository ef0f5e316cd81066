// k_modup_cluster.cu -- the key-switching digit transforms and key inner
// products (ModUp step) on a cluster of four blocks per (ciphertext, target
// prime), each block owning one quarter of the coefficients.
//
// Per digit u the forward transform of D_u (mod q_t) starts with two stages
// (distances N/2 and N/4) whose radix-4 groups {j, j + N/4, j + N/2, j + 3N/4}
// span the four quarters: each block computes a quarter of those groups from
// global memory and writes each output to the shared memory of the block
// that owns its quarter (distributed shared memory, plain st.shared::cluster
// stores), then the cluster synchronises.  The remaining log2 N - 2 stages
// are independent N/4-point problems on the full transform's twiddles (local
// stage s is global stage s + 2, local group g of quarter r is global group
// g + r 2^s), run in each block's shared memory.  The key products of the
// last pass go into two accumulators that stay in the block's shared memory
// for all L digits (no global read-modify-write per digit), and are written
// out once at the end.  No stage's work is repeated, and each block holds
// N/4 transform words plus 2 N/4 accumulator words, so two blocks share an
// SM.
#include "ops.cuh"

namespace fhe {

namespace {

constexpr int kClusterCtas = 4;
constexpr int kCqThreads = 256;

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// store v at the shared-memory word `local` (a shared::cta address of this
// block's layout) of cluster block `rank`
__device__ __forceinline__ void st_cluster(const u64* local, uint32_t rank, u64 v)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(ra), "l"(v) : "memory");
}

struct NoFetchC {};

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kCqThreads, 2)
    k_modup_cluster(const OpModUpMac op, NttTables T)
{
    extern __shared__ u64 smc[];
    const int logN = T.logN;
    const int N = 1 << logN, logNq = logN - 2, Nq = N >> 2;
    const int W = ntt_smem_words(Nq);
    u64* sm = smc;                     // this quarter of the transform
    u64* acc_s = smc + W;              // [2][W]: this quarter of both accumulators
    const int tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t r = cluster_rank();
    const int jq = (int)r * Nq;        // first coefficient of this quarter
    const int L = op.L, Ltop = op.Ltop;
    const int p = blockIdx.x / kClusterCtas;          // (ct, target) unit of this cluster
    const int ct = p / (L + 1), t = p % (L + 1);
    const int tk = t == L ? Ltop : t;
    const PrimeC P = T.pc[tk];
    const u64 q = P.q, q2 = 2 * q;
    const bool lazy = (op.lazy_mask >> t) & 1u;
    const bool wide = q < kFwdNoRedBound;
    const ulonglong2* tw = T.tw_fwd + (size_t)tk * N;

    // key product of output word j (global index) added into acc_s[k][spad(jl)]
    auto accumulate = [&](int u, int jl, u64 v, ulonglong2 k0, ulonglong2 k1) {
        u64* a0 = acc_s + spad(jl);
        u64* a1 = acc_s + W + spad(jl);
        if (lazy) {
            const u64 p0 = mul_shoup_lazy(v, k0.x, k0.y, q), p1 = mul_shoup_lazy(v, k1.x, k1.y, q);
            *a0 = u == 0 ? p0 : *a0 + p0;
            *a1 = u == 0 ? p1 : *a1 + p1;
        } else {
            const u64 p0 = mul_shoup(v, k0.x, k0.y, q), p1 = mul_shoup(v, k1.x, k1.y, q);
            *a0 = u == 0 ? p0 : add_mod(*a0, p0, q);
            *a1 = u == 0 ? p1 : add_mod(*a1, p1, q);
        }
    };
    auto key0 = [&](int u, int jg) { return __ldg(&op.ksk[(((size_t)u * 2 + 0) * (Ltop + 1) + tk) * N + jg]); };
    auto key1 = [&](int u, int jg) { return __ldg(&op.ksk[(((size_t)u * 2 + 1) * (Ltop + 1) + tk) * N + jg]); };

    for (int u = 0; u < L; ++u) {
        if (u == t) {
            // direct: NTT(d2_t) is d2_t itself
            for (int jl = tid; jl < Nq; jl += nthr) {
                const int jg = jq + jl;
                const u64 v = op.d3.get(ct, 2, L, N, t, jg, P);
                accumulate(u, jl, v, key0(u, jg), key1(u, jg));
            }
            continue;
        }
        // every block has finished reading its transform words of the previous digit
        cluster_sync();
        // global stages 0 and 1: radix-4 groups j in this block's share of [0, N/4)
        {
            const ulonglong2 w1 = __ldg(&tw[1]), w2 = __ldg(&tw[2]), w3 = __ldg(&tw[3]);
            const u64* Du = op.D + ((size_t)ct * L + u) * N;
            const bool red = (op.red_mask >> u) & 1u;
            for (int jj = tid; jj < Nq / kClusterCtas; jj += nthr) {
                const int j = jq / kClusterCtas + jj;     // quarter r of the groups
                u64 x[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const u64 d = Du[j + m * Nq];
                    x[m] = red ? reduce64(d, P) : d;
                }
                auto bfly = [&](u64& X, u64& Y, const ulonglong2& w) {
                    u64 a = X;
                    if (!wide) a = a >= q2 ? a - q2 : a;
                    const u64 Tv = mul_shoup_lazy(Y, w.x, w.y, q);
                    X = a + Tv;
                    Y = a + q2 - Tv;
                };
                bfly(x[0], x[2], w1);
                bfly(x[1], x[3], w1);
                bfly(x[0], x[1], w2);
                bfly(x[2], x[3], w3);
#pragma unroll
                for (int m = 0; m < 4; ++m) st_cluster(sm + spad(j), (uint32_t)m, x[m]);
            }
        }
        // every quarter holds its N/4 words
        cluster_sync();
        // local stages 0 .. logNq-1 (global 2 .. logN-1) on this quarter
        int s = 0;
        while (s < logNq) {
            constexpr int LOGR = 4;
            const int k = (logNq - s) < LOGR ? (logNq - s) : LOGR;
            const bool last = s + k >= logNq;
            const int goff = (int)r << s;
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
            auto nofetch = [&](auto, int, int) { return NoFetch{}; };
            // the last pass: keys of the first PF words loaded before the
            // butterflies, the rest in batches of 4; products into acc_s
            constexpr int PF = 4, EB = 4;
            struct Keys {
                ulonglong2 k0[PF], k1[PF];
            };
            auto efetch = [&](auto Rc, int j0, int lsh) {
                constexpr int R = decltype(Rc)::value;
                Keys f;
#pragma unroll
                for (int i = 0; i < PF; ++i)
                    if (i < R) {
                        const int jg = jq + j0 + (i << lsh);
                        f.k0[i] = key0(u, jg);
                        f.k1[i] = key1(u, jg);
                    }
                return f;
            };
            auto pepi = [&](auto Rc, int j0, int lsh, u64* x, const Keys& f) {
                constexpr int R = decltype(Rc)::value;
                auto val = [&](int i) { return wide ? x[i] : fwd_final(x[i], q); };
#pragma unroll
                for (int i = 0; i < PF; ++i)
                    if (i < R) accumulate(u, j0 + (i << lsh), val(i), f.k0[i], f.k1[i]);
#pragma unroll
                for (int i0 = PF; i0 < R; i0 += EB) {
                    ulonglong2 k0[EB], k1[EB];
#pragma unroll
                    for (int i = 0; i < EB; ++i)
                        if (i0 + i < R) {
                            const int jg = jq + j0 + ((i0 + i) << lsh);
                            k0[i] = key0(u, jg);
                            k1[i] = key1(u, jg);
                        }
#pragma unroll
                    for (int i = 0; i < EB; ++i)
                        if (i0 + i < R) accumulate(u, j0 + ((i0 + i) << lsh), val(i0 + i), k0[i], k1[i]);
                }
            };
            auto run = [&](auto redc, auto& get, auto& put, auto& fetch) {
                pass_io_k<false, LOGR, decltype(redc)::value>(k, logNq, s, tw, q, q2, tid, nthr, get, put, fetch, 2,
                                                              goff);
            };
            auto run_rw = [&](auto& get, auto& put, auto& fetch) {
                if (wide) run(std::false_type{}, get, put, fetch);
                else run(std::true_type{}, get, put, fetch);
            };
            if (last) run_rw(gsm, pepi, efetch);
            else run_rw(gsm, psm, nofetch);
            __syncthreads();
            s += k;
        }
    }
    // this quarter of both accumulators
    __syncthreads();
    for (int jl = tid; jl < Nq; jl += nthr) {
        op.acc[(((size_t)ct * 2 + 0) * (L + 1) + t) * N + jq + jl] = acc_s[spad(jl)];
        op.acc[(((size_t)ct * 2 + 1) * (L + 1) + t) * N + jq + jl] = acc_s[W + spad(jl)];
    }
    // no block leaves while another may still store into its shared memory
    cluster_sync();
}

}  // namespace

bool modup_cluster_fits(const fhe_ctx* c) { return c->N >= 256 && c->N <= kMaxSinglePassN; }

void launch_modup_cluster(const fhe_ctx* c, const OpModUpMac& op, cudaStream_t st)
{
    const int count = op.count();
    if (count <= 0) return;
    const int Nq = (int)c->N / 4;
    const size_t smem = (size_t)3 * ntt_smem_words(Nq) * sizeof(u64);
    ensure_smem((const void*)k_modup_cluster, smem);
    const int thr = std::min(kCqThreads, std::max(32, Nq >> 4));
    LaunchScope ls(c, OpModUpMac::family(), st);
    k_modup_cluster<<<kClusterCtas * count, thr, smem, st>>>(op, c->tabs());
}

}  // namespace fhe
