// k_keys.cu -- key generation (secret, public, relinearisation and rotation
// keys) and the Galois automorphism.
#include "launch.cuh"

namespace fhe {

// ---------------------------------------------------------------- keys

// s (ternary) in every key prime
struct OpSecret {
    static const char* family() { return "keygen"; }
    static constexpr bool kColdPath = true;       // once per context
    u64* s;
    u64 s0;
    int nprimes, N;
    __host__ __device__ int count() const { return nprimes; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int, int, int j, const PrimeC& P) const { return from_signed(draw_ternary(s0, j), P); }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { s[(size_t)p * N + j] = v; }
};

// pk = (-a s + e, a) over the data primes: sub 0 = a (uniform), sub 1 = e
struct OpPublicKey {
    static const char* family() { return "keygen"; }
    static constexpr bool kColdPath = true;       // once per context
    const u64* s;
    u64* pk;            // [2][Ltop][N]
    const u64* cdt;
    u64 sa, se;
    int Ltop, N;
    __host__ __device__ int count() const { return Ltop; }
    __host__ __device__ int nsub(int) const { return 2; }
    __device__ int prime(int p, int) const { return p; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        return u == 0 ? draw_uniform(sa, j, p, P) : from_signed(draw_gauss(se, j, cdt), P);
    }
    struct Pre { u64 x; };
    __device__ Pre pre(int p, int u, int j) const
    {
        return {u == 0 ? s[(size_t)p * N + j] : pk[(size_t)p * N + j]};
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        u64* b = pk + (size_t)p * N;
        u64* a = pk + ((size_t)Ltop + p) * N;
        if (u == 0) {
            a[j] = v;
            b[j] = sub_mod(0, mul_mod(v, pr.x, P), P.q);
        } else {
            b[j] = add_mod(pr.x, v, P.q);
        }
    }
};

// ksk_j = (-a_j s + e_j + [r == j] P s^2, a_j) over every key prime r; each
// key word is stored with its Shoup quotient floor(k 2^64 / q)
__device__ __forceinline__ ulonglong2 with_shoup(u64 k, u64 q)
{
    return make_ulonglong2(k, (u64)(((unsigned __int128)k << 64) / q));
}

// A rotation key (galois = k, the Galois element) has s(X^k) in place of s^2.
// In NTT form s(X^k) is a permutation of s: index j holds the evaluation at
// psi^(2 brv(j) + 1), and s(X^k) there is s at psi^((2 brv(j) + 1) k).
__device__ __forceinline__ int galois_index(int j, u64 k, int logN)
{
    const unsigned b = __brev((unsigned)j) >> (32 - logN);
    const u64 e = ((2ull * b + 1ull) * k) & ((2ull << logN) - 1ull);
    return (int)(__brev((unsigned)((e - 1) >> 1)) >> (32 - logN));
}

struct OpRelinKey {
    static const char* family() { return "keygen"; }
    static constexpr bool kColdPath = true;       // once per context
    const u64* s;
    ulonglong2* ksk;    // [Ltop][2][Ltop+1][N]
    const u64* cdt;
    const u64* sa;      // per digit stream keys (device array [Ltop])
    const u64* se;
    u64 Pmod[33];       // P mod q_r
    int Ltop, N;
    u64 galois = 0;     // 0: relinearisation key (s^2); else rotation key for this k
    int logN = 0;
    __host__ __device__ int count() const { return Ltop * (Ltop + 1); }
    __host__ __device__ int nsub(int) const { return 2; }
    __device__ int prime(int p, int) const { return p % (Ltop + 1); }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        const int dj = p / (Ltop + 1), r = p % (Ltop + 1);
        return u == 0 ? draw_uniform(sa[dj], j, r, P) : from_signed(draw_gauss(se[dj], j, cdt), P);
    }
    struct Pre { u64 sr, b, sk; };
    __device__ Pre pre(int p, int u, int j) const
    {
        const int dj = p / (Ltop + 1), r = p % (Ltop + 1);
        Pre x;
        x.sr = s[(size_t)r * N + j];
        x.b = u == 1 ? ksk[(((size_t)dj * 2 + 0) * (Ltop + 1) + r) * N + j].x : 0;
        x.sk = (galois && u == 1 && r == dj) ? s[(size_t)r * N + galois_index(j, galois, logN)] : 0;
        return x;
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        const int dj = p / (Ltop + 1), r = p % (Ltop + 1);
        ulonglong2* b = ksk + (((size_t)dj * 2 + 0) * (Ltop + 1) + r) * N;
        ulonglong2* a = ksk + (((size_t)dj * 2 + 1) * (Ltop + 1) + r) * N;
        if (u == 0) {
            a[j] = with_shoup(v, P.q);
            b[j] = make_ulonglong2(sub_mod(0, mul_mod(v, pr.sr, P), P.q), 0);
        } else {
            u64 x = add_mod(pr.b, v, P.q);
            if (r == dj) x = add_mod(x, mul_mod(Pmod[r], galois ? pr.sk : mul_mod(pr.sr, pr.sr, P), P), P.q);
            b[j] = with_shoup(x, P.q);
        }
    }
};

// Shoup quotients of the public key, so encryption multiplies by it with one
// Shoup product per word
__global__ void k_pk_shoup_kernel(const u64* __restrict__ pk, u64* __restrict__ pks, size_t total, int Lt, int logN,
                                  const PrimeC* __restrict__ pc)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)((i >> logN) % Lt);
        pks[i] = with_shoup(pk[i], pc[r].q).y;
    }
}

void k_keygen(fhe_ctx* c, cudaStream_t st)
{
    const int N = (int)c->N, Lt = (int)c->L_top;
    OpSecret os{c->d_s, stream_key(c->seed, DOM_SECRET, 0), Lt + 1, N};
    launch_ntt<false>(c, os, st);
    OpPublicKey op{c->d_s, c->d_pk, c->d_cdt, stream_key(c->seed, DOM_PK_A, 0), stream_key(c->seed, DOM_PK_E, 0), Lt, N};
    launch_ntt<false>(c, op, st);
    {
        const size_t total = (size_t)2 * Lt * N;
        LaunchScope ls(c, "keygen", st);
        k_pk_shoup_kernel<<<ew_grid(total), 256, 0, st>>>(c->d_pk, c->d_pks, total, Lt, (int)c->logN, c->d_pc);
    }
    std::vector<u64> h(2 * Lt);
    for (int j = 0; j < Lt; ++j) {
        h[j] = stream_key(c->seed, DOM_KSK_A, (u64)j);
        h[Lt + j] = stream_key(c->seed, DOM_KSK_E, (u64)j);
    }
    u64* dkeys = nullptr;
    cudaMallocAsync((void**)&dkeys, h.size() * 8, st);
    cudaMemcpyAsync(dkeys, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st);
    OpRelinKey ok;
    ok.s = c->d_s;
    ok.ksk = c->d_ksk;
    ok.cdt = c->d_cdt;
    ok.sa = dkeys;
    ok.se = dkeys + Lt;
    for (int r = 0; r <= Lt && r < 33; ++r) ok.Pmod[r] = c->primes[Lt] % c->primes[r];
    ok.Ltop = Lt;
    ok.N = N;
    launch_ntt<false>(c, ok, st);
    cudaFreeAsync(dkeys, st);
}

void k_galois_keygen(fhe_ctx* c, u64 k, ulonglong2* key, cudaStream_t st)
{
    const int N = (int)c->N, Lt = (int)c->L_top;
    std::vector<u64> h(2 * Lt);
    for (int j = 0; j < Lt; ++j) {
        h[j] = stream_key(c->seed, DOM_GAL_A, (k << 8) | (u64)j);
        h[Lt + j] = stream_key(c->seed, DOM_GAL_E, (k << 8) | (u64)j);
    }
    u64* dkeys = nullptr;
    cudaMallocAsync((void**)&dkeys, h.size() * 8, st);
    cudaMemcpyAsync(dkeys, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st);
    OpRelinKey ok;
    ok.s = c->d_s;
    ok.ksk = key;
    ok.cdt = c->d_cdt;
    ok.sa = dkeys;
    ok.se = dkeys + Lt;
    for (int r = 0; r <= Lt && r < 33; ++r) ok.Pmod[r] = c->primes[Lt] % c->primes[r];
    ok.Ltop = Lt;
    ok.N = N;
    ok.galois = k;
    ok.logN = (int)c->logN;
    launch_ntt<false>(c, ok, st);
    cudaFreeAsync(dkeys, st);
}

// (c0(X^k), 0, c1(X^k)): NTT-form automorphism is the index permutation above
__global__ void k_automorph_kernel(const u64* __restrict__ ct, u64* __restrict__ d3, size_t total, int L, int logN,
                                   u64 k)
{
    const size_t Nm = ((size_t)1 << logN) - 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t row = (uint32_t)(i >> logN);         // (ct, comp of d3, r), 32-bit index math
        const uint32_t rest = row / (uint32_t)L, r = row - rest * (uint32_t)L;
        const uint32_t n = rest / 3u;
        const int comp = (int)(rest - n * 3u);
        const int j = (int)(i & Nm);
        u64 v = 0;
        if (comp != 1) {
            const int src_comp = comp == 0 ? 0 : 1;
            v = ct[((((size_t)n * 2 + src_comp) * L + r) << logN) + galois_index(j, k, logN)];
        }
        d3[i] = v;
    }
}

void k_automorph(const fhe_ctx* c, const u64* ct, u64* d3, uint32_t n_ct, uint32_t L, u64 k, cudaStream_t st)
{
    const size_t total = (size_t)n_ct * 3 * L * c->N;
    if (!total) return;
    LaunchScope ls(c, "elementwise", st);
    k_automorph_kernel<<<ew_grid(total), 256, 0, st>>>(ct, d3, total, (int)L, (int)c->logN, k);
}

}  // namespace fhe
