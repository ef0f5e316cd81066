// k_encrypt.cu -- encryption and decryption.
#include "launch.cuh"

namespace fhe {

// ---------------------------------------------------------------- encrypt
// The integer samples of a ciphertext (u, e0, e1) are drawn once per
// coefficient by k_sample_enc (int8, [n][3][N]) and then reduced into every
// residue by the transform prologue.
__device__ __forceinline__ i64 draw_gauss_bs(u64 s0, int j, const u64* __restrict__ cdt)
{
    const u64 u = sm_out(s0, (u64)j);
    int lo = 0, hi = 38;                 // number of thresholds <= u (table increasing)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&cdt[mid]) <= u) lo = mid + 1;
        else hi = mid;
    }
    return (i64)lo - 19;
}

__global__ void k_sample_enc_kernel(int8_t* __restrict__ S, int n, int N, u64 seed, u64 first,
                                    const u64* __restrict__ cdt)
{
    const size_t total = (size_t)n * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i / N), j = (int)(i % N);
        const u64 id = first + (u64)ci;
        int8_t* o = S + (size_t)ci * 3 * N + j;
        o[0] = (int8_t)draw_ternary(sm_out(sm_out(seed, (u64)DOM_ENC_U), id), j);
        o[N] = (int8_t)draw_gauss_bs(sm_out(sm_out(seed, (u64)DOM_ENC_E0), id), j, cdt);
        o[2 * (size_t)N] = (int8_t)draw_gauss_bs(sm_out(sm_out(seed, (u64)DOM_ENC_E1), id), j, cdt);
    }
}

// per (ct, r): sub 0 = u, sub 1 = e0, sub 2 = e1
struct OpEncrypt {
    static const char* family() { return "encrypt"; }
    static constexpr bool kTransformBound = true;   // int8 samples in; three transforms per output pair
    const u64* pt;      // [n][Ltop][N]
    const u64* pk;      // [2][Ltop][N]
    const u64* pks;     // their Shoup quotients
    u64* ct;            // [n][2][Ltop][N]
    const int8_t* S;    // [n][3][N] samples
    const i64* M;       // optional [n][N] encoded coefficients (then pt is unused):
                        // NTT(e0) + NTT(m) = NTT(e0 + m), so the plaintext needs no transform of its own
    int n, Ltop, N;
    __host__ __device__ int count() const { return n * Ltop; }
    __host__ __device__ int nsub(int) const { return 3; }
    __device__ int prime(int p, int) const { return p % Ltop; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& P) const
    {
        const int ci = p / Ltop;
        i64 v = (i64)S[((size_t)ci * 3 + u) * N + j];
        if (u == 1 && M) return from_signed(v + M[(size_t)ci * N + j], P);
        return v >= 0 ? (u64)v : P.q - (u64)(-v);        // a sample, |v| <= 19 < q
    }
    struct Pre { u64 a, b, bs, c, cs; };
    __device__ Pre pre(int p, int u, int j) const
    {
        const int ci = p / Ltop, r = p % Ltop;
        Pre x;
        if (u == 0) {
            x.a = M ? 0 : pt[((size_t)ci * Ltop + r) * N + j];
            x.b = pk[(size_t)r * N + j];
            x.bs = pks[(size_t)r * N + j];
            x.c = pk[((size_t)Ltop + r) * N + j];
            x.cs = pks[((size_t)Ltop + r) * N + j];
        } else {
            x.a = ct[(((size_t)ci * 2 + (u == 1 ? 0 : 1)) * Ltop + r) * N + j];
            x.b = x.bs = x.c = x.cs = 0;
        }
        return x;
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& P) const
    {
        const int ci = p / Ltop, r = p % Ltop;
        u64* c0 = ct + (((size_t)ci * 2 + 0) * Ltop + r) * N;
        u64* c1 = ct + (((size_t)ci * 2 + 1) * Ltop + r) * N;
        if (u == 0) {
            c0[j] = add_mod(mul_shoup(v, pr.b, pr.bs, P.q), pr.a, P.q);
            c1[j] = mul_shoup(v, pr.c, pr.cs, P.q);
        } else if (u == 1) {
            c0[j] = add_mod(pr.a, v, P.q);
        } else {
            c1[j] = add_mod(pr.a, v, P.q);
        }
    }
};

size_t encrypt_scratch_bytes(const fhe_ctx* c, uint32_t n_ct) { return (size_t)n_ct * 3 * c->N; }

void k_encrypt(const fhe_ctx* c, const u64* pt, uint32_t n_ct, uint64_t first_id, u64* ct, void* scratch,
               cudaStream_t st)
{
    if (n_ct == 0) return;
    int8_t* S = (int8_t*)scratch;
    {
        const size_t total = (size_t)n_ct * c->N;
        LaunchScope ls(c, "encrypt", st);
        k_sample_enc_kernel<<<ew_grid(total), 256, 0, st>>>(S, (int)n_ct, (int)c->N, c->seed, first_id, c->d_cdt);
    }
    OpEncrypt op{pt, c->d_pk, c->d_pks, ct, S, nullptr, (int)n_ct, (int)c->L_top, (int)c->N};
    launch_ntt<false>(c, op, st);
}

size_t encode_encrypt_scratch_bytes(const fhe_ctx* c, uint32_t n_ct)
{
    return arena_need({encode_scratch_bytes(c, n_ct), encrypt_scratch_bytes(c, n_ct)});
}

void k_encode_encrypt(const fhe_ctx* c, const double* slots, uint32_t n_ct, double scale, uint64_t first_id, u64* ct,
                      void* scratch, cudaStream_t st)
{
    if (n_ct == 0) return;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = encode_encrypt_scratch_bytes(c, n_ct);
    i64* m = (i64*)ar.take(encode_scratch_bytes(c, n_ct));
    int8_t* S = (int8_t*)ar.take(encrypt_scratch_bytes(c, n_ct));
    encode_coefficients(c, slots, n_ct, scale, m, st);
    {
        const size_t total = (size_t)n_ct * c->N;
        LaunchScope ls(c, "encrypt", st);
        k_sample_enc_kernel<<<ew_grid(total), 256, 0, st>>>(S, (int)n_ct, (int)c->N, c->seed, first_id, c->d_cdt);
    }
    OpEncrypt op{nullptr, c->d_pk, c->d_pks, ct, S, m, (int)n_ct, (int)c->L_top, (int)c->N};
    launch_ntt<false>(c, op, st);
}

// ---------------------------------------------------------------- decrypt
// prologue: c0 + c1 s at residue 0 (NTT form); INTT; centred lift
struct OpDecrypt {
    static const char* family() { return "decrypt"; }
    const u64* ct;
    const u64* s;
    i64* m;
    int n, L, N;
    __host__ __device__ int count() const { return n; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return 0; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& P) const
    {
        const u64 c0 = ct[(((size_t)p * 2 + 0) * L) * N + j];
        const u64 c1 = ct[(((size_t)p * 2 + 1) * L) * N + j];
        return add_mod(c0, mul_mod_r(c1, s[j], P), P.q);
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC& P) const
    {
        m[(size_t)p * N + j] = v > P.half ? (i64)v - (i64)P.q : (i64)v;
    }
};

void k_decrypt(const fhe_ctx* c, const u64* ct, uint32_t n_ct, uint32_t L, i64* m, cudaStream_t st)
{
    OpDecrypt op{ct, c->d_s, m, (int)n_ct, (int)L, (int)c->N};
    launch_ntt<true>(c, op, st);
}


}  // namespace fhe
