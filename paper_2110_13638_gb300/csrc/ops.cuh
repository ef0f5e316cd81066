// ops.cuh -- the fused-transform ops of rescale and key switching, shared by
// their own launchers and the multi-batch (uneven level) launcher.
#pragma once
#include "launch.cuh"

namespace fhe {

// ---------------------------------------------------------------- rescale

// INTT of one residue row per (ct, comp) into scratch V (coefficient form)
struct OpTakeRowInv {
    static const char* family() { return "rescale_intt"; }
    const u64* in;
    u64* V;
    int n, L, row, N, pidx;
    const u64* mulc;    // optional: the input is first multiplied by this per-residue constant
    const u64* mulcs;   // its Shoup quotients (with mulc)
    __host__ __device__ int count() const { return n; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return pidx; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& P) const
    {
        const u64 x = in[((size_t)p * L + row) * N + j];
        return mulc ? mul_shoup(x, mulc[row], mulcs[row], P.q) : x;
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { V[(size_t)p * N + j] = v; }
};

// out_i = (in_i - NTT([v]_{q_i})) * p^{-1} (+ addc on comp 0)
struct OpDivFwd {
    static const char* family() { return "rescale_ntt"; }
    const u64* in;      // [n_poly][L_in][N]
    const u64* V;       // [n_poly][N]  coefficient form mod p
    u64* out;           // [n_poly][L_out][N]
    const u64* addc;    // optional: residues of a constant added to comp 0, [n_ct][addc_stride]
    int n_poly, comps, L_in, L_out, N, addc_stride;
    const u64* mulc;    // optional: the input is first multiplied by this per-residue constant
    const u64* mulcs;   // its Shoup quotients (with mulc)
    DivC d;
    uint32_t small_mask;   // targets i with p < 2 q_i (centred remainder by one conditional add)
    __host__ __device__ int count() const { return n_poly * L_out; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L_out; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int poly = p / L_out, i = p % L_out;
        const u64 v = V[(size_t)poly * N + j];
        // p < 2 q_i: v and v - p + q_i (for the negative lift) are below 2 q_i
        if ((small_mask >> i) & 1u) return v > d.p_half ? v + Q.q - d.p : v;
        return centred_to(v, d.p, d.p_half, d.pmod[i], Q);
    }
    struct Pre { u64 x, c; };
    __device__ Pre pre(int p, int, int j) const
    {
        const int poly = p / L_out, i = p % L_out;
        Pre r;
        r.x = in[((size_t)poly * L_in + i) * N + j];
        r.c = (addc && (poly % comps) == 0) ? addc[(size_t)(poly / comps) * addc_stride + i] : 0;
        return r;
    }
    __device__ void store(int p, int, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int poly = p / L_out, i = p % L_out;
        const u64 x = mulc ? mul_shoup(pr.x, mulc[i], mulcs[i], Q.q) : pr.x;
        const u64 r = mul_shoup(sub_mod(x, v, Q.q), d.inv[i], d.invs[i], Q.q);
        out[((size_t)poly * L_out + i) * N + j] = add_mod(r, pr.c, Q.q);
    }
};

// rescale of x C (per-residue constant C) fused with the tensor product of the
// result w and a second ciphertext x2 at the output level: unit (ct, i) runs
// the forward transforms of both components (sub k = 0, 1); sub 0 keeps w_0
// in scratch, sub 1 forms (x2_0 w_0, x2_0 w_1 + x2_1 w_0, x2_1 w_1) at residue
// i.  The element-to-thread mapping of both subs' epilogues is the same, so
// the w_0 word sub 1 reads was written by the same thread.
struct OpDivFwdTensor {
    static const char* family() { return "rescale_ntt"; }
    const u64* in;      // [n][2][L_in][N]: x
    const u64* V;       // [n][2][N] coefficient form mod q_{L_in-1} (of x C)
    const u64* mulc;    // C residues and their Shoup quotients
    const u64* mulcs;
    const u64* x2;      // [n][2][L_out][N]
    u64* W0;            // [n][L_out][N] scratch: w_0
    u64* out3;          // [n][3][L_out][N]
    int n, L_in, L_out, N;
    DivC d;
    uint32_t small_mask;
    __host__ __device__ int count() const { return n * L_out; }
    __host__ __device__ int nsub(int) const { return 2; }
    __device__ int prime(int p, int) const { return p % L_out; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int k, int j, const PrimeC& Q) const
    {
        const int ct = p / L_out, i = p % L_out;
        const u64 v = V[((size_t)ct * 2 + k) * N + j];
        if ((small_mask >> i) & 1u) return v > d.p_half ? v + Q.q - d.p : v;
        return centred_to(v, d.p, d.p_half, d.pmod[i], Q);
    }
    struct Pre { u64 x, w0, a0, a1; };
    __device__ Pre pre(int p, int k, int j) const
    {
        const int ct = p / L_out, i = p % L_out;
        Pre r;
        r.x = in[(((size_t)ct * 2 + k) * L_in + i) * N + j];
        r.w0 = k ? W0[((size_t)ct * L_out + i) * N + j] : 0;
        r.a0 = k ? x2[(((size_t)ct * 2 + 0) * L_out + i) * N + j] : 0;
        r.a1 = k ? x2[(((size_t)ct * 2 + 1) * L_out + i) * N + j] : 0;
        return r;
    }
    __device__ void store(int p, int k, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int ct = p / L_out, i = p % L_out;
        const u64 x = mul_shoup(pr.x, mulc[i], mulcs[i], Q.q);
        const u64 w = mul_shoup(sub_mod(x, v, Q.q), d.inv[i], d.invs[i], Q.q);
        if (k == 0) {
            W0[((size_t)ct * L_out + i) * N + j] = w;
            return;
        }
        const size_t o = (((size_t)ct * 3) * L_out + i) * N + j, st3 = (size_t)L_out * N;
        out3[o] = mul_mod_r(pr.a0, pr.w0, Q);
        out3[o + st3] = add_mod(mul_mod_r(pr.a0, w, Q), mul_mod_r(pr.a1, pr.w0, Q), Q.q);
        out3[o + 2 * st3] = mul_mod_r(pr.a1, w, Q);
    }
};

// ---------------------------------------------------------------- relinearise
// The three components of a tensor product d = (a0 b0, a0 b1 + a1 b0, a1 b1):
// read from a stored [n][3][L][N] batch (D3Src<false>), or recomputed from
// the factors a, b ([n][2][L][N]) where they are needed (D3Src<true>: no
// tensor is written to memory).
template <bool TENSOR>
struct D3Src;

template <>
struct D3Src<false> {
    const u64* d3 = nullptr;
    __host__ __device__ D3Src() {}
    __host__ __device__ D3Src(const u64* t) : d3(t) {}
    // component k, residue i (prime Q), coefficient j of ciphertext ct
    __device__ __forceinline__ u64 get(int ct, int k, int L, int N, int i, int j, const PrimeC&) const
    {
        return d3[(((size_t)ct * 3 + k) * L + i) * N + j];
    }
};

template <>
struct D3Src<true> {
    const u64* a = nullptr;
    const u64* b = nullptr;
    __host__ __device__ D3Src() {}
    __host__ __device__ D3Src(const u64* a_, const u64* b_) : a(a_), b(b_) {}
    __device__ __forceinline__ u64 get(int ct, int k, int L, int N, int i, int j, const PrimeC& Q) const
    {
        const size_t o0 = (((size_t)ct * 2) * L + i) * N + j, o1 = o0 + (size_t)L * N;
        if (k == 0) return mul_mod_r(a[o0], b[o0], Q);
        if (k == 2) return mul_mod_r(a[o1], b[o1], Q);
        return add_mod(mul_mod_r(a[o0], b[o1], Q), mul_mod_r(a[o1], b[o0], Q), Q.q);
    }
};

// step 1: digits D_j = INTT(d2_j) in [0, q_j)
template <bool TENSOR>
struct OpDigitsInvT {
    static const char* family() { return "keyswitch_intt"; }
    static constexpr bool kTransformBound = true;   // one row in, one row out
    D3Src<TENSOR> d3;   // [n][3][L][N]
    u64* D;             // [n][L][N]
    int n, L, N;
    __host__ __device__ int count() const { return n * L; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int ct = p / L, r = p % L;
        return d3.get(ct, 2, L, N, r, j, Q);
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { D[(size_t)p * N + j] = v; }
};
using OpDigitsInv = OpDigitsInvT<false>;

// digits u < L whose prime q_u exceeds 4 q_t for some target t in {q_0..q_{L-1}, P}:
// their lift into q_t must be reduced before the forward transform, which
// accepts inputs below 4 q_t
inline uint32_t modup_red_mask(const fhe_ctx* c, uint32_t L)
{
    u64 qmin = c->primes[c->L_top];
    for (uint32_t t = 0; t < L; ++t) qmin = c->primes[t] < qmin ? c->primes[t] : qmin;
    uint32_t m = 0;
    for (uint32_t u = 0; u < L; ++u)
        if (c->primes[u] / 4 >= qmin) m |= 1u << u;
    return m;
}

// targets t in 0..L (t = L: the special prime) whose accumulators may stay
// unreduced: L lazy Shoup products below 2 q_t each sum below 2^64
inline uint64_t modup_lazy_mask(const fhe_ctx* c, uint32_t L)
{
    uint64_t m = 0;
    for (uint32_t t = 0; t <= L; ++t) {
        const u64 q = c->primes[t == L ? c->L_top : t];
        if (q < (1ull << 63) / L) m |= 1ull << t;
    }
    return m;
}

// step 2: per (ct, target t in 0..L, t = L meaning P): for every digit u,
// NTT(D_u mod q_t) * ksk_u[k][t], accumulated over u into acc[ct][k][t].
// Keys carry their Shoup quotients, so each key product is one Shoup product.
template <bool TENSOR>
struct OpModUpMacT {
    static const char* family() { return "keyswitch_modup_mac"; }
    static constexpr bool kLazyStore = true;     // the key products reduce any v < 2^64
    static constexpr bool kKeySwitchMac = true;  // scheduled separately (heavy epilogue)
    D3Src<TENSOR> d3;
    const u64* D;
    const ulonglong2* ksk;  // [L_top][2][L_top+1][N] (k, floor(k 2^64 / q))
    u64* acc;               // [n][2][L+1][N]
    int n, L, N, Ltop;
    uint32_t red_mask;      // digits u whose prime exceeds 4 q_t for some target t:
                            // only these need reducing before the forward transform
    uint64_t lazy_mask;     // targets t (L = P) whose sums are kept unreduced: the L key
                            // products, each below 2 q_t, then sum below 2 L q_t < 2^64
    __host__ __device__ int count() const { return n * (L + 1); }
    __host__ __device__ int nsub(int) const { return L; }
    // unit p = ct (L + 1) + t: the L + 1 targets of one ciphertext run side
    // by side and share its digits' reads from L2
    __host__ __device__ __forceinline__ int ct_of(int p) const { return p / (L + 1); }
    __host__ __device__ __forceinline__ int t_of(int p) const { return p % (L + 1); }
    __device__ int prime(int p, int) const
    {
        const int t = t_of(p);
        return t == L ? Ltop : t;
    }
    __device__ bool direct(int p, int u) const { return t_of(p) == u; }
    __device__ u64 load(int p, int u, int j, const PrimeC& Q) const
    {
        const int ct = ct_of(p);
        const u64 d = D[((size_t)ct * L + u) * N + j];       // in [0, q_u)
        return ((red_mask >> u) & 1u) ? reduce64(d, Q) : d;
    }
    struct Pre {
        ulonglong2 k0, k1;
        u64 a0, a1;
    };
    __device__ Pre pre(int p, int u, int j) const
    {
        const int ct = ct_of(p), t = t_of(p);
        const int tk = t == L ? Ltop : t;
        Pre r;
        r.k0 = __ldg(&ksk[(((size_t)u * 2 + 0) * (Ltop + 1) + tk) * N + j]);
        r.k1 = __ldg(&ksk[(((size_t)u * 2 + 1) * (Ltop + 1) + tk) * N + j]);
        if (u > 0) {
            r.a0 = acc[(((size_t)ct * 2 + 0) * (L + 1) + t) * N + j];
            r.a1 = acc[(((size_t)ct * 2 + 1) * (L + 1) + t) * N + j];
        } else {
            r.a0 = r.a1 = 0;
        }
        return r;
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int ct = ct_of(p), t = t_of(p);
        if (t == u) v = d3.get(ct, 2, L, N, t, j, Q);                 // direct: NTT(d2_t) is d2_t
        u64* a0 = acc + (((size_t)ct * 2 + 0) * (L + 1) + t) * N + j;
        u64* a1 = acc + (((size_t)ct * 2 + 1) * (L + 1) + t) * N + j;
        if ((lazy_mask >> t) & 1u) {                                   // block-uniform
            const u64 p0 = mul_shoup_lazy(v, pr.k0.x, pr.k0.y, Q.q);
            const u64 p1 = mul_shoup_lazy(v, pr.k1.x, pr.k1.y, Q.q);
            *a0 = u == 0 ? p0 : pr.a0 + p0;
            *a1 = u == 0 ? p1 : pr.a1 + p1;
        } else {
            const u64 p0 = mul_shoup(v, pr.k0.x, pr.k0.y, Q.q);
            const u64 p1 = mul_shoup(v, pr.k1.x, pr.k1.y, Q.q);
            *a0 = u == 0 ? p0 : add_mod(pr.a0, p0, Q.q);
            *a1 = u == 0 ? p1 : add_mod(pr.a1, p1, Q.q);
        }
    }
};
using OpModUpMac = OpModUpMacT<false>;

// step 3: INTT of the P residue of both accumulators
struct OpAccPInv {
    static const char* family() { return "keyswitch_acc_intt"; }
    const u64* acc;
    u64* Vp;            // [n][2][N]
    int n, L, N, Ltop;
    __host__ __device__ int count() const { return n * 2; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return Ltop; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        return reduce64(acc[((size_t)p * (L + 1) + L) * N + j], Q);   // the sum may be unreduced
    }
    struct Pre {};
    __device__ Pre pre(int, int, int) const { return {}; }
    __device__ void store(int p, int, int j, u64 v, const Pre&, const PrimeC&) const { Vp[(size_t)p * N + j] = v; }
};

// step 4: ModDown + add: out_k,t = d_k,t + (acc_k,t - NTT([v]_{q_t})) * P^{-1}
struct OpModDown {
    static const char* family() { return "keyswitch_moddown"; }
    const u64* d3;
    const u64* acc;
    const u64* Vp;
    u64* out;           // [n][2][L][N]
    int n, L, N;
    DivC d;
    __host__ __device__ int count() const { return n * 2 * L; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % L; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int poly = p / L, t = p % L;             // poly = ct*2 + k
        return centred_to(Vp[(size_t)poly * N + j], d.p, d.p_half, d.pmod[t], Q);
    }
    struct Pre { u64 a, dk; };
    __device__ Pre pre(int p, int, int j) const
    {
        const int poly = p / L, t = p % L;
        const int ct = poly >> 1, k = poly & 1;
        Pre r;
        r.a = acc[((size_t)poly * (L + 1) + t) * N + j];
        r.dk = d3[(((size_t)ct * 3 + k) * L + t) * N + j];
        return r;
    }
    __device__ void store(int p, int, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int poly = p / L, t = p % L;
        const int ct = poly >> 1, k = poly & 1;
        const u64 ks = mul_shoup(sub_mod(reduce64(pr.a, Q), v, Q.q), d.inv[t], d.invs[t], Q.q);
        out[(((size_t)ct * 2 + k) * L + t) * N + j] = add_mod(pr.dk, ks, Q.q);
    }
};

// ---------------------------------------------------------------- relinearise + rescale
// ModDown and the rescale right after it, with the forward transforms of the
// two corrections merged.  With v = centred INTT_P(acc_P) (ModDown's
// remainder), R = d + E + (acc - NTT([v])) P^-1 the relinearised ciphertext
// (E an optional NTT-form term added before the rescale) and r = centred
// INTT_{q_{L-1}}(R_{L-1}) (the rescale's remainder):
//   INTT(R_{L-1}) = INTT(d_{L-1} + E_{L-1} + acc_{L-1} P^-1) - [v]_{L-1} P^-1
//   out_i = (d_i + E_i + acc_i P^-1 - NTT([v]_i P^-1 + [r]_i)) q_{L-1}^-1,  i < L-1
// The transforms are linear mod q_i, so out is word for word ModDown
// followed by the rescale: both centred roundings are taken exactly as
// there, but each output row needs one forward transform instead of two.

// step 4': INTT of row L-1 of the relinearised ciphertext, per (ct, comp)
template <bool TENSOR>
struct OpKsRowInvT {
    static const char* family() { return "keyswitch_rescale_intt"; }
    D3Src<TENSOR> d3;   // [n][3][L][N]
    const u64* acc;     // [n][2][L+1][N]
    const u64* Vp;      // [n][2][N] coefficient form mod P
    u64* V;             // [n][2][N] coefficient form mod q_{L-1}
    int n, L, N;
    KsExtra ex;
    u64 p, p_half, pmod, pinv, pinvs;    // P, (P-1)/2, P mod q_{L-1}, P^-1 mod q_{L-1} (+ Shoup)
    __host__ __device__ int count() const { return n * 2; }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int, int) const { return L - 1; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int ct = p >> 1, k = p & 1, i = L - 1;
        u64 s = d3.get(ct, k, L, N, i, j, Q);
        s = add_mod(s, mul_shoup(acc[((size_t)p * (L + 1) + i) * N + j], pinv, pinvs, Q.q), Q.q);
        if (ex.x2) s = add_mod(s, mul_shoup(ex.x2[((size_t)p * L + i) * N + j], ex.c2[i], ex.c2s[i], Q.q), Q.q);
        if (ex.x) s = add_mod(s, mul_shoup(ex.x[((size_t)p * ex.Lx + i) * N + j], ex.c1[i], ex.c1s[i], Q.q), Q.q);
        return s;
    }
    struct Pre { u64 v; };
    __device__ Pre pre(int p, int, int j) const { return {Vp[(size_t)p * N + j]}; }
    __device__ void store(int p, int, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const u64 vq = mul_shoup(centred_to(pr.v, this->p, p_half, pmod, Q), pinv, pinvs, Q.q);
        V[(size_t)p * N + j] = sub_mod(v, vq, Q.q);
    }
};
using OpKsRowInv = OpKsRowInvT<false>;

// steps 3 and 4' in one unit per (ct, comp): sub 0 is the inverse transform of
// the accumulator's P residue (into Vp), sub 1 that of row L-1 (into V), whose
// epilogue reads the Vp words sub 0 wrote (the same block, after its barrier)
template <bool TENSOR>
struct OpKsPRowInvT {
    static const char* family() { return "keyswitch_rescale_intt"; }
    OpKsRowInvT<TENSOR> row;    // its acc, V, constants; row.Vp is the array below
    u64* Vp;            // [n][2][N] written by sub 0
    int Ltop;
    __host__ __device__ int count() const { return row.n * 2; }
    __host__ __device__ int nsub(int) const { return 2; }
    __device__ int prime(int, int u) const { return u == 0 ? Ltop : row.L - 1; }
    __device__ bool direct(int, int) const { return false; }
    __device__ u64 load(int p, int u, int j, const PrimeC& Q) const
    {
        if (u == 0) return reduce64(row.acc[((size_t)p * (row.L + 1) + row.L) * row.N + j], Q);
        return row.load(p, 0, j, Q);
    }
    struct Pre { u64 v; };
    __device__ Pre pre(int p, int u, int j) const
    {
        return {u == 0 ? 0ull : Vp[(size_t)p * row.N + j]};
    }
    __device__ void store(int p, int u, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        if (u == 0) Vp[(size_t)p * row.N + j] = v;
        else row.store(p, 0, j, v, typename OpKsRowInvT<TENSOR>::Pre{pr.v}, Q);
    }
};
using OpKsPRowInv = OpKsPRowInvT<false>;

// step 5': the merged forward transform of both corrections into q_i, i < L-1,
// per (ct, comp, i), and the rescaled output row.  TENSOR: the tensor product
// is recomputed from its factors (the epilogue then loads the factors)
template <bool TENSOR>
struct OpKsDivFwdT {
    static const char* family() { return "keyswitch_rescale_ntt"; }
    D3Src<TENSOR> d3;   // [n][3][L][N] (TENSOR: the factors)
    const u64* acc;     // [n][2][L+1][N]
    const u64* Vp;      // [n][2][N] mod P
    const u64* V;       // [n][2][N] mod q_{L-1}
    u64* out;           // [n][2][L-1][N]
    const u64* addc;    // optional constants added to comp 0 of the result, [n][addc_stride]
    int n, L, N, addc_stride;
    KsExtra ex;
    DivC dp;            // division by P into q_0 .. q_{L-1}
    DivC dq;            // division by q_{L-1} into q_0 .. q_{L-2}
    uint32_t small_mask;   // targets i with q_{L-1} < 2 q_i
    __host__ __device__ int count() const { return n * 2 * (L - 1); }
    __host__ __device__ int nsub(int) const { return 1; }
    __device__ int prime(int p, int) const { return p % (L - 1); }
    __device__ bool direct(int, int) const { return false; }
    // the transform input [v]_i P^-1 + [r]_i, in [0, 4 q_i) (the forward
    // transforms accept that range)
    __device__ u64 load(int p, int, int j, const PrimeC& Q) const
    {
        const int poly = p / (L - 1), i = p % (L - 1);
        const u64 vp = Vp[(size_t)poly * N + j], vq = V[(size_t)poly * N + j];
        if ((small_mask >> i) & 1u) {
            // [v]_i P^-1 = v P^-1 - [v > P/2] (mod q_i) because P P^-1 = 1: a lazy
            // Shoup product of the unreduced v, less one, in [0, 2 q_i)
            u64 a = mul_shoup_lazy(vp, dp.inv[i], dp.invs[i], Q.q);
            if (vp > dp.p_half) a = a ? a - 1 : Q.q2 - 1;
            // [r]_i: r or r - q_{L-1} + q_i, both in [0, 2 q_i)
            const u64 b = vq > dq.p_half ? vq + Q.q - dq.p : vq;
            return a + b;
        }
        const u64 a = centred_to(vp, dp.p, dp.p_half, dp.pmod[i], Q);
        const u64 b = centred_to(vq, dq.p, dq.p_half, dq.pmod[i], Q);
        return add_mod(mul_shoup(a, dp.inv[i], dp.invs[i], Q.q), b, Q.q);
    }
    // d the stored component (or, TENSOR, the factors: d = a0 (b0 | b1), x2 = a1, x = b0)
    struct Pre { u64 d, a, x2, x, f; };
    __device__ Pre pre(int p, int, int j) const
    {
        const int poly = p / (L - 1), i = p % (L - 1);
        const int ct = poly >> 1, k = poly & 1;
        Pre r;
        r.a = acc[((size_t)poly * (L + 1) + i) * N + j];
        if constexpr (TENSOR) {
            const size_t o0 = (((size_t)ct * 2) * L + i) * N + j, o1 = o0 + (size_t)L * N;
            r.d = d3.a[o0];
            r.f = d3.b[k ? o1 : o0];
            r.x2 = k ? d3.a[o1] : 0;
            r.x = k ? d3.b[o0] : 0;
        } else {
            r.d = d3.d3[(((size_t)ct * 3 + k) * L + i) * N + j];
            r.f = 0;
            r.x2 = ex.x2 ? ex.x2[((size_t)poly * L + i) * N + j] : 0;
            r.x = ex.x ? ex.x[((size_t)poly * ex.Lx + i) * N + j] : 0;
        }
        return r;
    }
    __device__ void store(int p, int, int j, u64 v, const Pre& pr, const PrimeC& Q) const
    {
        const int poly = p / (L - 1), i = p % (L - 1);
        u64 d = pr.d;
        if constexpr (TENSOR) {
            d = mul_mod_r(pr.d, pr.f, Q);                        // a0 b0, or a0 b1
            if (poly & 1) d = add_mod(d, mul_mod_r(pr.x2, pr.x, Q), Q.q); // + a1 b0
        }
        u64 s = add_mod(d, mul_shoup(pr.a, dp.inv[i], dp.invs[i], Q.q), Q.q);
        if (!TENSOR && ex.x2) s = add_mod(s, mul_shoup(pr.x2, ex.c2[i], ex.c2s[i], Q.q), Q.q);
        if (!TENSOR && ex.x) s = add_mod(s, mul_shoup(pr.x, ex.c1[i], ex.c1s[i], Q.q), Q.q);
        u64 r = mul_shoup(sub_mod(s, v, Q.q), dq.inv[i], dq.invs[i], Q.q);
        if (addc && (poly & 1) == 0) r = add_mod(r, addc[(size_t)(poly >> 1) * addc_stride + i], Q.q);
        out[((size_t)poly * (L - 1) + i) * N + j] = r;
    }
};
using OpKsDivFwd = OpKsDivFwdT<false>;

// targets i < n with p < 2 q_i: there the centred lift of a residue mod p
// needs one conditional add instead of a reduction
inline uint32_t small_div_mask(const fhe_ctx* c, u64 p, uint32_t n)
{
    uint32_t m = 0;
    for (uint32_t i = 0; i < n && i < 32; ++i)
        if (p / 2 < c->primes[i]) m |= 1u << i;
    return m;
}

// Grouped (MultiOp) launches of the forward steps, each compiled in a
// translation unit of its own (k_groups_ks.cu, k_groups_fwd.cu) so the build
// runs them in parallel.
void launch_groups_modup_mac(const fhe_ctx* c, const MultiOp<OpModUpMac>& m, cudaStream_t st);
void launch_groups_ks_divfwd(const fhe_ctx* c, const MultiOp<OpKsDivFwd>& m, cudaStream_t st);

// Schedule 7 of the ModUp step (k_modup_cluster.cu): a cluster of four blocks
// per (ciphertext, target), accumulators in shared memory.
void launch_modup_cluster(const fhe_ctx* c, const OpModUpMac& op, cudaStream_t st);

// The ModUp step with the schedule the autotuner picked for it
// (k_relin_modup.cu, the only unit that instantiates the ModUp kernels of a
// stored tensor; k_relin_tensor.cu those of a recomputed one)
void launch_modup(const fhe_ctx* c, const OpModUpMac& op, cudaStream_t st, bool single_pass = false);
void launch_modup(const fhe_ctx* c, const OpModUpMacT<true>& op, cudaStream_t st);

// The merged ModDown + rescale of one batch (k_relin.cu): ops of steps 4' and 5'.
OpKsRowInv make_ks_row_inv(const fhe_ctx* c, const u64* d3, const u64* acc, const u64* Vp, u64* V, int n, int L,
                           const KsExtra& ex);
OpKsDivFwd make_ks_div_fwd(const fhe_ctx* c, const u64* d3, const u64* acc, const u64* Vp, const u64* V, u64* out,
                           int n, int L, const KsExtra& ex, const u64* addc, int addc_stride);

}  // namespace fhe
