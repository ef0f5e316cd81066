// k_relin.cu -- relinearisation: RNS key switching with per-prime digits.
#include "ops.cuh"

namespace fhe {

size_t relin_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L)
{
    const size_t N = c->N;
    return arena_need({(size_t)n_ct * L * N * 8, (size_t)n_ct * 2 * (L + 1) * N * 8, (size_t)n_ct * 2 * N * 8});
}

void k_relin(const fhe_ctx* c, const u64* d3, u64* out2, uint32_t n_ct, uint32_t L, void* scratch, cudaStream_t st,
             const ulonglong2* key, bool single_pass)
{
    if (n_ct == 0) return;
    const size_t N = c->N;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = relin_scratch_bytes(c, n_ct, L);
    u64* D = (u64*)ar.take((size_t)n_ct * L * N * 8);
    u64* acc = (u64*)ar.take((size_t)n_ct * 2 * (L + 1) * N * 8);
    u64* Vp = (u64*)ar.take((size_t)n_ct * 2 * N * 8);

    OpDigitsInv s1{d3, D, (int)n_ct, (int)L, (int)N};
    launch_ntt<true>(c, s1, st, single_pass);
    OpModUpMac s2{d3, D, key ? key : c->d_ksk, acc, (int)n_ct, (int)L, (int)N, (int)c->L_top, modup_red_mask(c, L),
                  modup_lazy_mask(c, L)};
    launch_modup(c, s2, st, single_pass);
    OpAccPInv s3{acc, Vp, (int)n_ct, (int)L, (int)N, (int)c->L_top};
    launch_ntt<true>(c, s3, st, single_pass);
    OpModDown s4;
    s4.d3 = d3;
    s4.acc = acc;
    s4.Vp = Vp;
    s4.out = out2;
    s4.n = (int)n_ct;
    s4.L = (int)L;
    s4.N = (int)N;
    s4.d = make_divc(c, c->L_top, L);
    launch_ntt<false>(c, s4, st, single_pass);
}


OpKsRowInv make_ks_row_inv(const fhe_ctx* c, const u64* d3, const u64* acc, const u64* Vp, u64* V, int n, int L,
                           const KsExtra& ex)
{
    const DivC dp = make_divc(c, c->L_top, (uint32_t)L);
    OpKsRowInv op;
    op.d3 = d3;
    op.acc = acc;
    op.Vp = Vp;
    op.V = V;
    op.n = n;
    op.L = L;
    op.N = (int)c->N;
    op.ex = ex;
    op.p = dp.p;
    op.p_half = dp.p_half;
    op.pmod = dp.pmod[L - 1];
    op.pinv = dp.inv[L - 1];
    op.pinvs = dp.invs[L - 1];
    return op;
}

OpKsDivFwd make_ks_div_fwd(const fhe_ctx* c, const u64* d3, const u64* acc, const u64* Vp, const u64* V, u64* out,
                           int n, int L, const KsExtra& ex, const u64* addc, int addc_stride)
{
    OpKsDivFwd op;
    op.d3 = d3;
    op.acc = acc;
    op.Vp = Vp;
    op.V = V;
    op.out = out;
    op.addc = addc;
    op.addc_stride = addc_stride;
    op.n = n;
    op.L = L;
    op.N = (int)c->N;
    op.ex = ex;
    op.dp = make_divc(c, c->L_top, (uint32_t)L);
    op.dq = make_divc(c, (uint32_t)L - 1, (uint32_t)L - 1);
    op.small_mask = small_div_mask(c, c->primes[L - 1], (uint32_t)L - 1);
    return op;
}

size_t relin_rescale_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L)
{
    const size_t N = c->N;
    return arena_need({(size_t)n_ct * L * N * 8, (size_t)n_ct * 2 * (L + 1) * N * 8, (size_t)n_ct * 2 * N * 8,
                       (size_t)n_ct * 2 * N * 8});
}

void k_relin_rescale(const fhe_ctx* c, const u64* d3, u64* out, uint32_t n_ct, uint32_t L, void* scratch,
                     cudaStream_t st, const KsExtra* ex, const u64* addc, uint32_t addc_stride)
{
    if (n_ct == 0) return;
    const size_t N = c->N;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = relin_rescale_scratch_bytes(c, n_ct, L);
    u64* D = (u64*)ar.take((size_t)n_ct * L * N * 8);
    u64* acc = (u64*)ar.take((size_t)n_ct * 2 * (L + 1) * N * 8);
    u64* Vp = (u64*)ar.take((size_t)n_ct * 2 * N * 8);
    u64* V = (u64*)ar.take((size_t)n_ct * 2 * N * 8);
    const KsExtra none{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    const KsExtra& e = ex ? *ex : none;

    OpDigitsInv s1{d3, D, (int)n_ct, (int)L, (int)N};
    launch_ntt<true>(c, s1, st);
    OpModUpMac s2{d3, D, c->d_ksk, acc, (int)n_ct, (int)L, (int)N, (int)c->L_top, modup_red_mask(c, L),
                  modup_lazy_mask(c, L)};
    launch_modup(c, s2, st);
    // the P residues' and row L-1's inverse transforms in one launch
    OpKsPRowInv s34{make_ks_row_inv(c, d3, acc, Vp, V, (int)n_ct, (int)L, e), Vp, (int)c->L_top};
    launch_ntt<true>(c, s34, st);
    launch_ntt<false>(c, make_ks_div_fwd(c, d3, acc, Vp, V, out, (int)n_ct, (int)L, e, addc, (int)addc_stride), st);
}

// The inner-product step alone on caller buffers (the autotuner times it):
// L digits, keys laid out for L data primes plus one more (index L).
void k_modup_mac_step(const fhe_ctx* c, const u64* d3, const u64* D, const ulonglong2* ksk, u64* acc, uint32_t n_ct,
                      uint32_t L, cudaStream_t st)
{
    OpModUpMac op{d3, D, ksk, acc, (int)n_ct, (int)L, (int)c->N, (int)L, modup_red_mask(c, L),
                  modup_lazy_mask(c, L)};
    launch_modup(c, op, st);
}

}  // namespace fhe
