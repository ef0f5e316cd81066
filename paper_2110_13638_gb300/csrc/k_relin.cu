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
    OpModUpMac s2{d3, D, key ? key : c->d_ksk, acc, (int)n_ct, (int)L, (int)N, (int)c->L_top, modup_red_mask(c, L)};
    launch_ntt<false>(c, s2, st, single_pass);
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


// The inner-product step alone on caller buffers (the autotuner times it):
// L digits, keys laid out for L data primes plus one more (index L).
void k_modup_mac_step(const fhe_ctx* c, const u64* d3, const u64* D, const ulonglong2* ksk, u64* acc, uint32_t n_ct,
                      uint32_t L, cudaStream_t st)
{
    OpModUpMac op{d3, D, ksk, acc, (int)n_ct, (int)L, (int)c->N, (int)L, modup_red_mask(c, L)};
    launch_ntt<false>(c, op, st);
}

}  // namespace fhe
