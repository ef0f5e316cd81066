// k_rescale.cu -- rescale: division by the last prime with the centred remainder.
#include "ops.cuh"

namespace fhe {

size_t rescale_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t comps)
{
    return (size_t)n_ct * comps * c->N * sizeof(u64);
}

void k_rescale(const fhe_ctx* c, const u64* in, u64* out, uint32_t n_ct, uint32_t comps, uint32_t L, const u64* addc,
               uint32_t addc_stride, void* scratch, cudaStream_t st, const u64* mulc, const u64* mulcs)
{
    if (n_ct == 0) return;
    u64* V = (u64*)scratch;
    OpTakeRowInv a;
    a.in = in;
    a.V = V;
    a.n = (int)(n_ct * comps);
    a.L = (int)L;
    a.row = (int)L - 1;
    a.N = (int)c->N;
    a.pidx = (int)L - 1;
    a.mulc = mulc;
    a.mulcs = mulcs;
    launch_ntt<true>(c, a, st);
    OpDivFwd b;
    b.in = in;
    b.V = V;
    b.out = out;
    b.addc = addc;
    b.addc_stride = (int)addc_stride;
    b.n_poly = (int)(n_ct * comps);
    b.comps = (int)comps;
    b.L_in = (int)L;
    b.L_out = (int)L - 1;
    b.N = (int)c->N;
    b.d = make_divc(c, L - 1, L - 1);
    b.small_mask = small_div_mask(c, c->primes[L - 1], L - 1);
    b.mulc = mulc;
    b.mulcs = mulcs;
    launch_ntt<false>(c, b, st);
}


size_t rescale_tensor_scratch_bytes(const fhe_ctx* c, uint32_t n_ct, uint32_t L)
{
    return arena_need({(size_t)n_ct * 2 * c->N * 8, (size_t)n_ct * (L - 1) * c->N * 8});
}

void k_rescale_tensor(const fhe_ctx* c, const u64* x, const u64* mulc, const u64* mulcs, const u64* x2, u64* out3,
                      uint32_t n_ct, uint32_t L, void* scratch, cudaStream_t st)
{
    if (n_ct == 0) return;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = rescale_tensor_scratch_bytes(c, n_ct, L);
    u64* V = (u64*)ar.take((size_t)n_ct * 2 * c->N * 8);
    u64* W0 = (u64*)ar.take((size_t)n_ct * (L - 1) * c->N * 8);
    OpTakeRowInv a;
    a.in = x;
    a.V = V;
    a.n = (int)(n_ct * 2);
    a.L = (int)L;
    a.row = (int)L - 1;
    a.N = (int)c->N;
    a.pidx = (int)L - 1;
    a.mulc = mulc;
    a.mulcs = mulcs;
    launch_ntt<true>(c, a, st);
    OpDivFwdTensor b;
    b.in = x;
    b.V = V;
    b.mulc = mulc;
    b.mulcs = mulcs;
    b.x2 = x2;
    b.W0 = W0;
    b.out3 = out3;
    b.n = (int)n_ct;
    b.L_in = (int)L;
    b.L_out = (int)L - 1;
    b.N = (int)c->N;
    b.d = make_divc(c, L - 1, L - 1);
    b.small_mask = small_div_mask(c, c->primes[L - 1], L - 1);
    launch_ntt<false>(c, b, st);
}

}  // namespace fhe
