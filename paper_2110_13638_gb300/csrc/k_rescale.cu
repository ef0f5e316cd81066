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


}  // namespace fhe
