// k_relin_tensor.cu -- relinearise + rescale of a tensor product a (x) b that
// is never stored: each step of the merged path (digit inverses, ModUp and
// key inner products, P and row L-1 inverses, merged ModDown + rescale
// forward transforms) recomputes the tensor component it needs from the
// factors (d2 = a1 b1 for the digits and the ModUp step's direct digit, row
// L-1 of d0 / d1 for the row inverse, d0 = a0 b0 and d1 = a0 b1 + a1 b0 in
// the forward epilogue), instead of a separate tensor launch writing 3 L rows
// per ciphertext that the steps read back.  In a translation unit of its own
// (its kernels are instantiations apart from the stored-tensor ones).
#include "ops.cuh"

namespace fhe {

// schedule 7 (the ModUp cluster kernel) takes a stored tensor; under it this
// step runs as schedule 6, which launch_ntt selects for it
void launch_modup(const fhe_ctx* c, const OpModUpMacT<true>& op, cudaStream_t st)
{
    launch_ntt<false>(c, op, st);
}

void k_mul_relin_rescale(const fhe_ctx* c, const u64* a, const u64* b, u64* out, uint32_t n_ct, uint32_t L,
                         void* scratch, cudaStream_t st)
{
    if (n_ct == 0) return;
    const int N = (int)c->N, n = (int)n_ct, l = (int)L;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = relin_rescale_scratch_bytes(c, n_ct, L);
    u64* D = (u64*)ar.take((size_t)n_ct * L * N * 8);
    u64* acc = (u64*)ar.take((size_t)n_ct * 2 * (L + 1) * N * 8);
    u64* Vp = (u64*)ar.take((size_t)n_ct * 2 * N * 8);
    u64* V = (u64*)ar.take((size_t)n_ct * 2 * N * 8);
    const KsExtra none{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    const D3Src<true> src(a, b);

    OpDigitsInvT<true> s1{src, D, n, l, N};
    launch_ntt<true>(c, s1, st);
    OpModUpMacT<true> s2{src, D, c->d_ksk, acc, n, l, N, (int)c->L_top, modup_red_mask(c, L), modup_lazy_mask(c, L)};
    launch_modup(c, s2, st);
    const OpKsRowInv r = make_ks_row_inv(c, nullptr, acc, Vp, V, n, l, none);
    OpKsPRowInvT<true> s34;
    s34.row = OpKsRowInvT<true>{src, r.acc, r.Vp, r.V, n, l, N, none, r.p, r.p_half, r.pmod, r.pinv, r.pinvs};
    s34.Vp = Vp;
    s34.Ltop = (int)c->L_top;
    launch_ntt<true>(c, s34, st);
    const OpKsDivFwd f = make_ks_div_fwd(c, nullptr, acc, Vp, V, out, n, l, none, nullptr, 0);
    OpKsDivFwdT<true> s5{src, f.acc, f.Vp, f.V, f.out, nullptr, n, l, N, 0, none, f.dp, f.dq, f.small_mask};
    launch_ntt<false>(c, s5, st);
}

}  // namespace fhe
