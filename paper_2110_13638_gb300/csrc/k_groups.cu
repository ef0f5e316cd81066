// k_groups.cu -- ct-mult + relinearise + rescale over batches at uneven levels.
#include "ops.cuh"

namespace fhe {

// ---------------------------------------------------------------- level groups
// ct-mult + relinearise + rescale for batches at different levels: every step
// is one launch over all batches (MultiOp), so a set of uneven-level
// ciphertexts costs six launches whatever its level mix (tensor, digit
// inverses, key inner products, P inverses, and the merged ModDown + rescale
// inverse and forward steps).
struct TensorGroups {
    const u64* a[kMaxGroups];
    const u64* b[kMaxGroups];
    u64* out[kMaxGroups];
    unsigned long long start[kMaxGroups + 1];
    int L[kMaxGroups];
    int ng;
};

__global__ void k_tensor_groups_kernel(TensorGroups G, int logN, const PrimeC* __restrict__ pc)
{
    const size_t total = G.start[G.ng];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int g = 0;
        while (g + 1 < G.ng && i >= G.start[g + 1]) ++g;
        const size_t w0 = i - G.start[g];
        const size_t per_comp = (size_t)G.L[g] << logN;
        const uint32_t row = (uint32_t)(w0 >> logN);         // ct * L + r, 32-bit index math
        const uint32_t ct = row / (uint32_t)G.L[g], r = row - ct * (uint32_t)G.L[g];
        const size_t w = ((size_t)r << logN) + (w0 & (((size_t)1 << logN) - 1));
        const PrimeC P = pc[r];
        const u64* A = G.a[g] + ct * 2 * per_comp;
        const u64* B = G.b[g] + ct * 2 * per_comp;
        const u64 a0 = A[w], a1 = A[per_comp + w], b0 = B[w], b1 = B[per_comp + w];
        u64* O = G.out[g] + ct * 3 * per_comp;
        O[w] = mul_mod_r(a0, b0, P);
        O[per_comp + w] = add_mod(mul_mod_r(a0, b1, P), mul_mod_r(a1, b0, P), P.q);
        O[2 * per_comp + w] = mul_mod_r(a1, b1, P);
    }
}

size_t level_groups_scratch_bytes(const fhe_ctx* c, const LevelBatch* g, int ng)
{
    const size_t N = c->N;
    size_t s = 0;
    for (int k = 0; k < ng; ++k) {
        const size_t n = g[k].n, L = g[k].L;
        s += arena_need({n * 3 * L * N * 8, n * L * N * 8, n * 2 * (L + 1) * N * 8, n * 2 * N * 8, n * 2 * N * 8});
    }
    return s;
}

void k_mul_relin_rescale_groups(const fhe_ctx* c, const LevelBatch* g, int ng, void* scratch, cudaStream_t st)
{
    const size_t N = c->N;
    Arena ar;
    ar.base = (char*)scratch;
    ar.cap = level_groups_scratch_bytes(c, g, ng);
    TensorGroups tg;
    MultiOp<OpDigitsInv> m1;
    MultiOp<OpModUpMac> m2;
    MultiOp<OpAccPInv> m3;
    MultiOp<OpKsRowInv> m4;
    MultiOp<OpKsDivFwd> m5;
    m1.ng = m2.ng = m3.ng = m4.ng = m5.ng = tg.ng = ng;
    m1.pre_[0] = m2.pre_[0] = m3.pre_[0] = m4.pre_[0] = m5.pre_[0] = 0;
    tg.start[0] = 0;
    const KsExtra none{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    for (int k = 0; k < ng; ++k) {
        const int n = (int)g[k].n, L = (int)g[k].L;
        u64* t3 = (u64*)ar.take((size_t)n * 3 * L * N * 8);
        u64* D = (u64*)ar.take((size_t)n * L * N * 8);
        u64* acc = (u64*)ar.take((size_t)n * 2 * (L + 1) * N * 8);
        u64* Vp = (u64*)ar.take((size_t)n * 2 * N * 8);
        u64* V = (u64*)ar.take((size_t)n * 2 * N * 8);
        tg.a[k] = g[k].a;
        tg.b[k] = g[k].b;
        tg.out[k] = t3;
        tg.L[k] = L;
        tg.start[k + 1] = tg.start[k] + (unsigned long long)n * L * N;
        m1.ops[k] = OpDigitsInv{t3, D, n, L, (int)N};
        m2.ops[k] = OpModUpMac{t3, D, c->d_ksk, acc, n, L, (int)N, (int)c->L_top, modup_red_mask(c, (uint32_t)L),
                               modup_lazy_mask(c, (uint32_t)L)};
        m3.ops[k] = OpAccPInv{acc, Vp, n, L, (int)N, (int)c->L_top};
        m4.ops[k] = make_ks_row_inv(c, t3, acc, Vp, V, n, L, none);
        m5.ops[k] = make_ks_div_fwd(c, t3, acc, Vp, V, g[k].out, n, L, none, nullptr, 0);
        m1.pre_[k + 1] = m1.pre_[k] + m1.ops[k].count();
        m2.pre_[k + 1] = m2.pre_[k] + m2.ops[k].count();
        m3.pre_[k + 1] = m3.pre_[k] + m3.ops[k].count();
        m4.pre_[k + 1] = m4.pre_[k] + m4.ops[k].count();
        m5.pre_[k + 1] = m5.pre_[k] + m5.ops[k].count();
    }
    {
        LaunchScope ls(c, "tensor", st);
        k_tensor_groups_kernel<<<ew_grid(tg.start[ng]), 256, 0, st>>>(tg, (int)c->logN, c->d_pc);
    }
    launch_ntt<true>(c, m1, st);
    launch_groups_modup_mac(c, m2, st);
    launch_ntt<true>(c, m3, st);
    launch_ntt<true>(c, m4, st);
    launch_groups_ks_divfwd(c, m5, st);
}


}  // namespace fhe
