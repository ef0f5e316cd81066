// k_relin_modup.cu -- the ModUp step (digit transforms and key inner
// products) with the schedule the autotuner picked for it.  Its kernels are
// instantiated here alone, in a translation unit of their own, so the build
// compiles them in parallel with the rest of the relinearisation.
#include "ops.cuh"

namespace fhe {

void launch_modup(const fhe_ctx* c, const OpModUpMac& op, cudaStream_t st, bool single_pass)
{
    if (c->ntt_variant_ks == 7 && modup_cluster_fits(c)) launch_modup_cluster(c, op, st);
    else launch_ntt<false>(c, op, st, single_pass);
}

}  // namespace fhe
