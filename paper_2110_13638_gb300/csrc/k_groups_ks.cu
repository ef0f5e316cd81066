// k_groups_ks.cu -- grouped launch of the key-switching inner product
// (digit transforms + key products over batches at uneven levels).
#include "ops.cuh"

namespace fhe {

void launch_groups_modup_mac(const fhe_ctx* c, const MultiOp<OpModUpMac>& m, cudaStream_t st)
{
    launch_ntt<false>(c, m, st);
}

}  // namespace fhe
