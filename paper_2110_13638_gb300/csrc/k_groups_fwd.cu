// k_groups_fwd.cu -- grouped launch of the merged ModDown + rescale forward
// transforms over batches at uneven levels.
#include "ops.cuh"

namespace fhe {

void launch_groups_ks_divfwd(const fhe_ctx* c, const MultiOp<OpKsDivFwd>& m, cudaStream_t st)
{
    launch_ntt<false>(c, m, st);
}

}  // namespace fhe
