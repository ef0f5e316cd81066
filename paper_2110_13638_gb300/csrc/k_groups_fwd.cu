// k_groups_fwd.cu -- grouped launches of ModDown and the rescale's forward
// transforms over batches at uneven levels.
#include "ops.cuh"

namespace fhe {

void launch_groups_moddown(const fhe_ctx* c, const MultiOp<OpModDown>& m, cudaStream_t st)
{
    launch_ntt<false>(c, m, st);
}

void launch_groups_divfwd(const fhe_ctx* c, const MultiOp<OpDivFwd>& m, cudaStream_t st)
{
    launch_ntt<false>(c, m, st);
}

}  // namespace fhe
