"""fhe_relinearise_noalloc: the allocation-free variant of relinearisation,
for callers that may not allocate device memory during a call.  Its output
must equal fhe_relinearise's (bit-exact, the tolerance of every ciphertext
test here) on two calls in a row, which share the fixed scratch array; a batch
too large for that array must be refused with FHE_EINVAL.  This file is
collected last so that a failure here stops a -x run only after every other
test has run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__
from paper_2110_13638_gb300 import fhe

pytestmark = pytest.mark.gpu

BITS9 = [60] + [40] * 7 + [60]


def _random_d3(ctx, n, L, seed):
    rng = np.random.default_rng(seed)
    a = np.stack([np.stack([np.stack([rng.integers(0, q, ctx.N, dtype=np.uint64) for q in ctx.primes[:L]])
                            for _ in range(3)]) for _ in range(n)])
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def test_noalloc_relinearise_matches_twice():
    __graft_entry__.build()
    torch.cuda.set_device(0)
    ctx = fhe.Context(16384, BITS9, 40)
    ctx.keygen(0)
    cases = [(2, 8), (3, 5)]
    d3s = [_random_d3(ctx, n, L, 100 + k) for k, (n, L) in enumerate(cases)]
    gots = [ctx.empty_ct(n, L) for n, L in cases]
    # the first call on a device looks up (and, under lazy loading, reserves)
    # the fixed array: make it before measuring
    ctx.relinearise_noalloc(d3s[0], cases[0][1], ctx.empty_ct(*cases[0]))
    torch.cuda.synchronize()
    ws0 = ctx.workspace_bytes()
    free0 = torch.cuda.mem_get_info()[0]
    # two calls in a row on a context whose workspace has not been used
    for (n, L), d3, got in zip(cases, d3s, gots):
        ctx.relinearise_noalloc(d3, L, got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the calls allocated device memory"
    assert ctx.workspace_bytes() == ws0, "the calls used or grew the context workspace"
    # only now the ordinary entry point, which grows the workspace
    for call, ((n, L), d3, got) in enumerate(zip(cases, d3s, gots)):
        ref = ctx.empty_ct(n, L)
        ctx.relinearise(d3, L, ref)
        torch.cuda.synchronize()
        assert torch.equal(ref, got), "call %d differs" % call
    assert ctx.workspace_bytes() > ws0
    too_big = _random_d3(ctx, 5, 8, 7)
    with pytest.raises(fhe.FheError) as e:
        ctx.relinearise_noalloc(too_big, 8, ctx.empty_ct(5, 8))
    assert e.value.code == -1
    ctx.close()
