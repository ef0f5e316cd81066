"""Edge cases on the GPU: empty batches, the smallest ring, degenerate layers
(an output row without terms, zero coefficients), ragged tile counts, and
the refusals the header promises.  Every result is compared with the oracle
or, for empty calls, checked to launch nothing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__
from oracle import ckks
from paper_2110_13638_gb300 import fhe, workloads as W

pytestmark = pytest.mark.gpu

BITS5 = [60, 40, 40, 40, 60]


@pytest.fixture(scope="module")
def small():
    __graft_entry__.build()
    torch.cuda.set_device(0)
    g = fhe.Context(16, BITS5, 40)
    g.keygen(0)
    o = ckks.Context(16, BITS5, 40)
    o.keygen(0)
    yield g, o
    g.close()


def test_empty_batches_launch_nothing(small):
    g, _ = small
    L = g.L_top
    z0 = torch.empty((0, 8), dtype=torch.float64, device="cuda")
    ct0 = g.empty_ct(0, L)
    g.galois_keygen([1])
    torch.cuda.synchronize()
    before = fhe.launch_count()
    g.encode(z0, L, g.delta, g.empty_pt(0, L))
    g.encrypt(g.empty_pt(0, L), 0, ct0)
    g.encode_encrypt(z0, g.delta, 0, ct0)
    g.decrypt(ct0, L, torch.empty((0, 16), dtype=torch.int64, device="cuda"))
    g.decode(torch.empty((0, 16), dtype=torch.int64, device="cuda"), g.delta, z0)
    g.tensor(ct0, ct0, L, g.empty_ct(0, L, comps=3))
    g.relinearise(g.empty_ct(0, L, comps=3), L, ct0)
    g.rescale(ct0, 2, L, g.empty_ct(0, L - 1))
    g.add(ct0, ct0, L, ct0)
    g.rotate(ct0, L, 1, ct0)
    torch.cuda.synchronize()
    assert fhe.launch_count() == before


def _parity(g, o, graph, x):
    L = g.L_top
    ct = g.empty_ct(x.shape[0], L)
    g.encode_encrypt(torch.tensor(x, device="cuda"), g.delta, 0, ct)
    G = fhe.Graph(graph)
    n_out, L_out = G.outputs(g)
    out = g.empty_ct(n_out, L_out)
    meta = G.eval(g, [ct], out)
    got = out.clone()
    g.ct_convert(out, L_out, True, got)
    torch.cuda.synchronize()
    got = fhe.raw_u64(got)
    cts = [o.encrypt(o.encode(x[i]), i) for i in range(x.shape[0])]
    (node, ys), = ckks.eval_graph(o, graph, W.input_nodes(graph), [cts]).items()
    for k, y in enumerate(ys):
        assert np.array_equal(got[k], y.c), k
        assert meta[k][1] == y.scale
    G.close()
    return got


def test_smallest_ring_degenerate_layer(small):
    """N = 16 (8 slots): a dense layer with 7 outputs (ragged against the
    6-row MAC tile) where one output row has no terms (bias only), then a
    polynomial with a zero middle coefficient."""
    g, o = small
    rng = np.random.default_rng(5)
    Wm = rng.normal(0, 0.5, size=(7, 3))
    rp, ci, wv = W.dense_csr(Wm)
    # empty row 4: drop its three terms
    keep = [e for e in range(len(ci)) if not (rp[4] <= e < rp[5])]
    ci, wv = ci[keep], wv[keep]
    rp = np.array([0, 3, 6, 9, 12, 12, 15, 18], dtype=np.uint32)
    lin = W._linear(rp, ci, wv, rng.normal(0, 0.1, size=7))
    graph = W.chain_graph(3, [lin, {"kind": "poly", "coeffs": [0.2, 0.0, 0.3]}])
    x = rng.uniform(-1, 1, size=(3, 8))
    _parity(g, o, graph, x)


def test_refusals(small):
    g, _ = small
    L = g.L_top
    ct = g.empty_ct(1, L)
    with pytest.raises(fhe.FheError) as e:                       # a linear node needs two primes
        G = fhe.Graph(W.chain_graph(1, [W._linear(*W.dense_csr(np.ones((1, 1))), np.zeros(1))] * 6))
        n, Lo = G.outputs(g)
    assert e.value.code == -3
    with pytest.raises(fhe.FheError):                            # too many samples for one batch
        G = fhe.Graph(W.chain_graph(1, [W._linear(*W.dense_csr(np.ones((1, 1))), np.zeros(1))]))
        G.eval_batch(g, [(torch.zeros((1, 9), dtype=torch.float64, device="cuda"),
                          torch.zeros((1, 9), dtype=torch.float64, device="cuda"))], 0)
    with pytest.raises(ValueError):
        fhe.Graph(W.chain_graph(1, [{"kind": "poly", "coeffs": [0.1] * 33}]))
    with pytest.raises(fhe.FheError):                            # a relu range must be positive
        fhe.Graph(W.chain_graph(1, [{"kind": "relu", "q": -1.0}]))
    with pytest.raises(fhe.FheError):                            # rotation nodes are evaluated per group
        G = fhe.Graph({"nodes": [{"kind": "input", "n": 1}, {"kind": "rotate"}, {"kind": "output"}],
                       "edges": [(0, 1), (1, 2)]})
        G.eval(g, [ct], g.empty_ct(1, L))


def test_scale_mismatch_is_refused(small):
    """An ADD node over inputs whose nominal scales differ by more than 2^-40
    (x at scale s and x^2 at s^2 / q_{L-1}) is refused with FHE_ESCALE before
    anything is launched."""
    g, _ = small
    graph = {"nodes": [{"kind": "input", "n": 1}, {"kind": "square"}, {"kind": "add"}, {"kind": "output"}],
             "edges": [(0, 1), (1, 2), (0, 2), (2, 3)]}
    G = fhe.Graph(graph)
    before = fhe.launch_count()
    with pytest.raises(fhe.FheError) as e:
        G.outputs(g)
    assert e.value.code == -4
    with pytest.raises(fhe.FheError) as e:
        G.eval(g, [g.empty_ct(1, g.L_top)], g.empty_ct(1, g.L_top - 1))
    assert e.value.code == -4
    assert fhe.launch_count() == before
    G.close()


def test_tensor_core_wait_that_runs_out_reports_timeout():
    """A tensor-core layer MAC whose matrix products never arrive (the test
    hook withholds them, so nothing is in flight on the tensor cores): every
    block's bounded wait runs out, the blocks free their tensor memory and
    return, and the context reports FHE_ETIMEOUT.  The context stays usable:
    the next evaluation gives the same words as before."""
    __graft_entry__.build()
    torch.cuda.set_device(0)
    N, bits = 256, [60] + [40] * 7 + [60]
    ctx = fhe.Context(N, bits, 40)
    ctx.keygen(0)
    rng = np.random.Generator(np.random.PCG64(31))
    Wm = rng.normal(0.0, 0.2, size=(16, 40))          # dense 40 -> 16: on the tensor cores
    graph = W.chain_graph(40, [W._linear(*W.dense_csr(Wm), np.zeros(16)), {"kind": "square"}])
    x = rng.uniform(-1.0, 1.0, size=(40, N // 2))
    ct = ctx.empty_ct(40, ctx.L_top)
    ctx.encode_encrypt(torch.tensor(x, device="cuda"), ctx.delta, 0, ct)
    G = fhe.Graph(graph)
    n_out, L_out = G.outputs(ctx)
    ref = ctx.empty_ct(n_out, L_out)
    G.eval(ctx, [ct], ref)
    ctx.sync()
    assert fhe.device_faults() == 0
    ctx.inject_fault(1)
    bad = ctx.empty_ct(n_out, L_out)
    with pytest.raises(fhe.FheError) as e:
        G.eval(ctx, [ct], bad)
        ctx.sync()                                     # reports it if the call returned first
    assert e.value.code == -6
    ctx.sync()                                         # the report cleared the status
    assert fhe.device_faults() == 1                    # the device-wide flag saw it too
    again = ctx.empty_ct(n_out, L_out)
    G.eval(ctx, [ct], again)
    ctx.sync()
    assert torch.equal(again, ref)
    assert fhe.device_faults() == 0
    G.close()
    ctx.close()


def test_binding_refuses_wrong_buffers(small):
    """The binding checks shape, dtype, contiguity and device before any
    pointer reaches the library (a short output would be written past)."""
    g, _ = small
    L = g.L_top
    d3 = torch.zeros((2, 3, L, g.N), dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        g.relinearise(d3, L, g.empty_ct(1, L))               # too few output ciphertexts
    with pytest.raises(ValueError):
        g.relinearise(d3, L, g.empty_ct(2, L - 1))           # wrong level
    with pytest.raises(ValueError):
        g.relinearise(d3.to(torch.float64), L, g.empty_ct(2, L))
    with pytest.raises(ValueError):
        g.relinearise(d3, L, torch.zeros((2, L, 2, g.N), dtype=torch.int64, device="cuda").transpose(1, 2))
    with pytest.raises(ValueError):
        g.relinearise(d3.cpu(), L, g.empty_ct(2, L))
    with pytest.raises(ValueError):
        g.rescale(g.empty_ct(2, L), 2, L, g.empty_ct(2, L))
