"""Full-size workloads on the GPU, in the launch configuration bench.py times.

- The encrypted CNN's first two blocks (conv 5x5x5 stride 2 over 784 input
  ciphertexts, then the degree-3 sigmoid fit over 720 ciphertexts) at
  N = 16384, L = 8: sampled outputs are recomputed one by one by the oracle
  (each needs only its 25 input encryptions) and must be bit-exact.
- The rest of the CNN at full size: each later block is recomputed by the
  oracle from the device's own inputs to that block (sampled rows of the
  720 -> 100 tensor-core layer at L = 5 across its row tiles, two outputs of
  the second sigmoid fit at L = 4, all ten outputs of the 100 -> 10 layer)
  and must be bit-exact.
- The whole CNN and the whole yield MLP: decrypted outputs within 1e-4 of the
  FP64 plaintext forward pass with the same polynomial activations.
- The yield MLP block by block the same way, and the uneven-level batching
  workload (4096 pairs, one persistent launch in a CUDA graph) with one
  sampled pair per level recomputed by the oracle.
- The dense layers give the same words on the tensor cores as on the integer
  pipes.
- Every NTT schedule the autotuner can pick gives bit-exact results."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__
from oracle import ckks
from paper_2110_13638_gb300 import fhe, workloads as W

pytestmark = pytest.mark.gpu

BITS9 = [60] + [40] * 7 + [60]


@pytest.fixture(scope="module")
def ctx():
    __graft_entry__.build()
    torch.cuda.set_device(0)
    c = fhe.Context(16384, BITS9, 40)
    c.keygen(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def octx():
    o = ckks.Context(16384, BITS9, 40)
    o.keygen(0)
    return o


def encrypt_all(ctx, x, first=0):
    n = x.shape[0]
    pt = ctx.empty_pt(n, ctx.L_top)
    ctx.encode(torch.tensor(x, device="cuda"), ctx.L_top, ctx.delta, pt)
    ct = ctx.empty_ct(n, ctx.L_top)
    ctx.encrypt(pt, first, ct)
    return ct


def run_graph(ctx, graph, ct):
    G = fhe.Graph(graph)
    n_out, L_out = G.outputs(ctx)
    out = ctx.empty_ct(n_out, L_out)
    meta = G.eval(ctx, [ct], out)
    return out, meta, L_out


def test_cnn_first_blocks_sampled_bit_exact(ctx, octx):
    g, x = W.cfg1()
    head = W.chain_graph(784, [g["nodes"][1], g["nodes"][2]])      # conv, sigmoid fit
    ct = encrypt_all(ctx, x)
    out, meta, L_out = run_graph(ctx, head, ct)
    assert out.shape[0] == 720 and L_out == 5
    rows = ckks.csr_rows(g["nodes"][1])
    for k in (0, 363, 719):
        idx, ws = rows[k]
        xs = [octx.encrypt(octx.encode(x[int(i)]), int(i)) for i in idx]
        y = octx.linear(xs, [(np.arange(len(idx)), ws)], [g["nodes"][1]["bias"][k]])[0]
        y = octx.poly3(y, g["nodes"][2]["coeffs"])
        got = out[k:k + 1].clone()
        ctx.ct_convert(got, L_out, True, got)
        torch.cuda.synchronize()
        assert np.array_equal(fhe.raw_u64(got)[0], y.c), k
        assert meta[k][1] == y.scale


def _coeff(ctx, t, level):
    c = t.clone()
    ctx.ct_convert(c, level, True, c)
    torch.cuda.synchronize()
    return fhe.raw_u64(c)


def test_cnn_tail_sampled_bit_exact(ctx, octx):
    """Each block after the first sigmoid fit, recomputed by the oracle from
    the ciphertexts the device fed it (the device's evaluation is
    deterministic, so the prefix runs reproduce the inputs of the full run)."""
    g, x = W.cfg1()
    nodes = g["nodes"]
    ct = encrypt_all(ctx, x)
    runs = {}
    for k in (2, 3, 4, 5):                   # the first k blocks after the input
        out, meta, L = run_graph(ctx, W.chain_graph(784, nodes[1:1 + k]), ct)
        runs[k] = (_coeff(ctx, out, L), meta, L)
        del out
    X5, m5, L5 = runs[2]                     # 720 ciphertexts at L = 5
    Y4, m4, L4 = runs[3]                     # 100 at L = 4 (dense 720 -> 100)
    Y2, m2, L2 = runs[4]                     # 100 at L = 2 (second sigmoid fit)
    Y1, m1, L1 = runs[5]                     # 10 at L = 1 (dense 100 -> 10)
    assert (L5, L4, L2, L1) == (5, 4, 2, 1)
    # dense 720 -> 100 on the tensor cores: rows at both ends of the 48-row
    # (five-limb) and 32-row (eight-limb) tiles
    xs = [ckks.Ciphertext(X5[i], L5, m5[i][1]) for i in range(720)]
    rows = ckks.csr_rows(nodes[3])
    for k in (0, 31, 47, 48, 99):
        y = octx.linear(xs, [rows[k]], [nodes[3]["bias"][k]])[0]
        assert np.array_equal(Y4[k], y.c), k
        assert m4[k][1] == y.scale
    del xs, X5
    # second sigmoid fit
    for k in (0, 77):
        y = octx.poly3(ckks.Ciphertext(Y4[k], L4, m4[k][1]), nodes[4]["coeffs"])
        assert np.array_equal(Y2[k], y.c), k
        assert m2[k][1] == y.scale
    # dense 100 -> 10 on the integer MAC, every output
    xs = [ckks.Ciphertext(Y2[i], L2, m2[i][1]) for i in range(100)]
    ys = octx.linear(xs, ckks.csr_rows(nodes[5]), nodes[5]["bias"])
    for k in range(10):
        assert np.array_equal(Y1[k], ys[k].c), k
        assert m1[k][1] == ys[k].scale


def _decrypted(ctx, out, meta, L_out):
    n = out.shape[0]
    m = torch.empty((n, ctx.N), dtype=torch.int64, device="cuda")
    ctx.decrypt(out, L_out, m)
    z = torch.empty((n, ctx.N // 2), dtype=torch.float64, device="cuda")
    ctx.decode(m, meta[0][1], z)
    return z.cpu().numpy()


@pytest.mark.parametrize("builder", [W.cfg1, W.cfg2, W.cnn_relu])
def test_full_network_matches_fp64(ctx, builder):
    g, x = builder()
    ct = encrypt_all(ctx, x, first=5000)
    out, meta, L_out = run_graph(ctx, g, ct)
    assert L_out == 1
    z = _decrypted(ctx, out, meta, L_out)
    ref = ckks.forward_fp64(g, W.input_nodes(g), [x])
    (node, r), = ref.items()
    err = float(np.max(np.abs(z - r)))
    assert err < 1e-4, (err, float(np.max(np.abs(r))))


@pytest.mark.parametrize("builder", [W.cfg1, W.cfg2])
def test_tensor_core_mac_equals_integer_mac(ctx, builder, monkeypatch):
    """The dense layers on the tensor cores give the same words as on the
    integer pipes, through the whole network.  CNN: 720 -> 100 at L = 5.
    MLP: 64 -> 128 at L = 8 and 128 -> 32 at L = 5."""
    g, x = builder()
    ct = encrypt_all(ctx, x, first=7000)
    monkeypatch.setenv("FHE_MAC_TC", "0")
    ref, _, _ = run_graph(ctx, g, ct)
    monkeypatch.setenv("FHE_MAC_TC", "1")
    got, _, _ = run_graph(ctx, g, ct)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert fhe.device_faults() == 0


def test_dense_square_full_matches_fp64():
    __graft_entry__.build()
    c = fhe.Context(8192, [60, 40, 40, 60], 40)
    c.keygen(0)
    g, x = W.cfg0()
    ct = encrypt_all(c, x)
    out, meta, L_out = run_graph(c, g, ct)
    z = _decrypted(c, out, meta, L_out)
    ref = ckks.forward_fp64(g, W.input_nodes(g), [x])
    (node, r), = ref.items()
    assert float(np.max(np.abs(z - r))) < 1e-4
    c.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8])
def test_every_ntt_schedule_bit_exact(octx, variant):
    __graft_entry__.build()
    os.environ["FHE_NTT_VARIANT"] = str(variant)
    try:
        c = fhe.Context(16384, BITS9, 40)
    finally:
        del os.environ["FHE_NTT_VARIANT"]
    assert c.ntt_variant == variant
    c.keygen(0)
    rng = np.random.default_rng(variant)
    L = 6
    A = np.stack([np.stack([rng.integers(0, q, 16384, dtype=np.uint64) for q in octx.q[:L]]) for _ in range(2)])
    B = np.stack([np.stack([rng.integers(0, q, 16384, dtype=np.uint64) for q in octx.q[:L]]) for _ in range(2)])
    ta = torch.from_numpy(A[None].view(np.int64).copy()).cuda()
    tb = torch.from_numpy(B[None].view(np.int64).copy()).cuda()
    c.ct_convert(ta, L, False, ta)
    c.ct_convert(tb, L, False, tb)
    out = c.empty_ct(1, L - 1)
    c.mul_relin_rescale(ta, tb, L, out)
    c.ct_convert(out, L - 1, True, out)
    torch.cuda.synchronize()
    want = octx.rescale(octx.relinearise(octx.tensor(ckks.Ciphertext(A, L, 1.0), ckks.Ciphertext(B, L, 1.0)))).c
    assert np.array_equal(fhe.raw_u64(out)[0], want)
    c.close()


def test_mlp_blocks_sampled_bit_exact(ctx, octx):
    """The yield MLP (config 2) at full size, block by block: each block is
    recomputed by the oracle from the ciphertexts the device fed it (rows at both ends
    of the 64 -> 128 and 128 -> 32 tensor-core layers' tiles, outputs of both
    sigmoid fits, the 32 -> 1 integer-MAC layer), bit-exact with equal
    nominal scales."""
    g, x = W.cfg2()
    nodes = g["nodes"]
    ct = encrypt_all(ctx, x, first=900)
    X = _coeff(ctx, ct, ctx.L_top)
    runs = {}
    for k in (1, 2, 3, 4, 5):
        out, meta, L = run_graph(ctx, W.chain_graph(64, nodes[1:1 + k]), ct)
        runs[k] = (_coeff(ctx, out, L), meta, L)
        del out
    (Y1, m1, L1), (Y2, m2, L2), (Y3, m3, L3), (Y4, m4, L4), (Y5, m5, L5) = (runs[k] for k in (1, 2, 3, 4, 5))
    assert (L1, L2, L3, L4, L5) == (7, 5, 4, 2, 1)
    xs = [ckks.Ciphertext(X[i], ctx.L_top, ctx.delta) for i in range(64)]
    rows = ckks.csr_rows(nodes[1])
    for k in (0, 31, 47, 48, 127):
        y = octx.linear(xs, [rows[k]], [nodes[1]["bias"][k]])[0]
        assert np.array_equal(Y1[k], y.c), k
        assert m1[k][1] == y.scale
    for k in (0, 100):
        y = octx.poly3(ckks.Ciphertext(Y1[k], L1, m1[k][1]), nodes[2]["coeffs"])
        assert np.array_equal(Y2[k], y.c), k
        assert m2[k][1] == y.scale
    xs = [ckks.Ciphertext(Y2[i], L2, m2[i][1]) for i in range(128)]
    rows = ckks.csr_rows(nodes[3])
    for k in (0, 31):
        y = octx.linear(xs, [rows[k]], [nodes[3]["bias"][k]])[0]
        assert np.array_equal(Y3[k], y.c), k
    y = octx.poly3(ckks.Ciphertext(Y3[5], L3, m3[5][1]), nodes[4]["coeffs"])
    assert np.array_equal(Y4[5], y.c)
    xs = [ckks.Ciphertext(Y4[i], L4, m4[i][1]) for i in range(32)]
    y = octx.linear(xs, ckks.csr_rows(nodes[5]), nodes[5]["bias"])[0]
    assert np.array_equal(Y5[0], y.c)
    assert m5[0][1] == y.scale


def test_uneven_level_batch_full_size_sampled_bit_exact(ctx, octx):
    """The batching workload at full size in the launch configuration the
    bench times: 4096 ciphertext pairs at levels 1 + U{1..7} (seed 3) in one
    persistent launch captured in a CUDA graph; one sampled pair per level is
    recomputed by the oracle (tensor, relinearise, rescale), bit-exact."""
    levels = 1 + np.random.Generator(np.random.PCG64(3)).integers(1, 8, size=4096)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    batches = []
    for L in range(2, 9):
        n = int((levels == L).sum())
        def rnd():
            t = torch.empty((n, 2, L, 16384), dtype=torch.int64, device="cuda")
            for r in range(L):
                t[:, :, r, :] = torch.randint(0, ctx.primes[r], (n, 2, 16384), device="cuda", generator=gen)
            return t
        batches.append((rnd(), rnd(), ctx.empty_ct(n, L - 1), L))
    ctx.mul_relin_rescale_levels(batches)           # sizes the workspace
    ctx.sync()
    for b in batches:
        b[2].zero_()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            ctx.mul_relin_rescale_levels(batches)
    torch.cuda.current_stream().wait_stream(s)
    graph.replay()
    ctx.sync()
    rng = np.random.default_rng(12)
    for a, b, out, L in batches:
        k = int(rng.integers(0, a.shape[0]))
        A = _coeff(ctx, a[k:k + 1].clone(), L)[0]
        B = _coeff(ctx, b[k:k + 1].clone(), L)[0]
        got = _coeff(ctx, out[k:k + 1].clone(), L - 1)[0]
        want = octx.rescale(octx.relinearise(octx.tensor(ckks.Ciphertext(A, L, 1.0),
                                                         ckks.Ciphertext(B, L, 1.0)))).c
        assert np.array_equal(got, want), (L, k)
