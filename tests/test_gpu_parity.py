"""GPU parity: every step of the path through the C ABI against the CPU oracle.

Ciphertext residues must be bit-exact (compared in coefficient form, so the
device's internal NTT order and root choice do not matter).  Encoded
coefficients may differ by 1 only where the oracle's unrounded value lies
within 1e-6 of a rounding boundary.  Decoded slots are compared within the
FP64 bound derived in the test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__
from oracle import ckks
from paper_2110_13638_gb300 import fhe, workloads as W

pytestmark = pytest.mark.gpu

BITS5 = [60, 40, 40, 40, 40, 60]
BITS9 = [60] + [40] * 7 + [60]


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


_CTX = {}


def pair(N, bits, seed=0):
    key = (N, tuple(bits), seed)
    if key not in _CTX:
        g = fhe.Context(N, bits, 40)
        g.keygen(seed)
        o = ckks.Context(N, bits, 40)
        o.keygen(seed)
        _CTX[key] = (g, o)
    return _CTX[key]


def upload(ctx, arrs, level):
    """oracle coefficient-form arrays [k][L][N] -> device NTT form [n][k][L][N]"""
    a = np.stack(arrs).astype(np.uint64)
    t = torch.from_numpy(a.view(np.int64).copy()).cuda()
    comps = a.shape[1]
    flat = t.view(-1, level, ctx.N)
    ctx.ntt(flat, level, True)
    return t


def download(ctx, t, level):
    """device NTT form [n][k][L][N] -> coefficient form uint64"""
    c = t.clone()
    ctx.ntt(c.view(-1, level, ctx.N), level, False)
    torch.cuda.synchronize()
    return fhe.raw_u64(c)


def rand_ct(o, L, rng, comps=2):
    return np.stack([np.stack([rng.integers(0, q, o.N, dtype=np.uint64) for q in o.q[:L]]) for _ in range(comps)])


# ---------------------------------------------------------------- keys
@pytest.mark.parametrize("N,bits", [(16, BITS5), (1024, BITS5), (16384, BITS9)])
def test_secret_key_matches_oracle(N, bits):
    g, o = pair(N, bits)
    s = torch.empty((g.L_top + 1, N), dtype=torch.int64, device="cuda")
    g.export_secret(s)
    got = download(g, s.view(1, g.L_top + 1, N), g.L_top + 1)[0]
    for r in range(g.L_top + 1):
        assert np.array_equal(got[r], o.s[r]), r


# ---------------------------------------------------------------- NTT / ring
@pytest.mark.parametrize("N,bits,n", [(16, BITS5, 3), (256, BITS5, 5), (4096, BITS5, 2), (16384, BITS9, 2)])
def test_ntt_roundtrip_and_tensor(N, bits, n):
    g, o = pair(N, bits)
    rng = np.random.default_rng(N + n)
    L = g.L_top
    A = [rand_ct(o, L, rng) for _ in range(n)]
    B = [rand_ct(o, L, rng) for _ in range(n)]
    ta, tb = upload(g, A, L), upload(g, B, L)
    assert np.array_equal(download(g, ta, L), np.stack(A))
    t3 = g.empty_ct(n, L, comps=3)
    g.tensor(ta, tb, L, t3)
    got = download(g, t3, L)
    for k in range(n):
        want = o.tensor(ckks.Ciphertext(A[k], L, 1.0), ckks.Ciphertext(B[k], L, 1.0)).c
        assert np.array_equal(got[k], want), k


# ---------------------------------------------------------------- encode
def _encode_check(g, o, z, got_res, L):
    """got_res: [n][L][N] coefficient-form residues of the device encoding"""
    for i in range(z.shape[0]):
        m, frac = o.encode(z[i], want_frac=True)
        for r in range(L):
            want = ckks.to_residue(m, o.q[r])
            bad = np.nonzero(got_res[i, r] != want)[0]
            for k in bad:
                d = (int(got_res[i, r, k]) - int(want[k])) % o.q[r]
                assert frac[k] < 1e-6 and d in (1, o.q[r] - 1), (i, r, k)


@pytest.mark.parametrize("N,bits,n", [(16, BITS5, 3), (1024, BITS5, 3), (8192, [60, 40, 40, 60], 2),
                                      (16384, BITS9, 2), (32768, [60, 40, 60], 2), (65536, [60, 40, 60], 1)])
def test_encode_matches_oracle(N, bits, n):
    g, o = pair(N, bits)
    rng = np.random.default_rng(7)
    z = rng.uniform(-1, 1, size=(n, N // 2))
    z[0, :] = rng.uniform(0, 1, N // 2) * 50.0          # larger magnitudes
    L = g.L_top
    pt = g.empty_pt(n, L)
    g.encode(torch.tensor(z, device="cuda"), L, g.delta, pt)
    got = download(g, pt.view(n, 1, L, N), L)[:, 0]
    _encode_check(g, o, z, got, L)


# ---------------------------------------------------------------- encrypt / decrypt / decode
@pytest.mark.parametrize("N,bits,n", [(16, BITS5, 2), (1024, BITS5, 3), (16384, BITS9, 2), (32768, [60, 40, 60], 2),
                                      (65536, [60, 40, 60], 1)])
def test_encrypt_decrypt_decode(N, bits, n):
    g, o = pair(N, bits)
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, size=(n, N // 2))
    L = g.L_top
    pt = g.empty_pt(n, L)
    g.encode(torch.tensor(z, device="cuda"), L, g.delta, pt)
    ct = g.empty_ct(n, L)
    first = 1000
    g.encrypt(pt, first, ct)
    got = download(g, ct, L)
    for i in range(n):
        want = o.encrypt(o.encode(z[i]), first + i)
        assert np.array_equal(got[i], want.c), i
    # decrypt the oracle's own ciphertexts on the device
    octs = [o.encrypt(o.encode(z[i]), 77 + i) for i in range(n)]
    t = upload(g, [c.c for c in octs], L)
    m = torch.empty((n, N), dtype=torch.int64, device="cuda")
    g.decrypt(t, L, m)
    md = m.cpu().numpy()
    for i in range(n):
        assert np.array_equal(md[i], o.decrypt(octs[i])), i
    zs = torch.empty((n, N // 2), dtype=torch.float64, device="cuda")
    g.decode(m, g.delta, zs)
    zd = zs.cpu().numpy()
    for i in range(n):
        ref = o.decode(md[i], g.delta)
        # FP64 FFT of integers < 2^62: error <= log2(N) * 2^-52 * sum|m| / scale
        bound = np.log2(N) * 2.0 ** -52 * np.abs(md[i]).astype(np.float64).sum() / g.delta + 1e-15
        assert np.max(np.abs(zd[i] - ref)) <= bound, i
        assert np.max(np.abs(zd[i] - z[i])) < 1e-5


# ---------------------------------------------------------------- key switching / rescale
@pytest.mark.parametrize("N,bits,L,n", [(16, BITS5, 1, 2), (64, BITS5, 3, 3), (1024, BITS5, 5, 2),
                                        (16384, BITS9, 8, 1)])
def test_relinearise_bit_exact(N, bits, L, n):
    g, o = pair(N, bits)
    rng = np.random.default_rng(L * 100 + n)
    D = [rand_ct(o, L, rng, comps=3) for _ in range(n)]
    t3 = upload(g, D, L)
    out = g.empty_ct(n, L)
    g.relinearise(t3, L, out)
    got = download(g, out, L)
    for k in range(n):
        assert np.array_equal(got[k], o.relinearise(ckks.Ciphertext(D[k], L, 1.0)).c), k


@pytest.mark.parametrize("N,bits,L,comps,n", [(16, BITS5, 2, 2, 3), (1024, BITS5, 5, 3, 2), (16384, BITS9, 8, 2, 2)])
def test_rescale_bit_exact(N, bits, L, comps, n):
    g, o = pair(N, bits)
    rng = np.random.default_rng(L + comps)
    X = [rand_ct(o, L, rng, comps=comps) for _ in range(n)]
    t = upload(g, X, L)
    out = g.empty_ct(n, L - 1, comps=comps)
    g.rescale(t, comps, L, out)
    got = download(g, out, L - 1)
    for k in range(n):
        assert np.array_equal(got[k], o.rescale(ckks.Ciphertext(X[k], L, 1.0)).c), k


@pytest.mark.parametrize("N,bits,L,n", [(1024, BITS5, 3, 3), (16384, BITS9, 8, 2), (16384, BITS9, 2, 1)])
def test_mul_relin_rescale_bit_exact(N, bits, L, n):
    g, o = pair(N, bits)
    rng = np.random.default_rng(5 * L + n)
    A = [rand_ct(o, L, rng) for _ in range(n)]
    B = [rand_ct(o, L, rng) for _ in range(n)]
    out = g.empty_ct(n, L - 1)
    g.mul_relin_rescale(upload(g, A, L), upload(g, B, L), L, out)
    got = download(g, out, L - 1)
    for k in range(n):
        a, b = ckks.Ciphertext(A[k], L, 1.0), ckks.Ciphertext(B[k], L, 1.0)
        assert np.array_equal(got[k], o.rescale(o.relinearise(o.tensor(a, b))).c), k


def test_const_ops_bit_exact():
    g, o = pair(256, BITS5)
    rng = np.random.default_rng(3)
    L = 3
    X = [rand_ct(o, L, rng) for _ in range(3)]
    C = [123456789012, -987654321, 0]
    t = upload(g, X, L)
    out = g.empty_ct(3, L)
    g.mul_const(t, C, L, out)
    g.add_const(out, [5, -7, 2 ** 50], L)
    got = download(g, out, L)
    for k in range(3):
        y = o.add_const(o.mul_const(ckks.Ciphertext(X[k], L, 1.0), C[k], 1.0), [5, -7, 2 ** 50][k])
        assert np.array_equal(got[k], y.c), k


def test_level_errors():
    g, _ = pair(16, BITS5)
    t = g.empty_ct(1, 1)
    with pytest.raises(fhe.FheError) as e:
        g.rescale(t, 2, 1, g.empty_ct(1, 1))
    assert e.value.code == -3
    with pytest.raises(fhe.FheError):
        g.encode(torch.zeros((1, 8), dtype=torch.float64, device="cuda"), 9, g.delta, g.empty_pt(1, 4))


# ---------------------------------------------------------------- graphs
def _graph_parity(g, o, graph, xs, first_ids):
    ins = W.input_nodes(graph)
    N = g.N
    L = g.L_top
    dev_in, orc_in = [], []
    for x, first in zip(xs, first_ids):
        n = x.shape[0]
        pt = g.empty_pt(n, L)
        g.encode(torch.tensor(x, device="cuda"), L, g.delta, pt)
        ct = g.empty_ct(n, L)
        g.encrypt(pt, first, ct)
        dev_in.append(ct)
        orc_in.append([o.encrypt(o.encode(x[i]), first + i) for i in range(n)])
    G = fhe.Graph(graph)
    n_out, L_out = G.outputs(g)
    out = g.empty_ct(n_out, L_out)
    meta = G.eval(g, dev_in, out)
    got = download(g, out, L_out)
    res = ckks.eval_graph(o, graph, ins, orc_in)
    want = [ct for node in sorted(res) for ct in res[node]]
    assert len(want) == n_out
    for k, y in enumerate(want):
        assert y.level == L_out and meta[k][0] == L_out
        assert meta[k][1] == y.scale
        assert np.array_equal(got[k], y.c), k
    m = torch.empty((n_out, N), dtype=torch.int64, device="cuda")
    g.decrypt(out, L_out, m)
    z = torch.empty((n_out, N // 2), dtype=torch.float64, device="cuda")
    g.decode(m, meta[0][1], z)
    ref = ckks.forward_fp64(graph, ins, xs)
    refs = np.concatenate([ref[node] for node in sorted(ref)], axis=0)
    return float(np.max(np.abs(z.cpu().numpy() - refs)))


def test_graph_mini_cnn_bit_exact():
    g, o = pair(1024, BITS9)
    graph, x = W.mini_cnn(n_slots=512)
    err = _graph_parity(g, o, graph, [x], [0])
    assert err < 1e-4


@pytest.mark.parametrize("N,bits", [(1024, BITS9), (256, [61, 40, 40, 61])])
def test_dense_layer_on_tensor_cores_bit_exact(N, bits):
    """A dense 150 -> 100 layer, then x^2.  With [60, 40 x 7, 60] every residue
    goes through the tensor-core MAC: the 40-bit ones with five limbs
    (three 48-row tiles, the last holding 4 rows), the 60-bit one with eight
    (four 32-row tiles); five 32-term chunks, the last one ragged.  With
    [61, 40, 40, 61] the 61-bit residue is left to the integer MAC.  Every
    output word must equal the oracle's, and no bounded wait may have given up."""
    g, o = pair(N, bits)
    rng = np.random.Generator(np.random.PCG64(29))
    Wm = rng.normal(0.0, 0.2, size=(100, 150))
    graph = W.chain_graph(150, [W._linear(*W.dense_csr(Wm), rng.normal(0.0, 0.1, 100)), {"kind": "square"}])
    x = rng.uniform(-1.0, 1.0, size=(150, N // 2))
    err = _graph_parity(g, o, graph, [x], [0])
    assert err < 1e-4
    assert fhe.device_faults() == 0


def test_graph_branches_bit_exact():
    g, o = pair(256, [60, 40, 40, 40, 60])
    graph, xs = W.branch_graph(n_slots=128)
    err = _graph_parity(g, o, graph, xs, [0, 100])
    assert err < 1e-4


def test_graph_cfg0_full_size_bit_exact():
    """Dense 8->4 then x^2 at N = 8192, [60,40,40,60], 4096 samples."""
    N, bits = 8192, [60, 40, 40, 60]
    g, o = pair(N, bits)
    graph, x = W.cfg0()
    err = _graph_parity(g, o, graph, [x], [0])
    assert err < 1e-4


@pytest.mark.parametrize("N,bits,L,steps", [(1024, BITS9, 8, [1, 3, -2, 100]), (1024, BITS9, 3, [5]),
                                             (16384, BITS9, 8, [1, 28])])
def test_rotation_bit_exact(N, bits, L, steps):
    """Galois automorphism in NTT form (index permutation) + key switch with
    the rotation key: bit-exact against the oracle's coefficient-form
    substitution and its rotation keys."""
    g, o = pair(N, bits)
    g.galois_keygen(steps)
    rng = np.random.default_rng(N + L)
    A = rand_ct(o, L, rng)
    ta = upload(g, [A], L)
    for r in steps:
        out = g.empty_ct(1, L)
        g.rotate(ta, L, r, out)
        want = o.rotate(ckks.Ciphertext(A, L, 1.0), r).c
        assert np.array_equal(download(g, out, L)[0], want), r
    # an encrypted vector decrypts rolled
    z = rng.uniform(-1, 1, size=(1, N // 2))
    ct = g.empty_ct(1, g.L_top)
    g.encode_encrypt(torch.tensor(z, device="cuda"), g.delta, 4242, ct)
    g.galois_keygen([7])
    rot = g.empty_ct(1, g.L_top)
    g.rotate(ct, g.L_top, 7, rot)
    m = torch.empty((1, N), dtype=torch.int64, device="cuda")
    g.decrypt(rot, g.L_top, m)
    zs = torch.empty((1, N // 2), dtype=torch.float64, device="cuda")
    g.decode(m, g.delta, zs)
    assert float(np.max(np.abs(zs.cpu().numpy()[0] - np.roll(z[0], -7)))) < 1e-6
    with pytest.raises(fhe.FheError):
        g.rotate(ct, g.L_top, 11, rot)          # no key for this step


def test_grouped_rotation_between_rings():
    """Groups of cost 2 and 4 get N = 8192 and N = 16384 from Alg.
    parameterise; the refresh widens the decoded slots to the larger ring.
    Group 1 bit-exact from the device's refreshed ciphertexts; decoded
    outputs within 1e-4 of FP64 on the samples that entered."""
    from paper_2110_13638_gb300 import groups
    graph, x = W.two_rings(n_slots=4096)
    net = groups.GroupedNetwork(graph, seed=0)
    assert [net.ctx[i].N for i in range(2)] == [8192, 16384]
    res = net.evaluate([torch.tensor(x, device="cuda")], first_ct_id=0)
    torch.cuda.synchronize()
    rot = [i for i, n in enumerate(graph["nodes"]) if n["kind"] == "rotate"][0]
    out_node = len(graph["nodes"]) - 1
    g1 = net.ctx[1]
    o1 = ckks.Context(16384, fhe.parameterise(4, 40, 1.5)[1], 40)
    o1.keygen(1)                                   # group g keys from seed + g
    fresh = download(g1, net.last_ingress[rot], g1.L_top)
    cts1 = [ckks.Ciphertext(fresh[k], g1.L_top, o1.delta) for k in range(fresh.shape[0])]
    seg1 = W.chain_graph(fresh.shape[0], graph["nodes"][rot + 1:out_node])
    (_, y1), = ckks.eval_graph(o1, seg1, [0], [cts1]).items()
    dev1, L1, _ = net.last_sinks[out_node]
    got1 = download(g1, dev1.contiguous(), L1)
    for k, y in enumerate(y1):
        assert np.array_equal(got1[k], y.c), k
    ref = ckks.forward_fp64(graph, W.input_nodes(graph), [x])
    assert float(np.max(np.abs(res[out_node].cpu().numpy()[:, :4096] - ref[out_node]))) < 1e-4
    net.close()


def test_masquerade_cnn_bit_exact_per_group():
    """Kernel masquerading on packed 8x8 images (8 per ciphertext at
    N = 1024): group 0 (packed conv through rotations + sigmoid) bit-exact
    against the oracle; the client re-packs the conv outputs one feature per
    ciphertext; group 1 (dense, sigmoid, dense) bit-exact from the device's
    refreshed ciphertexts; decoded outputs within 1e-4 of FP64."""
    from oracle import params
    from paper_2110_13638_gb300 import groups
    N = 1024
    graph, x = W.cnn_masquerade(4, N // 2)
    cost = params.autohe(graph, params.ingress_nodes(graph))[1]
    assert cost == [3, 4]
    pairs = [pair(N, params.parameterise(c)["coeff_modulus"], seed=gi) for gi, c in enumerate(cost)]
    net = groups.GroupedNetwork(graph, contexts={gi: p[0] for gi, p in enumerate(pairs)})
    res = net.evaluate([torch.tensor(x, device="cuda")], first_ct_id=0)
    torch.cuda.synchronize()
    rot, out_node = 3, 7
    g0, o0 = pairs[0]
    cts = [o0.encrypt(o0.encode(x[i]), i) for i in range(x.shape[0])]
    seg0 = {"nodes": [{"kind": "input", "n": x.shape[0]}, graph["nodes"][1], graph["nodes"][2], {"kind": "output"}],
            "edges": [(0, 1), (1, 2), (2, 3)]}
    (_, y0), = ckks.eval_graph(o0, seg0, [0], [cts]).items()
    dev0, L0, sc0 = net.last_sinks[rot]
    got0 = download(g0, dev0.contiguous(), L0)
    assert len(y0) == got0.shape[0] == 8
    for k, y in enumerate(y0):
        assert y.level == L0 and sc0[k] == y.scale
        assert np.array_equal(got0[k], y.c), k
    g1, o1 = pairs[1]
    fresh = download(g1, net.last_ingress[rot], g1.L_top)
    cts1 = [ckks.Ciphertext(fresh[k], g1.L_top, o1.delta) for k in range(fresh.shape[0])]
    seg1 = W.chain_graph(fresh.shape[0], graph["nodes"][4:7])
    (_, y1), = ckks.eval_graph(o1, seg1, [0], [cts1]).items()
    dev1, L1, _ = net.last_sinks[out_node]
    got1 = download(g1, dev1.contiguous(), L1)
    for k, y in enumerate(y1):
        assert np.array_equal(got1[k], y.c), k
    ref = ckks.forward_fp64(graph, W.input_nodes(graph), [x])
    n_img = x.shape[0] * graph["nodes"][1]["images"]
    err = float(np.max(np.abs(res[out_node].cpu().numpy()[:, :n_img] - ref[out_node][:, :n_img])))
    assert err < 1e-4
    net.close()


def test_mul_relin_rescale_output_overlapping_an_input():
    """fhe_mul_relin_rescale recomputes the tensor from its factors in every
    step, unless the output overlaps a factor (then the tensor is formed
    first): both give the oracle's words."""
    g, o = pair(1024, BITS5)
    rng = np.random.default_rng(11)
    L, n = 4, 3
    A = [rand_ct(o, L, rng) for _ in range(n)]
    B = [rand_ct(o, L, rng) for _ in range(n)]
    ta, tb = upload(g, A, L), upload(g, B, L)
    out = g.empty_ct(n, L - 1)
    g.mul_relin_rescale(ta, tb, L, out)
    got = download(g, out, L - 1)
    for k in range(n):
        want = o.rescale(o.relinearise(o.tensor(ckks.Ciphertext(A[k], L, 1.0), ckks.Ciphertext(B[k], L, 1.0)))).c
        assert np.array_equal(got[k], want), k
    # the output over the front of a's storage
    ta2 = ta.clone()
    alias = ta2.view(-1)[: n * 2 * (L - 1) * g.N].view(n, 2, L - 1, g.N)
    g.mul_relin_rescale(ta2, tb, L, alias)
    assert torch.equal(alias, out)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("N", [256, 4096])
def test_every_schedule_at_small_rings(N, variant):
    """Rings whose last register pass is a full radix-16 pass (log2 N a
    multiple of 4) or shorter: every schedule gives the oracle's
    mul + relinearise + rescale and key-switching results."""
    import os
    bits = [60, 40, 40, 40, 60]
    os.environ["FHE_NTT_VARIANT"] = str(variant)
    try:
        g = fhe.Context(N, bits, 40)
    finally:
        del os.environ["FHE_NTT_VARIANT"]
    g.keygen(0)
    o = ckks.Context(N, bits, 40)
    o.keygen(0)
    rng = np.random.default_rng(N + variant)
    L = 4
    A, B = rand_ct(o, L, rng), rand_ct(o, L, rng)
    ta, tb = upload(g, [A], L), upload(g, [B], L)
    out = g.empty_ct(1, L - 1)
    g.mul_relin_rescale(ta, tb, L, out)
    want = o.rescale(o.relinearise(o.tensor(ckks.Ciphertext(A, L, 1.0), ckks.Ciphertext(B, L, 1.0)))).c
    assert np.array_equal(download(g, out, L - 1)[0], want)
    g.close()


@pytest.mark.parametrize("variant", [6, 7])
@pytest.mark.parametrize("N", [64, 128, 512, 1024, 2048])
def test_split_transform_schedules_every_pass_split(N, variant):
    """Schedules 6 (key-switching digit transforms split over two blocks per
    polynomial) and 7 (a cluster of four blocks per polynomial, accumulators
    in shared memory; rings below 256 fall back to 6) on rings whose parts
    take every pass split: relinearisation and mul + relinearise + rescale
    equal the oracle's."""
    import os
    bits = [60, 40, 40, 40, 60]
    os.environ["FHE_NTT_VARIANT"] = str(variant)
    try:
        g = fhe.Context(N, bits, 40)
    finally:
        del os.environ["FHE_NTT_VARIANT"]
    assert g.ntt_variant_ks == variant
    g.keygen(0)
    o = ckks.Context(N, bits, 40)
    o.keygen(0)
    rng = np.random.default_rng(N)
    L = 4
    D3 = rand_ct(o, L, rng, comps=3)
    t3 = upload(g, [D3], L)
    r = g.empty_ct(1, L)
    g.relinearise(t3, L, r)
    assert np.array_equal(download(g, r, L)[0], o.relinearise(ckks.Ciphertext(D3, L, 1.0)).c)
    A, B = rand_ct(o, L, rng), rand_ct(o, L, rng)
    out = g.empty_ct(1, L - 1)
    g.mul_relin_rescale(upload(g, [A], L), upload(g, [B], L), L, out)
    want = o.rescale(o.relinearise(o.tensor(ckks.Ciphertext(A, L, 1.0), ckks.Ciphertext(B, L, 1.0)))).c
    assert np.array_equal(download(g, out, L - 1)[0], want)
    g.close()


@pytest.mark.parametrize("N", [512, 1024, 2048, 8192])
def test_warp_local_schedule_every_block_stage_count(N):
    """Schedule 8 (warp-local transforms) with 0, 1 and 3 block-wide stages
    before the per-warp 1024-point sub-transforms, and below 1024 its
    stand-in: relinearisation and mul + relinearise + rescale equal the
    oracle's (forward and inverse transforms, both butterfly forms: the
    60-bit primes take the reduced one)."""
    import os
    bits = [60, 40, 40, 40, 60]
    os.environ["FHE_NTT_VARIANT"] = "8"
    try:
        g = fhe.Context(N, bits, 40)
    finally:
        del os.environ["FHE_NTT_VARIANT"]
    assert g.ntt_variant == 8 and g.ntt_variant_ks == 8
    g.keygen(0)
    o = ckks.Context(N, bits, 40)
    o.keygen(0)
    rng = np.random.default_rng(N + 8)
    L = 4
    D3 = rand_ct(o, L, rng, comps=3)
    r = g.empty_ct(1, L)
    g.relinearise(upload(g, [D3], L), L, r)
    assert np.array_equal(download(g, r, L)[0], o.relinearise(ckks.Ciphertext(D3, L, 1.0)).c)
    A, B = rand_ct(o, L, rng), rand_ct(o, L, rng)
    out = g.empty_ct(1, L - 1)
    g.mul_relin_rescale(upload(g, [A], L), upload(g, [B], L), L, out)
    want = o.rescale(o.relinearise(o.tensor(ckks.Ciphertext(A, L, 1.0), ckks.Ciphertext(B, L, 1.0)))).c
    assert np.array_equal(download(g, out, L - 1)[0], want)
    g.close()


def test_graph_generic_degree_polynomials_bit_exact():
    """Polynomials of degree 5 and 4 (powers by products, one combining
    rescale) inside a graph: bit-exact against the oracle."""
    graph, x = W.poly_chain(n_slots=512)
    gof, gcost = fhe.autohe(graph)
    assert gcost == [1 + 4 + 1 + 3]
    g, o = pair(1024, [60] + [40] * 9 + [60])
    err = _graph_parity(g, o, graph, [x], [0])
    assert err < 1e-4


def test_graph_relu_and_affine_bit_exact():
    """Eq. relu_approximate (degree 2) after the convolution and the linear
    sigmoid 0.5 + 0.197 x (degree 1) after the dense layer."""
    graph, x = W.mini_cnn_relu(n_slots=512)
    g, o = pair(1024, [60] + [40] * 6 + [60])
    err = _graph_parity(g, o, graph, [x], [0])
    assert err < 1e-4


def test_graph_depth8_ring32768_bit_exact():
    """Depth 8: Alg. autoHE / parameterise choose N = 32768, [60, 40 x 8, 60];
    every stage (encode, encrypt, layers, relinearise, rescale, decode) runs on
    the two-pass transform."""
    graph, _ = W.deep_mlp(n_slots=4)
    gof, gcost = fhe.autohe(graph)
    assert max(gcost) == 8
    N, bits = fhe.parameterise(max(gcost), 40, 1.5)
    assert N == 32768 and bits == [60] + [40] * 8 + [60]
    g, o = pair(N, bits)
    assert g.ntt_variant in (2, 3)
    graph, x = W.deep_mlp(n_slots=N // 2)
    err = _graph_parity(g, o, graph, [x], [0])
    assert err < 1e-4


def test_grouped_rotation_bit_exact_per_group():
    """A rotation (client refresh) after the first sigmoid: groups of cost 3
    and 4, each on its own context.  Group 0's ciphertexts at the rotation and
    group 1's outputs (from the device's refreshed inputs) are bit-exact
    against the oracle; the decoded outputs are within 1e-4 of FP64."""
    from oracle import params
    from paper_2110_13638_gb300 import groups
    graph, x = W.mini_cnn_rotate(n_slots=512)
    N = 1024
    cost = params.autohe(graph, params.ingress_nodes(graph))[1]
    assert cost == [3, 4]
    pairs = [pair(N, params.parameterise(c)["coeff_modulus"], seed=gi) for gi, c in enumerate(cost)]
    net = groups.GroupedNetwork(graph, contexts={gi: p[0] for gi, p in enumerate(pairs)})
    assert net.order == [0, 1]
    res = net.evaluate([torch.tensor(x, device="cuda")], first_ct_id=0)
    torch.cuda.synchronize()
    rot, out_node = 3, 7
    assert graph["nodes"][rot]["kind"] == "rotate" and graph["nodes"][out_node]["kind"] == "output"
    # group 0: input -> conv -> sigmoid -> (rotation)
    g0, o0 = pairs[0]
    cts = [o0.encrypt(o0.encode(x[i]), i) for i in range(x.shape[0])]
    seg0 = W.chain_graph(x.shape[0], graph["nodes"][1:3])
    want0 = ckks.eval_graph(o0, seg0, [0], [cts])
    (_, y0), = want0.items()
    dev0, L0, sc0 = net.last_sinks[rot]
    got0 = download(g0, dev0.contiguous(), L0)
    for k, y in enumerate(y0):
        assert y.level == L0 and sc0[k] == y.scale
        assert np.array_equal(got0[k], y.c), k
    # group 1 from the device's refreshed ciphertexts: dense -> sigmoid -> dense
    g1, o1 = pairs[1]
    ref_in = net.last_ingress[rot]
    fresh = download(g1, ref_in, g1.L_top)
    cts1 = [ckks.Ciphertext(fresh[k], g1.L_top, o1.delta) for k in range(fresh.shape[0])]
    seg1 = W.chain_graph(fresh.shape[0], graph["nodes"][4:7])
    want1 = ckks.eval_graph(o1, seg1, [0], [cts1])
    (_, y1), = want1.items()
    dev1, L1, sc1 = net.last_sinks[out_node]
    got1 = download(g1, dev1.contiguous(), L1)
    for k, y in enumerate(y1):
        assert np.array_equal(got1[k], y.c), k
    ref = ckks.forward_fp64(graph, W.input_nodes(graph), [x])
    assert float(np.max(np.abs(res[out_node].cpu().numpy() - ref[out_node]))) < 1e-4
    net.close()


# ---------------------------------------------------------------- uneven levels, one persistent launch
@pytest.mark.parametrize("N", [512, 1024])
def test_mul_relin_rescale_levels_matches_per_batch_and_oracle(N):
    """One persistent launch over levels 2..8 at two ring degrees: equal to
    the per-level calls and to the oracle."""
    g, o = pair(N, BITS9)
    rng = np.random.default_rng(42)
    batches, ref_outs = [], []
    keep = {}
    for L in range(2, 9):
        n = int(rng.integers(1, 4))
        A = [rand_ct(o, L, rng) for _ in range(n)]
        B = [rand_ct(o, L, rng) for _ in range(n)]
        ta, tb = upload(g, A, L), upload(g, B, L)
        out = g.empty_ct(n, L - 1)
        ref = g.empty_ct(n, L - 1)
        g.mul_relin_rescale(ta, tb, L, ref)
        batches.append((ta, tb, out, L))
        ref_outs.append(ref)
        keep[L] = (A, B)
    torch.cuda.synchronize()
    before = fhe.launch_count()
    g.mul_relin_rescale_levels(batches)
    g.sync()
    assert fhe.launch_count() - before == 1           # one persistent launch for every level
    for (ta, tb, out, L), ref in zip(batches, ref_outs):
        assert torch.equal(out, ref), L
    # every level against the oracle directly
    for L in range(2, 9):
        A, B = keep[L]
        got = download(g, batches[L - 2][2], L - 1)
        for k in range(len(A)):
            want = o.rescale(o.relinearise(o.tensor(ckks.Ciphertext(A[k], L, 1.0),
                                                    ckks.Ciphertext(B[k], L, 1.0)))).c
            assert np.array_equal(got[k], want), (L, k)


@pytest.mark.parametrize("N", [4096, 16384])
def test_mul_relin_rescale_levels_persistent_equals_separate_launches(monkeypatch, N):
    """The persistent launch and the six-launch form (FHE_PERSISTENT=0) give
    the same words, on a batch large enough that many units wait for their
    ciphertext's previous step; at N = 16384 the six-launch form runs the
    grouped radix-8 transforms whose later passes use warp barriers."""
    if N == 4096:
        g, o = pair(N, BITS9)
    else:
        monkeypatch.setenv("FHE_NTT_VARIANT", "4")
        monkeypatch.setenv("FHE_NTT_VARIANT_KS", "8")
        g = fhe.Context(N, BITS9, 40)
        monkeypatch.delenv("FHE_NTT_VARIANT")
        monkeypatch.delenv("FHE_NTT_VARIANT_KS")
        g.keygen(0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9)
    batches = []
    for L, n in ((2, 40), (5, 33), (8, 21)):
        def rnd():
            t = torch.empty((n, 2, L, g.N), dtype=torch.int64, device="cuda")
            for r in range(L):
                t[:, :, r, :] = torch.randint(0, g.primes[r], (n, 2, g.N), device="cuda", generator=gen)
            return t
        batches.append((rnd(), rnd(), g.empty_ct(n, L - 1), L))
    g.mul_relin_rescale_levels(batches)
    g.sync()
    want = [b[2].clone() for b in batches]
    monkeypatch.setenv("FHE_PERSISTENT", "0")
    for b in batches:
        b[2].zero_()
    before = fhe.launch_count()
    g.mul_relin_rescale_levels(batches)
    g.sync()
    assert fhe.launch_count() - before == 6
    for b, w in zip(batches, want):
        assert torch.equal(b[2], w), b[3]
    if N != 4096:
        g.close()


def test_persistent_wait_that_runs_out_reports_timeout():
    """The persistent launch's waits are bounded: with the first step's
    completions withheld (test hook) the second step's waits run out, the
    launch abandons its remaining units and the context reports
    FHE_ETIMEOUT; the next call gives the right words again."""
    g, o = pair(1024, BITS9)
    rng = np.random.default_rng(44)
    batches = []
    for L in (4, 7):
        A = [rand_ct(o, L, rng) for _ in range(3)]
        B = [rand_ct(o, L, rng) for _ in range(3)]
        batches.append((upload(g, A, L), upload(g, B, L), g.empty_ct(3, L - 1), L))
    g.mul_relin_rescale_levels(batches)
    g.sync()
    want = [b[2].clone() for b in batches]
    g.inject_fault(2)
    with pytest.raises(fhe.FheError) as e:
        g.mul_relin_rescale_levels(batches)
        g.sync()
    assert e.value.code == -6
    for b in batches:
        b[2].zero_()
    g.mul_relin_rescale_levels(batches)
    g.sync()
    for b, w in zip(batches, want):
        assert torch.equal(b[2], w)


def test_mul_relin_rescale_levels_in_cuda_graph():
    g, o = pair(1024, BITS9)
    rng = np.random.default_rng(43)
    batches = []
    for L in (3, 8, 6):
        A = [rand_ct(o, L, rng) for _ in range(2)]
        B = [rand_ct(o, L, rng) for _ in range(2)]
        batches.append((upload(g, A, L), upload(g, B, L), g.empty_ct(2, L - 1), L))
    g.mul_relin_rescale_levels(batches)          # sizes the workspace
    torch.cuda.synchronize()
    want = [b[2].clone() for b in batches]
    for b in batches:
        b[2].zero_()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            g.mul_relin_rescale_levels(batches)
    torch.cuda.current_stream().wait_stream(s)
    graph.replay()
    torch.cuda.synchronize()
    for b, w in zip(batches, want):
        assert torch.equal(b[2], w)


# ---------------------------------------------------------------- rings above 16384 (two-pass NTT only)
@pytest.mark.parametrize("N", [32768, 65536])
def test_large_ring_transform_tensor_relin(N):
    bits = [60, 40, 60]
    g, o = pair(N, bits)
    assert g.ntt_variant in (2, 3)
    rng = np.random.default_rng(N)
    L = 2
    A = [rand_ct(o, L, rng)]
    B = [rand_ct(o, L, rng)]
    ta, tb = upload(g, A, L), upload(g, B, L)
    assert np.array_equal(download(g, ta, L), np.stack(A))
    t3 = g.empty_ct(1, L, comps=3)
    g.tensor(ta, tb, L, t3)
    want = o.tensor(ckks.Ciphertext(A[0], L, 1.0), ckks.Ciphertext(B[0], L, 1.0))
    assert np.array_equal(download(g, t3, L)[0], want.c)
    out = g.empty_ct(1, L)
    g.relinearise(t3, L, out)
    assert np.array_equal(download(g, out, L)[0], o.relinearise(want).c)


@pytest.mark.parametrize("N,bits,n", [(1024, BITS5, 3), (16384, BITS9, 2), (32768, [60, 40, 40, 60], 2)])
def test_encode_encrypt_fused_equals_two_calls(N, bits, n):
    g, o = pair(N, bits)
    z = torch.tensor(np.random.default_rng(N).uniform(-2, 2, size=(n, N // 2)), device="cuda")
    pt = g.empty_pt(n, g.L_top)
    a = g.empty_ct(n, g.L_top)
    b = g.empty_ct(n, g.L_top)
    g.encode(z, g.L_top, g.delta, pt)
    g.encrypt(pt, 333, a)
    g.encode_encrypt(z, g.delta, 333, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
