"""Pins of the oracle's scheme: encryption, CRT, tensor, key switching,
ModDown, rescale, the network blocks and graph evaluation (Alg. firing)."""
import numpy as np
import pytest

from oracle import ckks, core
from paper_2110_13638_gb300 import workloads as W
import golden_io

BITS4 = [60, 40, 40, 40, 60]


@pytest.fixture(scope="module")
def ctx16():
    c = ckks.Context(16, BITS4)
    c.keygen(3)
    return c


@pytest.fixture(scope="module")
def ctx64():
    c = ckks.Context(64, BITS4)
    c.keygen(0)
    return c


def _schoolbook_z(a, b):
    """negacyclic product over the integers (lists of Python ints)"""
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            if i + j < N:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - N] -= a[i] * b[j]
    return c


def _crt(ctx, res, primes):
    """residues [len(primes)][N] -> list of integers in [0, prod)"""
    Q = 1
    for p in primes:
        Q *= p
    out = []
    for k in range(res.shape[1]):
        x = 0
        for r, p in enumerate(primes):
            Qr = Q // p
            x += int(res[r, k]) * Qr * pow(Qr, -1, p)
        out.append(x % Q)
    return out, Q


def _centre(x, Q):
    return x - Q if x > (Q - 1) // 2 else x


def _s_int(ctx):
    return [int(v) for v in ctx.s_int]


def _phase(ctx, c, level):
    """c0 + c1 s (+ c2 s^2) over the integers mod Q_level, centred."""
    primes = ctx.q[:level]
    s = _s_int(ctx)
    comps = [_crt(ctx, c[k], primes)[0] for k in range(c.shape[0])]
    Q = 1
    for p in primes:
        Q *= p
    acc = list(comps[0])
    spow = s
    for k in range(1, c.shape[0]):
        prod = _schoolbook_z(comps[k], spow)
        acc = [a + b for a, b in zip(acc, prod)]
        spow = _schoolbook_z(spow, s)
    return [_centre(a % Q, Q) for a in acc]


# ---------------------------------------------------------------- keys / enc
def test_keys_have_the_stated_form(ctx16):
    """pk0 + pk1 s is small (the Gaussian e); ksk_j[0] + ksk_j[1] s is
    e_j + P s^2 in residue j and e_j elsewhere."""
    ctx = ctx16
    N = ctx.N
    s = _s_int(ctx)
    for r in range(ctx.L_top):
        q = ctx.q[r]
        v = [(int(a) + b) % q for a, b in zip(ctx.pk[0, r], _schoolbook_z([int(x) for x in ctx.pk[1, r]], s))]
        v = [_centre(x, q) for x in v]
        assert max(abs(x) for x in v) <= 19
    s2 = _schoolbook_z(s, s)
    for j in range(ctx.L_top):
        for r, p in enumerate(ctx.key_primes):
            v = [(int(a) + b) % p for a, b in zip(ctx.ksk[j, 0, r], _schoolbook_z([int(x) for x in ctx.ksk[j, 1, r]], s))]
            if r == j:
                v = [(x - ctx.P * t) % p for x, t in zip(v, s2)]
            v = [_centre(x, p) for x in v]
            assert max(abs(x) for x in v) <= 19, (j, r)


def test_encrypt_decrypt_roundtrip(ctx64):
    ctx = ctx64
    N = ctx.N
    z = np.random.default_rng(0).uniform(-1, 1, N // 2)
    m = ctx.encode(z)
    ct = ctx.encrypt(m, 17)
    d = ctx.decrypt(ct, check_crt=True)
    bound = 2 * 19 * N + 19          # |u e| + |e1 s| + |e0|
    assert np.max(np.abs(d - m)) <= bound
    assert np.max(np.abs(d - m)) > 0   # noise is present
    assert np.max(np.abs(ctx.decode(d, ct.scale) - z)) < bound / ctx.delta + N / ctx.delta


def test_encryptions_differ_by_ct_id(ctx16):
    m = np.zeros(16, dtype=np.int64)
    a = ctx16.encrypt(m, 1).c
    b = ctx16.encrypt(m, 2).c
    assert not np.array_equal(a, b)
    assert np.array_equal(a, ctx16.encrypt(m, 1).c)


# ---------------------------------------------------------------- tensor
def test_tensor_phase_is_product_of_phases(ctx16):
    ctx = ctx16
    rng = np.random.default_rng(1)
    L = 3
    a = ckks.Ciphertext(np.stack([np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in ctx.q[:L]]) for _ in range(2)]), L, 1.0)
    b = ckks.Ciphertext(np.stack([np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in ctx.q[:L]]) for _ in range(2)]), L, 1.0)
    d = ctx.tensor(a, b)
    Q = ctx.q[0] * ctx.q[1] * ctx.q[2]
    pa, pb, pd = _phase(ctx, a.c, L), _phase(ctx, b.c, L), _phase(ctx, d.c, L)
    want = [_centre(x % Q, Q) for x in _schoolbook_z(pa, pb)]
    assert pd == want


# ---------------------------------------------------------------- rescale
def test_rescale_is_rounded_division(ctx16):
    ctx = ctx16
    rng = np.random.default_rng(2)
    L = 4
    c = np.stack([np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in ctx.q[:L]]) for _ in range(2)])
    out = ctx.rescale(ckks.Ciphertext(c, L, 2.0 ** 80))
    ql = ctx.q[L - 1]
    for k in range(2):
        X, Q = _crt(ctx, c[k], ctx.q[:L])
        for i in range(L - 1):
            for n in range(16):
                want = ((X[n] + ql // 2) // ql) % ctx.q[i]     # round(X / q_{L-1}), no ties
                assert int(out.c[k, i, n]) == want
    assert out.level == L - 1 and out.scale == 2.0 ** 80 / float(ql)


def test_mod_down_is_rounded_division(ctx16):
    ctx = ctx16
    rng = np.random.default_rng(3)
    L = 3
    primes = ctx.q[:L] + [ctx.P]
    acc = np.stack([np.stack([rng.integers(0, p, 16, dtype=np.uint64) for p in primes]) for _ in range(2)])
    out = ctx.mod_down(acc, L)
    P = ctx.P
    for k in range(2):
        X, _ = _crt(ctx, acc[k], primes)
        for t in range(L):
            for n in range(16):
                assert int(out[k, t, n]) == ((X[n] + P // 2) // P) % ctx.q[t]


def test_keyswitch_accumulator_definition(ctx16):
    """acc_k = sum_j [d2]_{q_j} ksk_j[k] in every prime (schoolbook)."""
    ctx = ctx16
    rng = np.random.default_rng(4)
    L = 2
    d2 = np.stack([rng.integers(0, q, 16, dtype=np.uint64) for q in ctx.q[:L]])
    acc = ctx.keyswitch_accumulate(d2, L)
    for ti, kr in enumerate(list(range(L)) + [ctx.L_top]):
        p = ctx.key_primes[kr]
        for k in range(2):
            want = [0] * 16
            for j in range(L):
                prod = _schoolbook_z([int(x) for x in d2[j]], [int(x) for x in ctx.ksk[j, k, kr]])
                want = [a + b for a, b in zip(want, prod)]
            assert [int(x) for x in acc[k, ti]] == [w % p for w in want]


@pytest.mark.parametrize("L", [1, 2, 4])
def test_relinearise_preserves_phase(ctx16, L):
    """decrypt(relin(d0, d1, d2)) = d0 + d1 s + d2 s^2 up to the key-switching
    noise: rounding (<= 1/2 per coefficient of each component, times |s|)
    plus sum_j |digit_j| |e_j| N / P."""
    ctx = ctx16
    N = 16
    rng = np.random.default_rng(5 + L)
    d = np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in ctx.q[:L]]) for _ in range(3)])
    before = _phase(ctx, d, L)
    r = ctx.relinearise(ckks.Ciphertext(d, L, 1.0))
    after = _phase(ctx, r.c, L)
    bound = 0.5 + 0.5 * N + L * max(ctx.q) * 19 * N / ctx.P + 1
    assert max(abs(a - b) for a, b in zip(after, before)) <= bound


# ---------------------------------------------------------------- blocks
def test_linear_block(ctx64):
    ctx = ctx64
    N = ctx.N
    rng = np.random.default_rng(7)
    xs = rng.uniform(-1, 1, size=(3, N // 2))
    cts = [ctx.encrypt(ctx.encode(x), 100 + i) for i, x in enumerate(xs)]
    Wt = rng.normal(0, 0.5, size=(2, 3))
    b = np.array([0.3, -0.2])
    rows = [(np.arange(3), Wt[o]) for o in range(2)]
    ys = ctx.linear(cts, rows, b)
    for o in range(2):
        assert ys[o].level == ctx.L_top - 1
        assert ys[o].scale == ctx.delta
        got = ctx.decode(ctx.decrypt(ys[o]), ys[o].scale)
        assert np.max(np.abs(got - (Wt[o] @ xs + b[o]))) < 1e-6


def test_square_and_poly3_blocks(ctx64):
    ctx = ctx64
    N = ctx.N
    z = np.random.default_rng(8).uniform(-4, 4, N // 2)
    ct = ctx.encrypt(ctx.encode(z), 5)
    sq = ctx.square(ct)
    assert sq.level == ctx.L_top - 1
    assert np.max(np.abs(ctx.decode(ctx.decrypt(sq), sq.scale) - z * z)) < 1e-6
    a = [0.5, 0.2, 0.01, -0.004]
    y = ctx.poly3(ct, a)
    assert y.level == ctx.L_top - 2
    assert abs(y.scale / ctx.delta - 1) < 1e-9
    ref = a[0] + a[1] * z + a[2] * z * z + a[3] * z ** 3
    assert np.max(np.abs(ctx.decode(ctx.decrypt(y), y.scale) - ref)) < 1e-6


def test_affine_and_poly2_blocks(ctx64):
    ctx = ctx64
    N = ctx.N
    z = np.random.default_rng(9).uniform(-3, 3, N // 2)
    ct = ctx.encrypt(ctx.encode(z), 6)
    y1 = ctx.poly(ct, [0.5, 0.197])
    assert y1.level == ctx.L_top - 1 and y1.scale == ctx.delta
    assert np.max(np.abs(ctx.decode(ctx.decrypt(y1), y1.scale) - (0.5 + 0.197 * z))) < 1e-6
    a = [0.3, 0.5, 0.11]
    y2 = ctx.poly(ct, a)
    assert y2.level == ctx.L_top - 2
    assert abs(y2.scale / ctx.delta - 1) < 1e-9
    ref = a[0] + a[1] * z + a[2] * z * z
    assert np.max(np.abs(ctx.decode(ctx.decrypt(y2), y2.scale) - ref)) < 1e-6
    with pytest.raises(ValueError):
        ctx.poly(ct, [0.1] * 33)                 # degree 32: above the supported 31


@pytest.mark.parametrize("d", [4, 5, 7, 8])
def test_higher_degree_polynomial_block(d):
    """Degree >= 4 by products of powers and one combining rescale: decrypts
    to the plaintext polynomial, uses ceil(log2 d) + 1 levels, keeps the
    scale, and its node cost says the same."""
    from oracle import params
    depth = (d - 1).bit_length() + 1
    ctx = ckks.Context(64, [60] + [40] * (depth + 1) + [60])
    ctx.keygen(1)
    z = np.random.default_rng(d).uniform(-1.2, 1.2, ctx.N // 2)
    ct = ctx.encrypt(ctx.encode(z), 11)
    a = list(np.random.default_rng(100 + d).normal(0.0, 0.3, d + 1))
    a[2] = 0.0                                 # a zero coefficient is skipped
    y = ctx.poly(ct, a)
    assert ctx.L_top - y.level == depth == params.node_cost({"kind": "poly", "coeffs": a})
    assert abs(y.scale / ctx.delta - 1) < 1e-9
    ref = sum(a[i] * z ** i for i in range(d + 1))
    assert np.max(np.abs(ctx.decode(ctx.decrypt(y), y.scale) - ref)) < 1e-6


@pytest.mark.parametrize("q", [1.0, 3.0, 4.0, 10.0])
def test_relu_approximation_is_the_degree2_chebyshev_truncation(q):
    """Eq. relu_approximate equals the first three terms of the Chebyshev
    series of max(0, x) on [-q, q] (Gauss-Chebyshev quadrature), in the power
    basis; at x = +-q it is off max(0, x) by 5q/(3 pi) - q/2 (about 0.031 q)."""
    n = 200000
    t = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    f = np.maximum(0.0, q * t)
    c = [(2.0 / n) * np.sum(f * np.cos(k * np.arccos(t))) for k in range(3)]
    # c0/2 + c1 T1(x/q) + c2 T2(x/q), T2(u) = 2u^2 - 1
    a0 = c[0] / 2 - c[2]
    a1 = c[1] / q
    a2 = 2 * c[2] / (q * q)
    got = ckks.relu_coeffs(q)
    assert np.allclose(got, [a0, a1, a2], rtol=1e-6, atol=1e-9)
    r = lambda x: got[0] + got[1] * x + got[2] * x * x
    assert abs(r(0.0) - q / (3 * np.pi)) < 1e-12
    assert abs(r(q) - q) < q * 0.05 and abs(r(-q)) < q * 0.05


def test_node_costs_of_activations():
    from oracle import params
    assert params.node_cost({"kind": "poly", "coeffs": [0.5, 0.197]}) == 1
    assert params.node_cost({"kind": "poly", "coeffs": [0.1, 0.2, 0.3]}) == 2
    assert params.node_cost({"kind": "poly", "coeffs": [0.1, 0.2, 0.3, 0.4]}) == 2
    assert params.node_cost({"kind": "relu", "q": 3.0}) == 2
    g, _ = W.mini_cnn_relu(8)
    assert ckks.graph_depth(g, W.input_nodes(g)) == 6
    g, _ = W.cnn_relu(8)
    assert ckks.graph_depth(g, W.input_nodes(g)) == 7


# ---------------------------------------------------------------- rotations
def _eval_at(coeffs, x, q):
    acc = 0
    for c in reversed([int(v) for v in coeffs]):
        acc = (acc * x + c) % q
    return acc


def test_automorphism_is_substitution_at_the_roots(ctx16):
    """(a o X^k)(psi^e) = a(psi^(e k)) at every odd power e (the roots of
    X^N + 1), by Horner evaluation with Python integers."""
    ctx = ctx16
    N, q = ctx.N, ctx.q[0]
    psi = ctx.psi[0]
    rng = np.random.default_rng(21)
    a = rng.integers(0, q, N, dtype=np.uint64)
    for k in (5, 25, 2 * N - 1, ctx.galois_element(3)):
        b = ctx.automorphism(a[None], k, [q])[0]
        for e in (1, 3, 7, 2 * N - 1):
            x = pow(psi, e, q)
            assert _eval_at(b, x, q) == _eval_at(a, pow(psi, e * k, q), q), (k, e)


def test_galois_elements_cycle_with_order_half_n():
    ctx = ckks.Context(64, BITS4)
    ks = [ctx.galois_element(r) for r in range(32)]
    assert len(set(ks)) == 32 and all(k % 2 == 1 for k in ks)
    assert ctx.galois_element(32) == 1 and ctx.galois_element(-1) == ks[31]


def test_rotation_rolls_the_slots(ctx64):
    ctx = ctx64
    N = ctx.N
    z = np.random.default_rng(22).uniform(-1, 1, N // 2)
    ct = ctx.encrypt(ctx.encode(z), 9)
    for r in (1, 3, -2, 17):
        y = ctx.rotate(ct, r)
        assert y.level == ct.level and y.scale == ct.scale
        got = ctx.decode(ctx.decrypt(y), y.scale)
        assert np.max(np.abs(got - np.roll(z, -r))) < 1e-6, r
    # rotations compose: rot(rot(x, 2), 3) = rot(x, 5)
    y = ctx.rotate(ctx.rotate(ct, 2), 3)
    assert np.max(np.abs(ctx.decode(ctx.decrypt(y), y.scale) - np.roll(z, -5))) < 1e-6


def test_galois_key_switches_from_the_rotated_secret(ctx16):
    """The key-switched component decrypts to c1(X^k) s(X^k) up to small noise:
    ks_0 + ks_1 s - c1(X^k) s(X^k) is small modulo Q_L."""
    ctx = ctx16
    L = ctx.L_top
    rng = np.random.default_rng(23)
    c1 = np.stack([rng.integers(0, q, ctx.N, dtype=np.uint64) for q in ctx.q[:L]])
    k = ctx.galois_element(1)
    ks = ctx.mod_down(ctx.keyswitch_accumulate(c1, L, ctx.galois_keygen(k)), L)
    sk = [int(v) for v in ctx.automorphism(np.array([[int(x) % ctx.q[0] for x in ctx.s_int]], dtype=np.uint64), k,
                                                    [ctx.q[0]])[0]]
    # reduce everything mod q_0 and compare phases there
    q = ctx.q[0]
    s = [int(x) % q for x in ctx.s_int]
    lhs = [(int(a) + int(b)) % q for a, b in zip(ks[0, 0], _schoolbook_z([int(v) for v in ks[1, 0]], s))]
    rhs = [x % q for x in _schoolbook_z([int(v) for v in c1[0]], sk)]
    diff = [((a - b + q // 2) % q) - q // 2 for a, b in zip(lhs, rhs)]
    assert max(abs(d) for d in diff) < 2 ** 20


# ---------------------------------------------------------------- kernel masquerading
def _direct_conv(x, node, images, slots_per_img):
    """features [F * OH * OW][n_ct * images] by plain loops over unpacked images"""
    F, k, st, H, Wd = node["filters"], node["k"], node["stride"], node["H"], node["W"]
    OH, OW = (H - k) // st + 1, (Wd - k) // st + 1
    K = np.asarray(node["weight"])
    cols = []
    for i in range(x.shape[0]):
        for b in range(images):
            img = x[i, b * slots_per_img:b * slots_per_img + H * Wd].reshape(H, Wd)
            col = np.zeros(F * OH * OW)
            for f in range(F):
                for r in range(OH):
                    for c in range(OW):
                        v = sum(K[f, dr, dc] * img[st * r + dr, st * c + dc] for dr in range(k) for dc in range(k))
                        col[f * OH * OW + r * OW + c] = v + node["bias"][f]
            cols.append(col)
    return np.stack(cols, axis=1)


def test_packed_conv_and_relayout_equal_the_direct_convolution():
    g, x = W.cnn_masquerade(3, 32, side=4, k=2, stride=2)
    conv = g["nodes"][1]
    sub = {"nodes": [g["nodes"][0], conv, dict(g["nodes"][3]), {"kind": "output"}],
           "edges": [(0, 1), (1, 2), (2, 3)]}
    got = ckks.forward_fp64(sub, [0], [x])[3]
    want = _direct_conv(x, conv, conv["images"], conv["slot_stride"])
    assert np.allclose(got[:, :want.shape[1]], want, atol=1e-12)
    assert np.all(got[:, want.shape[1]:] == 0)


def test_conv_packed_decrypts_to_the_convolution(ctx64):
    ctx = ctx64
    g, x = W.cnn_masquerade(2, ctx.N // 2, side=4, k=3, stride=1)
    conv = g["nodes"][1]
    cts = [ctx.encrypt(ctx.encode(v), 300 + i) for i, v in enumerate(x)]
    ys = ctx.conv_packed(cts, conv)
    assert len(ys) == conv["filters"] * 2 and ys[0].level == ctx.L_top - 1
    z = np.stack([ctx.decode(ctx.decrypt(y), y.scale) for y in ys])
    feats = ckks.relayout_packed(z, conv, 2)
    want = _direct_conv(x, conv, conv["images"], conv["slot_stride"])
    assert np.max(np.abs(feats[:, :want.shape[1]] - want)) < 1e-6
    invalid = np.ones(ctx.N // 2, dtype=bool)
    invalid[ckks.packed_valid_slots(conv, ctx.N // 2)] = False
    assert np.max(np.abs(z[:, invalid])) < 1e-6      # the masks zero every other slot


def test_grouped_masquerade_cnn_matches_fp64():
    from oracle import params
    g, x = W.cnn_masquerade(2, 32, side=4, k=2, stride=2)
    cost = params.autohe(g, params.ingress_nodes(g))[1]
    assert cost == [3, 4]
    ctxs = {}
    for grp, c in enumerate(cost):
        ctxs[grp] = ckks.Context(64, params.parameterise(c)["coeff_modulus"])
        ctxs[grp].keygen(grp)
    cts = [ctxs[0].encrypt(ctxs[0].encode(v), i) for i, v in enumerate(x)]
    out = ckks.eval_graph_grouped(ctxs, g, [cts])
    ref = ckks.forward_fp64(g, W.input_nodes(g), [x])
    (o, ys), = out.items()
    for y, r in zip(ys, ref[o]):
        assert np.max(np.abs(ctxs[1].decode(ctxs[1].decrypt(y), y.scale) - r)) < 1e-4


def test_sigmoid_fit_reproduces_printed_coefficients():
    got = W.sigmoid_fit()
    want = golden_io.sigmoid_coeffs()
    # the paper prints three decimals
    for g, w in zip(got, want):
        assert abs(g - w) < 1.5e-3
    assert abs(got[1] - want[1]) > 1e-4       # a1 really is 0.198..., not 0.197


# ---------------------------------------------------------------- graphs
def test_graph_eval_mini_cnn_matches_fp64():
    g, x = W.mini_cnn(n_slots=32)
    assert ckks.graph_depth(g, W.input_nodes(g)) == 7
    ctx = ckks.Context(64, [60] + [40] * 7 + [60])
    ctx.keygen(0)
    cts = [ctx.encrypt(ctx.encode(v), i) for i, v in enumerate(x)]
    out = ckks.eval_graph(ctx, g, W.input_nodes(g), [cts])
    ref = ckks.forward_fp64(g, W.input_nodes(g), [x])
    (o, ys), = out.items()
    assert len(ys) == ref[o].shape[0] == 3
    for y, r in zip(ys, ref[o]):
        assert y.level == 1
        assert np.max(np.abs(ctx.decode(ctx.decrypt(y), y.scale) - r)) < 1e-4


def test_graph_eval_relu_and_affine_match_fp64():
    g, x = W.mini_cnn_relu(n_slots=32)
    ctx = ckks.Context(64, [60] + [40] * 6 + [60])
    ctx.keygen(0)
    cts = [ctx.encrypt(ctx.encode(v), i) for i, v in enumerate(x)]
    out = ckks.eval_graph(ctx, g, W.input_nodes(g), [cts])
    ref = ckks.forward_fp64(g, W.input_nodes(g), [x])
    (o, ys), = out.items()
    for y, r in zip(ys, ref[o]):
        assert y.level == 1
        assert np.max(np.abs(ctx.decode(ctx.decrypt(y), y.scale) - r)) < 1e-4


def test_grouped_eval_with_rotation_matches_fp64():
    """A rotation (client refresh) splits the CNN into parameter groups of
    cost 3 and 4; each group evaluates under its own keys and the refreshed
    ciphertexts restart at the second group's top level."""
    from oracle import params
    g, x = W.mini_cnn_rotate(n_slots=32)
    ing = params.ingress_nodes(g)
    assert [g["nodes"][i]["kind"] for i in ing] == ["input", "rotate"]
    group_of, cost, _ = params.autohe(g, ing)
    assert cost == [3, 4] and group_of[ing[0]] == 0 and group_of[ing[1]] == 1
    ctxs = {}
    for grp, c in enumerate(cost):
        bits = params.parameterise(c)["coeff_modulus"]
        ctxs[grp] = ckks.Context(64, bits)
        ctxs[grp].keygen(grp)
    cts = [ctxs[0].encrypt(ctxs[0].encode(v), i) for i, v in enumerate(x)]
    out = ckks.eval_graph_grouped(ctxs, g, [cts])
    ref = ckks.forward_fp64(g, W.input_nodes(g), [x])
    (o, ys), = out.items()
    for y, r in zip(ys, ref[o]):
        assert y.level == 1
        assert np.max(np.abs(ctxs[1].decode(ctxs[1].decrypt(y), y.scale) - r)) < 1e-4
    # the same network without the rotation needs one group of cost 7
    g1, _ = W.mini_cnn(n_slots=32)
    assert params.autohe(g1, W.input_nodes(g1))[1] == [7]


def test_graph_eval_branches_level_match():
    g, xs = W.branch_graph(n_slots=32)
    ins = W.input_nodes(g)
    ctx = ckks.Context(64, [60, 40, 40, 40, 60])
    ctx.keygen(1)
    sig = [[ctx.encrypt(ctx.encode(v), 10 * k + i) for i, v in enumerate(x)] for k, x in enumerate(xs)]
    out = ckks.eval_graph(ctx, g, ins, sig)
    ref = ckks.forward_fp64(g, ins, xs)
    (o, ys), = out.items()
    assert len(ys) == 4
    for y, r in zip(ys, ref[o]):
        assert y.level == 1
        assert np.max(np.abs(ctx.decode(ctx.decrypt(y), y.scale) - r)) < 1e-5


def test_firing_waits_for_all_inbound_edges():
    order = []
    nodes = [{"kind": "input"}, {"kind": "input"}, {"kind": "add"}, {"kind": "output"}]
    g = {"nodes": nodes, "edges": [(0, 2), (1, 2), (2, 3)]}

    def apply_fn(n, node, s):
        order.append(n)
        if isinstance(s, dict):
            return sum(s["edges"])
        return s

    out = ckks.fire(g, [0, 1], [5, 7], apply_fn, lambda sigs: {"edges": sigs})
    assert order == [0, 1, 2, 3]          # node 2 fired only after input 1 arrived
    assert out == {3: 12}
