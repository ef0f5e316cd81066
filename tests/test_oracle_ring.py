"""Pins of the oracle's ring arithmetic: modular products, the negacyclic NTT
(against the O(N^2) definition and big-integer sums) and the sampling spec."""
import math

import numpy as np
import pytest

from oracle import core, params
import golden_io

Q60 = 0x1000000000024001      # 2^60 < q, q = 1 mod 2^14
Q40 = 0x10000048001


def test_mulmod_against_python_integers():
    rng = np.random.default_rng(0)
    for q in (Q60, Q40, 97, 2 ** 61 - 1):
        for _ in range(200):
            a = int(rng.integers(0, 2 ** 63)) % q
            b = int(rng.integers(0, 2 ** 63)) % q
            assert core.mulmod(a, b, q) == a * b % q
        assert int(core.lib().o_powmod(3, q - 1, q)) == pow(3, q - 1, q)


def _bigint_negacyclic(a, b, q):
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                c[k] += int(a[i]) * int(b[j])
            else:
                c[k - N] -= int(a[i]) * int(b[j])
    return [x % q for x in c]


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
def test_ntt_product_equals_schoolbook(N):
    rng = np.random.default_rng(N)
    for q in (params.prime_chain(N, [60, 40, 60])):
        psi = params.primitive_2n_root(q, N)
        a = rng.integers(0, q, size=N, dtype=np.uint64)
        b = rng.integers(0, q, size=N, dtype=np.uint64)
        want = _bigint_negacyclic(a, b, q)
        assert [int(x) for x in core.polymul_schoolbook(a, b, q)] == want
        assert [int(x) for x in core.polymul(a, b, q, psi)] == want


@pytest.mark.parametrize("N", [16, 64])
def test_ntt_is_evaluation_at_odd_powers(N):
    """A_k = a(psi^(2k+1)): checked by Horner in Python integers."""
    q = params.prime_chain(N, [40, 60])[0]
    psi = params.primitive_2n_root(q, N)
    a = np.random.default_rng(3).integers(0, q, size=N, dtype=np.uint64)
    A = core.ntt(a, q, psi)
    for k in range(N):
        x = pow(psi, 2 * k + 1, q)
        acc = 0
        for c in reversed([int(v) for v in a]):
            acc = (acc * x + c) % q
        assert int(A[k]) == acc


@pytest.mark.parametrize("N", [1024, 16384])
def test_ntt_roundtrip_and_spot_product(N):
    rng = np.random.default_rng(1)
    q = params.prime_chain(N, [60, 40, 60])[1]
    psi = params.primitive_2n_root(q, N)
    a = rng.integers(0, q, size=N, dtype=np.uint64)
    b = rng.integers(0, q, size=N, dtype=np.uint64)
    assert np.array_equal(core.intt(core.ntt(a, q, psi), q, psi), a)
    c = core.polymul(a, b, q, psi)
    ai = [int(x) for x in a]
    bi = [int(x) for x in b]
    for k in (0, 1, N // 2, N - 1, 12345 % N):
        s = 0
        for i in range(N):
            j = k - i
            s += ai[i] * bi[j] if j >= 0 else -ai[i] * bi[j + N]
        assert int(c[k]) == s % q


# ---------------------------------------------------------------- sampling
def test_splitmix64_published_vector():
    assert [core.splitmix_out(0, i) for i in range(3)] == golden_io.splitmix64()


def test_gaussian_table_against_float_cdf():
    cdt = params.gauss_cdt()
    assert len(cdt) == 38
    assert all(cdt[i] < cdt[i + 1] for i in range(37))
    s = 3.2
    ks = range(-19, 20)
    rho = [math.exp(-k * k / (2 * s * s)) for k in ks]
    S = math.fsum(rho)
    acc = 0.0
    for i in range(38):
        acc += rho[i]
        assert abs(cdt[i] / 2.0 ** 64 - acc / S) < 1e-13
    # symmetric distribution: T_i + T_{37-i} ~ 2^64
    for i in range(19):
        assert abs((cdt[i] + cdt[37 - i]) / 2.0 ** 64 - 1.0) < 1e-13


def test_sampler_statistics():
    N = 1 << 16
    cdt = np.array(params.gauss_cdt(), dtype=np.uint64)
    e = core.sample_gauss(core.stream(42, 3, 0), N, cdt)
    assert e.min() >= -19 and e.max() <= 19
    assert abs(e.mean()) < 4 * 3.2 / math.sqrt(N)
    var_true = 10.24                     # sigma^2 (the truncation changes it < 1e-15)
    assert abs(e.var() - var_true) < 4 * math.sqrt(2 * var_true ** 2 / N)
    t = core.sample_ternary(core.stream(42, 1, 0), N)
    assert set(np.unique(t)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        p = np.mean(t == v)
        assert abs(p - 1 / 3) < 4 * math.sqrt(2 / 9 / N)
    for q in (Q60, Q40):
        u = core.sample_uniform(core.stream(42, 2, 0), 3, q, N)
        assert int(u.max()) < q
        m = u.astype(np.float64).mean() / q
        assert abs(m - 0.5) < 4 * math.sqrt(1 / 12 / N)


def test_sampler_follows_counter_spec():
    """Every draw is out(stream, coef | residue << 16 | retry << 24)."""
    s0 = core.stream(9, 4, 2)
    assert s0 == core.splitmix_out(core.splitmix_out(9, 4), 2)
    q = Q40
    u = core.sample_uniform(s0, 5, q, 32)
    bound = (2 ** 64 // q) * q
    for c in range(32):
        t = 0
        while True:
            v = core.splitmix_out(s0, c | (5 << 16) | (t << 24))
            if v < bound:
                break
            t += 1
        assert int(u[c]) == v % q
    cdt = params.gauss_cdt()
    g = core.sample_gauss(s0, 32, np.array(cdt, dtype=np.uint64))
    for c in range(32):
        v = core.splitmix_out(s0, c)
        assert int(g[c]) == -19 + sum(1 for T in cdt if v >= T)
    tt = core.sample_ternary(s0, 32)
    for c in range(32):
        v = core.splitmix_out(s0, c)
        assert int(tt[c]) == v % 3 - 1        # no rejection at these indices
