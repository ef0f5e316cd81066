"""Pins of the oracle's canonical-embedding encode / decode (binary128)."""
import cmath
import math

import numpy as np
import pytest

from oracle import core

DELTA = 2.0 ** 40


def _direct_coeffs(z, N, scale):
    """m_k = scale * (2/N) * Re sum_j z_j zeta_j^{-k}, zeta_j = e^{i pi 5^j / N},
    summed in double precision (O(N^2))."""
    out = []
    roots = [pow(5, j, 2 * N) for j in range(N // 2)]
    for k in range(N):
        s = 0j
        for j, e in enumerate(roots):
            s += z[j] * cmath.exp(-1j * math.pi * e * k / N)
        out.append(scale * 2.0 / N * s.real)
    return out


def test_encode_constant_vector_closed_form():
    for N in (16, 1024, 8192):
        for c in (0.25, -0.7, 1.0, 3.5):
            m = core.encode(np.full(N // 2, c), N, DELTA)
            want = np.zeros(N, dtype=np.int64)
            want[0] = round(c * DELTA)
            assert np.array_equal(m, want)


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_encode_matches_direct_sum(N):
    rng = np.random.default_rng(N)
    z = rng.uniform(-1, 1, N // 2)
    m, frac = core.encode(z, N, DELTA, want_frac=True)
    ref = _direct_coeffs(z, N, DELTA)
    for k in range(N):
        assert abs(float(m[k]) - ref[k]) <= 0.5 + 1e-3
        if frac[k] > 1e-3:        # away from a rounding boundary: exact agreement
            assert int(m[k]) == int(math.floor(abs(ref[k]) + 0.5)) * (1 if ref[k] >= 0 else -1)


@pytest.mark.parametrize("N", [64, 4096, 16384])
def test_decode_inverts_encode(N):
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, N // 2)
    m = core.encode(z, N, DELTA)
    re, im = core.decode(m, N, DELTA)
    # rounding error per coefficient <= 1/2, so slot error <= N/2 / DELTA
    assert np.max(np.abs(re - z)) <= N / 2 / DELTA
    assert np.max(np.abs(im)) <= N / 2 / DELTA


def test_decode_matches_direct_evaluation():
    N = 32
    rng = np.random.default_rng(4)
    m = rng.integers(-2 ** 40, 2 ** 40, size=N)
    re, im = core.decode(m, N, 1.0)
    for j in range(N // 2):
        zeta = cmath.exp(1j * math.pi * pow(5, j, 2 * N) / N)
        v = sum(int(m[k]) * zeta ** k for k in range(N))
        # double-precision direct sum: error well below 1e-9 * 2^40 * N
        assert abs(v.real - re[j]) < 1e-9 * 2 ** 40 * N
        assert abs(v.imag - im[j]) < 1e-9 * 2 ** 40 * N


def test_embedding_is_a_ring_homomorphism():
    """The negacyclic product of two encodings decodes to the slot-wise product:
    pins the slot order (5^j) and the sign of X^N = -1."""
    N = 64
    rng = np.random.default_rng(6)
    z1 = rng.uniform(-1, 1, N // 2)
    z2 = rng.uniform(-1, 1, N // 2)
    s = 2.0 ** 20
    m1 = [int(v) for v in core.encode(z1, N, s)]
    m2 = [int(v) for v in core.encode(z2, N, s)]
    prod = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                prod[k] += m1[i] * m2[j]
            else:
                prod[k - N] -= m1[i] * m2[j]
    re, _ = core.decode(np.array(prod, dtype=np.int64), N, s * s)
    assert np.max(np.abs(re - z1 * z2)) < 1e-4
