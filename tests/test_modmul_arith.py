"""The Barrett product the library uses for reduced operands (mul_mod_r),
restated with Python integers and checked on the CPU: for every prime size
the chains use (20..61 bits) and operands a, b < q, the quotient estimate
t = floor(floor(a b / 2^(b-1)) mu' / 2^64), mu' = floor(2^(2b) / q) << (63 - b),
lies within 2 below floor(a b / q), so a b - t q is in [0, 3q), fits 64 bits,
and two conditional subtractions give a b mod q."""
import numpy as np
import pytest

from oracle import params

M64 = (1 << 64) - 1


def barrett(a, b, q):
    bl = q.bit_length()
    sh = bl - 1
    mu = ((1 << (2 * bl)) // q) << (63 - bl)
    assert mu <= M64
    x = a * b
    lo, hi = x & M64, x >> 64
    xh = ((hi << (64 - sh)) | (lo >> sh)) & M64
    assert xh == x >> sh                      # the funnel shift loses nothing
    t = (xh * mu) >> 64
    assert 0 <= x // q - t <= 2
    r = (lo - t * q) & M64
    assert r == x - t * q and r < 3 * q < 1 << 64
    for _ in range(2):
        r = r - q if r >= q else r
    return r


def _primes():
    out = []
    for N, bits in ((8192, [60, 40, 40, 60]), (16384, [60] + [40] * 7 + [60]), (1024, [20, 30, 50, 61])):
        out += params.prime_chain(N, bits)
    return out


@pytest.mark.parametrize("q", _primes())
def test_barrett_product_of_reduced_operands(q):
    rng = np.random.default_rng(q & 0xFFFF)
    cases = [(0, 0), (1, 1), (q - 1, q - 1), (q - 1, 1), (q // 2, q // 2 + 1), (q - 2, q - 1)]
    cases += [(int(a), int(b)) for a, b in rng.integers(0, q, size=(2000, 2), dtype=np.uint64)]
    for a, b in cases:
        assert barrett(a, b, q) == a * b % q, (a, b)
