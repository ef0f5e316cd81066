"""The exactness argument of the tensor-core layer MAC, checked on the CPU.

The dense-layer MAC runs as bf16 limb GEMMs with fp32 accumulators: residues
are centred and split into balanced base-256 limbs (five for primes below
2^41, eight below 2^61), limb products are summed per shift class over
32-term chunks, and the class sums are turned into integers with the
1.5 * 2^23 magic constant and added, paired in 32 bits, into 64-bit sums.
These tests check the bounds that make every step exact, at the extremes of
the ranges, with numpy float32 arithmetic standing in for the accumulators."""
import numpy as np
import pytest

CHUNK = 32          # terms per chunk
MAX_TERMS = 8192    # terms per layer the host admits
MAGIC = np.float32(12582912.0)   # 1.5 * 2^23
MAGIC_BITS = 0x4B400000


def limbs(v, n):
    """balanced base-256 limbs: n - 1 digits in [-128, 127] and a top digit"""
    bias = sum(128 << (8 * a) for a in range(n - 1))
    u = v + bias
    span = 1 << (8 * (n - 1))
    low = u % span
    d = [((low >> (8 * a)) & 255) - 128 for a in range(n - 1)]
    d.append((u - low) // span)
    return d


def bf16_exact(x):
    f = np.float32(x)
    return int(f) == x and (int(f.view(np.uint32)) & 0xFFFF) == 0


@pytest.mark.parametrize("n,qbits,top", [(5, 41, 256), (8, 61, 16)])
def test_limbs_reconstruct_and_fit_bf16(n, qbits, top):
    rng = np.random.default_rng(n)
    half = (1 << (qbits - 1)) - 1          # |centred residue| < q/2 < 2^(qbits-1)
    vals = [0, 1, -1, half, -half, 127, -128, 128] + [int(v) for v in rng.integers(-half, half, 2000)]
    for v in vals:
        d = limbs(v, n)
        assert sum(x << (8 * a) for a, x in enumerate(d)) == v
        assert all(-128 <= x <= 127 for x in d[:-1])
        assert abs(d[-1]) <= top
        assert all(bf16_exact(x) for x in d)


@pytest.mark.parametrize("n,top", [(5, 256), (8, 16)])
def test_class_sums_below_2_22(n, top):
    """worst case of every shift class over a chunk: each limb at its bound"""
    bound = [128] * (n - 1) + [top]
    worst = 0
    for s in range(2 * n - 1):
        per_term = sum(bound[a] * bound[s - a] for a in range(n) if 0 <= s - a < n)
        worst = max(worst, per_term * CHUNK)
    assert worst < 1 << 22


def test_magic_conversion_and_pairing_exact():
    lim = (1 << 22) - 1
    rng = np.random.default_rng(3)
    c = rng.integers(-lim, lim + 1, size=(100000, 2)).astype(np.int64)
    c[:4] = [[lim, lim], [-lim, -lim], [lim, -lim], [-lim, lim]]
    f = c.astype(np.float32)
    assert (f.astype(np.int64) == c).all()                 # class sums are exact in fp32
    b = (f + MAGIC).view(np.uint32).astype(np.uint64)
    single = ((b[:, 0] - MAGIC_BITS) & 0xFFFFFFFF).astype(np.uint32).view(np.int32).astype(np.int64)
    assert (single == c[:, 0]).all()
    pair = ((b[:, 0] + (b[:, 1] << 8) - MAGIC_BITS * 257) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    assert (pair.astype(np.int64) == c[:, 0] + 256 * c[:, 1]).all()


@pytest.mark.parametrize("n", [5, 8])
def test_64bit_sums_do_not_overflow(n):
    """A_i = sum_{p<5} C_{5i+p} 2^{8p} summed over every chunk of the largest layer"""
    per_chunk = ((1 << 22) - 1) * sum(1 << (8 * p) for p in range(5))
    chunks = MAX_TERMS // CHUNK
    assert per_chunk * chunks < 1 << 63
    # the recombination covers every class: sum_i A_i 2^{40 i} = sum_s C_s 2^{8 s}
    n_classes = 2 * n - 1
    rng = np.random.default_rng(n)
    C = [int(x) for x in rng.integers(-(1 << 21), 1 << 21, n_classes)]
    A = [sum(C[s] << (8 * (s - 5 * i)) for s in range(5 * i, min(5 * i + 5, n_classes)))
         for i in range((n_classes + 4) // 5)]
    assert sum(a << (40 * i) for i, a in enumerate(A)) == sum(c << (8 * s) for s, c in enumerate(C))


def test_limb_dot_product_equals_modular_product():
    """the whole chain on random residues: limbs -> class sums -> 64-bit sums -> y mod q"""
    rng = np.random.default_rng(7)
    for n, q in [(5, (1 << 40) + 0x1C001), (8, (1 << 60) + 0x8001)]:
        K = 45
        x = [int(v) for v in rng.integers(0, q, K, dtype=np.uint64)]
        w = [int(v) for v in rng.integers(0, q, K, dtype=np.uint64)]
        cen = lambda v: v - q if v > (q - 1) // 2 else v
        xl = [limbs(cen(v), n) for v in x]
        wl = [limbs(cen(v), n) for v in w]
        acc = [0] * ((2 * n - 1 + 4) // 5)
        for c0 in range(0, K, CHUNK):
            for s in range(2 * n - 1):
                cs = sum(xl[e][a] * wl[e][s - a] for e in range(c0, min(c0 + CHUNK, K))
                         for a in range(n) if 0 <= s - a < n)
                assert abs(cs) < 1 << 22
                acc[s // 5] += cs << (8 * (s % 5))
        y = sum(a * pow(2, 40 * i, q) for i, a in enumerate(acc)) % q
        assert y == sum(a * b for a, b in zip(x, w)) % q
