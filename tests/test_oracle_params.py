"""Pins of the oracle's parameter side: Alg. parameterise, Alg. autoHE /
autoHE_discover, the prime chain and the primitive roots."""
import math
import random

import pytest

from oracle import params
from paper_2110_13638_gb300 import workloads as W
import golden_io


# ---------------------------------------------------------------- parameterise
def test_parameterise_matches_stated_parameters():
    for cost, (N, bits) in golden_io.parameterise().items():
        p = params.parameterise(cost, 40, 1.5)
        assert p["poly_modulus_degree"] == N
        assert p["coeff_modulus"] == bits
        assert p["scale"] == 2 ** 40
        assert p["scheme"] == 2


def test_parameterise_stays_inside_128_bit_security():
    """The chosen N always admits the chain under the HE-standard bound."""
    table = golden_io.he_standard()
    for c in range(0, 19):          # c = 19 needs N = 65536, beyond the table
        p = params.parameterise(c)
        N = p["poly_modulus_degree"]
        assert N in table
        assert sum(p["coeff_modulus"]) <= table[N]
        # and N is the smallest power of two that does (for N > 1024)
        if N > 8192:
            assert sum(p["coeff_modulus"]) > table[N // 2] or N // 2 < 8192


def test_parameterise_other_defaults():
    p = params.parameterise(3, 30, 2.0)
    assert p["coeff_modulus"] == [60, 30, 30, 30, 60]
    assert p["poly_modulus_degree"] == 8192     # 210 bits <= 216
    assert params.parameterise(0)["coeff_modulus"] == [60, 60]


# ---------------------------------------------------------------- autoHE
def _depth(graph):
    ins = W.input_nodes(graph)
    group_of, group_cost, _ = params.autohe(graph, ins)
    return group_of, group_cost


@pytest.mark.parametrize("builder,cost", [(W.cfg0, 2), (W.cfg1, 7), (W.cfg2, 7)])
def test_autohe_depth_of_evaluated_networks(builder, cost):
    g, _ = builder(n_slots=4)
    group_of, group_cost = _depth(g)
    assert group_cost == [cost]
    assert params.parameterise(cost)["poly_modulus_degree"] == golden_io.parameterise()[cost][0]


def test_autohe_merges_sources_that_meet():
    """x1 passes two computations, x0 one; they meet, so they share one group
    whose cost is the longer path (linear+linear+square = 3)."""
    g, _ = W.branch_graph(4)
    group_of, group_cost = _depth(g)
    assert group_of[0] == group_of[1]
    assert group_cost == [3]


def test_autohe_separates_disjoint_graphs():
    g0, _ = W.cfg0(n_slots=4)              # cost 2
    g2, _ = W.cfg2(n_slots=4)              # cost 7
    off = len(g0["nodes"])
    g = {"nodes": g0["nodes"] + g2["nodes"],
         "edges": g0["edges"] + [(a + off, b + off) for a, b in g2["edges"]]}
    group_of, group_cost = _depth(g)
    assert group_of[0] != group_of[off]
    assert sorted(group_cost) == [2, 7]
    assert group_cost[group_of[0]] == 2 and group_cost[group_of[off]] == 7


def test_autohe_restarts_at_concern_nodes():
    """A decrypt node with successors (a key rotation) starts a new source
    with cost 0: the input's group only counts up to it."""
    lin = {"kind": "linear"}
    nodes = [{"kind": "input"}, lin, lin, {"kind": "output"}, lin, {"kind": "poly"}, {"kind": "output"}]
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    g = {"nodes": nodes, "edges": edges}
    group_of, group_cost, sources = params.autohe(g, [0])
    assert group_cost == [2]
    assert sources[3] == {0: 2}
    assert sources[6] == {3: 3}       # linear + poly after the rotation
    assert 0 not in sources[6]


def test_autohe_takes_longest_of_parallel_paths():
    lin, sq = {"kind": "linear"}, {"kind": "square"}
    nodes = [{"kind": "input"}, lin, sq, sq, {"kind": "add"}, {"kind": "output"}]
    # 0 -> 1 -> 4 and 0 -> 2 -> 3 -> 4 (parallel edge 1->4 twice)
    edges = [(0, 1), (1, 4), (1, 4), (0, 2), (2, 3), (3, 4), (4, 5)]
    _, group_cost, sources = params.autohe({"nodes": nodes, "edges": edges}, [0])
    assert group_cost == [2]
    assert sources[4] == {0: 2}


# ---------------------------------------------------------------- primes
def _pollard_rho(n):
    if n % 2 == 0:
        return 2
    rnd = random.Random(n)
    while True:
        x = y = rnd.randrange(2, n)
        c = rnd.randrange(1, n)
        d = 1
        while d == 1:
            x = (x * x + c) % n
            y = (y * y + c) % n
            y = (y * y + c) % n
            d = math.gcd(abs(x - y), n)
        if d != n:
            return d


def _trial_prime(n):
    if n < 2:
        return False
    i = 2
    while i * i <= n:
        if n % i == 0:
            return False
        i += 1
    return True


def _factor(n, out):
    """Full factorisation: trial division by small numbers, then Pollard rho;
    a cofactor that passes a Fermat test is certified prime by Lucas."""
    d = 2
    while d < 10000 and d * d <= n:
        while n % d == 0:
            out.append(d)
            n //= d
        d += 1
    if n == 1:
        return
    if n < 10 ** 8:
        out.append(n)            # no factor below 10^4 and n < 10^8: prime
        return
    if pow(2, n - 1, n) == 1 and _lucas_certify(n):
        out.append(n)
        return
    d = _pollard_rho(n)
    _factor(d, out)
    _factor(n // d, out)


def _lucas_certify(n):
    """Lucas primality proof: some a has a^(n-1) = 1 and a^((n-1)/p) != 1 for
    every prime p | n-1 (needs the full factorisation of n-1)."""
    if n < 2 ** 32:
        return _trial_prime(n)
    fs = []
    _factor(n - 1, fs)
    ps = sorted(set(fs))
    assert math.prod(fs) == n - 1
    for a in range(2, 200):
        if pow(a, n - 1, n) != 1:
            return False           # Fermat witness: composite
        if all(pow(a, (n - 1) // p, n) != 1 for p in ps):
            return True
    return False


def test_prime_chain_golden_and_certified():
    gold = golden_io.primes()
    for N, chain in gold.items():
        bits = [60] + [40] * (len(chain) - 2) + [60]
        assert params.prime_chain(N, bits) == chain
        for q in chain:
            assert q % (2 * N) == 1
            assert _lucas_certify(q)
        assert len(set(chain)) == len(chain)


def test_prime_chain_is_smallest_above():
    """No prime = 1 mod 2N lies between 2^b and the first chosen prime, nor
    between successive chosen primes of one size (Fermat witnesses)."""
    N = 8192
    chain = golden_io.primes()[N]
    for b, lo_hi in ((60, (2 ** 60, chain[-1])), (40, (2 ** 40, chain[2]))):
        lo, hi = lo_hi
        x = (lo // (2 * N)) * (2 * N) + 1
        if x <= lo:
            x += 2 * N
        found = []
        while x <= hi:
            if pow(2, x - 1, x) == 1 and _lucas_certify(x):
                found.append(x)
            x += 2 * N
        if b == 60:
            assert found == [chain[0], chain[-1]]
        else:
            assert found == [chain[1], chain[2]]


def test_miller_rabin_against_trial_division():
    rnd = random.Random(5)
    for _ in range(300):
        n = rnd.randrange(2, 10 ** 6)
        assert params.is_prime(n) == _trial_prime(n)
    # strong pseudoprimes to several bases
    for n in (2047, 1373653, 3215031751, 2152302898747, 3474749660383, 341550071728321):
        assert not params.is_prime(n)


@pytest.mark.parametrize("N", [16, 1024, 8192, 16384])
def test_primitive_root(N):
    bits = [60, 40, 40, 60]
    for q in params.prime_chain(N, bits):
        psi = params.primitive_2n_root(q, N)
        assert pow(psi, N, q) == q - 1
        assert pow(psi, 2 * N, q) == 1
