"""Parameter side of the oracle: graph cost discovery, the parameterisation
heuristic, the RNS prime chain, primitive roots and the Gaussian table.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Shares no code with the
CUDA library.

Each function cites the passage of arXiv 2110.13638 it follows.
"""
from decimal import Decimal, getcontext

# ---------------------------------------------------------------------------
# Node costs (Sec. 3.1 "FHE parameterisation": the edge A->B carries the
# computational depth of B).  Encrypt/decrypt nodes are the "type of concern".
# ---------------------------------------------------------------------------
CONCERN_KINDS = ("input", "output", "rotate")


def ingress_nodes(graph):
    """Sources of parameter groups: encrypted inputs and rotations (client
    refresh points), in node order."""
    return [i for i, n in enumerate(graph["nodes"]) if n["kind"] in ("input", "rotate")]


def node_cost(node):
    k = node["kind"]
    if k in ("linear", "square", "conv_packed"):
        return 1
    if k == "poly":
        d = len(node.get("coeffs", (0, 0, 0, 0))) - 1
        if d == 1:
            return 1                                       # affine: one rescale
        if d <= 3:
            return 2
        return (d - 1).bit_length() + 1                    # ceil(log2 d) powers + the combining rescale
    if k == "relu":
        return 2                                         # degree 2 (Eq. relu_approximate)
    return 0


def successors(graph, n):
    """Distinct successors of n in first-edge order (parallel edges collapse)."""
    out = []
    for (a, b) in graph["edges"]:
        if a == n and b not in out:
            out.append(b)
    return out


def autohe_discover(graph, n, s, c, sources):
    """Alg. autoHE_discover: record, at every node reached from source s, the
    largest accumulated cost c; a node of the concern type restarts discovery
    as a new source with cost 0.

    Reading (the printed recursion at a concern node calls itself with the
    same arguments): the restart happens only when the concern node was
    reached from another source (s != n); a concern node that is its own
    source walks on to its successors."""
    d = sources.setdefault(n, {})
    if s != n:
        if d.get(s) is None or d[s] < c:
            d[s] = c
    if graph["nodes"][n]["kind"] in CONCERN_KINDS and s != n:
        autohe_discover(graph, n, n, 0, sources)
    else:
        for i in successors(graph, n):
            nxt = c + node_cost(graph["nodes"][i])
            autohe_discover(graph, i, s, nxt, sources)


def autohe(graph, inputs):
    """Alg. autoHE: label sources and costs, then assign and merge parameter
    groups.  Returns (group_of: dict source-node -> group id,
    group_cost: list group id -> largest cost), plus the per-node source map."""
    sources = {}
    for i in inputs:
        autohe_discover(graph, i, i, 0, sources)
    group_of = {}
    group_cost = []
    for i in inputs:
        if group_of.get(i) is None:
            group_of[i] = len(group_cost)
            group_cost.append(0)
        for j in range(len(graph["nodes"])):
            src = sources.get(j, {})
            if i in src:
                for k in src:
                    group_of[k] = group_of[i]
                    if src[k] > group_cost[group_of[i]]:
                        group_cost[group_of[i]] = src[k]
    return group_of, group_cost, sources


def parameterise(c, s=40, p=1.5):
    """Alg. parameterise: cost c -> MS-SEAL CKKS parameter dict.

    Reading: the printed listing builds the bit list m but never stores it;
    it is returned as parms["coeff_modulus"] (the first and last entries are
    the scale-stabilised outer primes; the last is the special prime)."""
    parms = {}
    parms["scheme"] = 2
    parms["scale"] = pow(2, s)
    m = [s for _ in range(c + 2)]
    m[0] = int(m[0] * p)
    m[-1] = int(m[-1] * p)
    b = 27
    while b < sum(m):
        b = b * 2
    parms["poly_modulus_degree"] = int(1024 * (b / 27))
    parms["coeff_modulus"] = m
    return parms


# ---------------------------------------------------------------------------
# Primes.  Reading: for every bit size b of the list, the primes q > 2^b with
# q = 1 (mod 2N) in increasing order; a size that repeats takes the next one.
# ---------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n):
    """Deterministic Miller-Rabin for n < 3.3e24 (bases: first 12 primes)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_above(b, N, count):
    """The first `count` primes q > 2^b with q = 1 mod 2N, increasing."""
    out = []
    q = (2 ** b // (2 * N)) * (2 * N) + 1
    while q <= 2 ** b:
        q += 2 * N
    while len(out) < count:
        if is_prime(q):
            out.append(q)
        q += 2 * N
    return out


def prime_chain(N, bits):
    """Primes for the bit list `bits` (last entry = special prime P)."""
    need = {}
    for b in bits:
        need[b] = need.get(b, 0) + 1
    pools = {b: primes_above(b, N, k) for b, k in need.items()}
    taken = {b: 0 for b in need}
    chain = []
    for b in bits:
        chain.append(pools[b][taken[b]])
        taken[b] += 1
    return chain


def primitive_2n_root(q, N):
    """Smallest-base primitive 2N-th root: psi = x^((q-1)/2N) with psi^N = -1."""
    assert (q - 1) % (2 * N) == 0
    x = 2
    while True:
        psi = pow(x, (q - 1) // (2 * N), q)
        if pow(psi, N, q) == q - 1:
            return psi
        x += 1


# ---------------------------------------------------------------------------
# Discrete Gaussian table (SEAL default sigma = 3.2; the paper keeps SEAL's
# 128-bit defaults, Sec. 3.1).  Support [-19, 19]; thresholds
# T_i = floor(2^64 * sum_{k=-19}^{-19+i} rho(k) / S), i = 0..37,
# rho(k) = exp(-k^2 / (2 sigma^2)), S = sum over the support.
# Computed with 80 significant decimal digits.
# ---------------------------------------------------------------------------
GAUSS_SIGMA = Decimal("3.2")
GAUSS_KMAX = 19


def gauss_cdt():
    getcontext().prec = 80
    two_s2 = 2 * GAUSS_SIGMA * GAUSS_SIGMA
    ks = list(range(-GAUSS_KMAX, GAUSS_KMAX + 1))
    rho = [(-Decimal(k * k) / two_s2).exp() for k in ks]
    S = sum(rho)
    out = []
    acc = Decimal(0)
    for i in range(2 * GAUSS_KMAX):
        acc += rho[i]
        t = int((acc / S * Decimal(2 ** 64)).to_integral_value(rounding="ROUND_FLOOR"))
        out.append(t)
    return out
