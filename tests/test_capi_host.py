"""CPU checks of the C ABI: the library builds and exports every symbol that
include/fhe.h declares, and its host-only logic (Alg. parameterise, Alg.
autoHE, prime chains, the Gaussian table) agrees with the oracle.  No device
computation runs here."""
import os
import re

import pytest

import __graft_entry__
from oracle import params
from paper_2110_13638_gb300 import fhe, workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fhe.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(fhe_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert len(names) >= 25
    L = fhe.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fhe.SIGNATURES), "binding and header disagree"


def test_parameterise_matches_oracle():
    for c in range(0, 19):
        N, bits = fhe.parameterise(c, 40, 1.5)
        p = params.parameterise(c, 40, 1.5)
        assert N == p["poly_modulus_degree"] and bits == p["coeff_modulus"]


@pytest.mark.parametrize("N", [16, 1024, 8192, 16384])
def test_prime_chain_matches_oracle(N):
    bits = [60, 40, 40, 40, 40, 60]
    assert fhe.prime_chain(N, bits) == params.prime_chain(N, bits)


def test_gaussian_table_matches_oracle():
    assert fhe.gauss_table() == params.gauss_cdt()


@pytest.mark.parametrize("builder", [W.cfg0, W.cfg1, W.cfg2, W.cnn_relu, W.mini_cnn_relu, W.deep_mlp, W.poly_chain])
def test_autohe_matches_oracle(builder):
    g, _ = builder(n_slots=4)
    gof, gcost = fhe.autohe(g)
    o_gof, o_cost, _ = params.autohe(g, W.input_nodes(g))
    assert gcost == o_cost
    assert gof == [o_gof[i] for i in W.input_nodes(g)]


def test_autohe_groups_rotation_nodes():
    from oracle import params as P
    g, _ = W.mini_cnn_rotate(4)
    gof, gcost = fhe.autohe(g)
    o_gof, o_cost, _ = P.autohe(g, P.ingress_nodes(g))
    assert gcost == o_cost == [3, 4]
    assert gof == [o_gof[i] for i in P.ingress_nodes(g)]
    g, _ = W.cnn_rotate(4)
    assert fhe.autohe(g)[1] == [3, 4]


def test_autohe_branches_and_disjoint():
    g, _ = W.branch_graph(4)
    assert fhe.autohe(g) == ([0, 0], [3])
    g0, _ = W.cfg0(n_slots=4)
    g2, _ = W.cfg2(n_slots=4)
    off = len(g0["nodes"])
    g = {"nodes": g0["nodes"] + g2["nodes"],
         "edges": g0["edges"] + [(a + off, b + off) for a, b in g2["edges"]]}
    assert fhe.autohe(g) == ([0, 1], [2, 7])


@pytest.mark.parametrize("builder", [W.cfg0, W.cfg1, W.cfg2, W.deep_mlp, W.branch_graph, W.cnn_relu,
                                     W.mini_cnn_relu])
def test_autoparam_matches_oracle(builder):
    g, _ = builder(n_slots=4)
    _, o_cost, _ = params.autohe(g, W.input_nodes(g))
    G = fhe.Graph(g)
    p = params.parameterise(max(o_cost), 40, 1.5)
    assert G.autoparam(40, 1.5) == (p["poly_modulus_degree"], p["coeff_modulus"])
    G.close()


def test_autoparam_takes_the_largest_group():
    g0, _ = W.cfg0(n_slots=4)
    g2, _ = W.cfg2(n_slots=4)
    off = len(g0["nodes"])
    g = {"nodes": g0["nodes"] + g2["nodes"],
         "edges": g0["edges"] + [(a + off, b + off) for a, b in g2["edges"]]}
    G = fhe.Graph(g)
    p = params.parameterise(7, 40, 1.5)
    assert G.autoparam() == (p["poly_modulus_degree"], p["coeff_modulus"])
    G.close()


def test_host_errors_are_reported():
    with pytest.raises(fhe.FheError) as e:
        fhe.prime_chain(1000, [60, 40])
    assert e.value.code == -1
    with pytest.raises(fhe.FheError):
        fhe.prime_chain(1024, [70, 40])


def test_health_hooks_reject_null_outputs():
    """fhe_device_faults and fhe_launch_count check their output pointer
    before touching the device."""
    lib = fhe.lib()
    assert lib.fhe_device_faults(None) == -1
    assert lib.fhe_launch_count(None) == -1
