"""Serving with continuous batching: every request's result is the same
whether it is evaluated alone or packed with others into shared batches and
run concurrently with other networks' batches (within 1e-4, the tolerance of
the decrypted outputs), and each matches the FP64 plaintext forward pass."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import __graft_entry__
from oracle import ckks
from paper_2110_13638_gb300 import fhe, serve, workloads as W

pytestmark = pytest.mark.gpu


def _nets():
    __graft_entry__.build()
    torch.cuda.set_device(0)
    out = []
    ctxs = {}
    for name, builder in (("dense_square", W.cfg0), ("mlp", W.cfg2)):
        g, x = builder()
        gof, gcost = fhe.autohe(g)
        N, bits = fhe.parameterise(max(gcost), 40, 1.5)
        if (N, tuple(bits)) not in ctxs:
            c = fhe.Context(N, bits, 40)
            c.keygen(0)
            ctxs[(N, tuple(bits))] = c
        out.append(serve.Network(name, g, x, ctxs[(N, tuple(bits))]))
    return out


def _requests(nets):
    spec = [(0, 1500, 0), (1, 3000, 10), (0, 2500, 20), (0, 700, 30), (1, 6000, 40), (0, 5000, 50)]
    return [serve.Request(i, nets[k], 0.0, n, nets[k].inputs(off, n)) for i, (k, n, off) in enumerate(spec)]


def test_results_alone_equal_results_in_the_mix():
    nets = _nets()
    # alone: one request per run, one slot, no packing
    alone = []
    for r in _requests(nets):
        srv = serve.Server(nets, {"dense_square": 1, "mlp": 1}, 150e9, pack=False, max_inflight=1)
        done, wall, backlog = srv.run([r])
        assert len(done) == 1 and backlog == 0
        alone.append(done[0].y.copy())
        del srv
    # in the mix: all at once, packing and two slots per network
    srv = serve.Server(nets, {"dense_square": 2, "mlp": 2}, 150e9, pack=True)
    reqs = _requests(nets)
    done, wall, backlog = srv.run(reqs)
    assert backlog == 0 and len(done) == len(reqs)
    assert max(r.issued for r in reqs) >= 2          # the 5000-sample request was split across batches
    for r, ya in zip(reqs, alone):
        assert np.max(np.abs(r.y - ya)) < 1e-4, r.rid
        ref = ckks.forward_fp64(r.net.graph, W.input_nodes(r.net.graph), [r.x])
        (node, want), = ref.items()
        assert np.max(np.abs(r.y - want)) < 1e-4, r.rid
