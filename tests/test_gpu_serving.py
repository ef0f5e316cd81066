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
    for name, builder in (("dense_square", W.cfg0), ("cnn", W.cfg1), ("mlp", W.cfg2)):
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
    spec = [(0, 1500, 0), (2, 3000, 10), (1, 2000, 60), (0, 2500, 20), (0, 700, 30), (2, 6000, 40),
            (1, 7000, 70), (0, 5000, 50)]
    return [serve.Request(i, nets[k], 0.0, n, nets[k].inputs(off, n)) for i, (k, n, off) in enumerate(spec)]


def test_results_alone_equal_results_in_the_mix():
    nets = _nets()
    # alone: one request per run, one slot, no packing
    alone = []
    for r in _requests(nets):
        srv = serve.Server(nets, {"dense_square": 1, "cnn": 1, "mlp": 1}, 150e9, pack=False, max_inflight=1)
        done, wall, backlog = srv.run([r])
        assert len(done) == 1 and backlog == 0
        alone.append(done[0].y.copy())
        del srv
    # in the mix: all at once, packing and two slots per network
    srv = serve.Server(nets, {"dense_square": 2, "cnn": 2, "mlp": 2}, 150e9, pack=True)
    reqs = _requests(nets)
    done, wall, backlog = srv.run(reqs)
    assert backlog == 0 and len(done) == len(reqs)
    assert max(r.issued for r in reqs) >= 2          # a request was split across batches
    for r, ya in zip(reqs, alone):
        assert np.max(np.abs(r.y - ya)) < 1e-4, r.rid
        ref = ckks.forward_fp64(r.net.graph, W.input_nodes(r.net.graph), [r.x])
        (node, want), = ref.items()
        assert np.max(np.abs(r.y - want)) < 1e-4, r.rid


def test_eval_batch_equals_the_separate_calls():
    """fhe_eval_batch (gather, encode+encrypt, graph, decrypt, decode,
    scatter in one call) gives exactly what the separate entry points give on
    the packed slots; host (pinned) request buffers give the same."""
    __graft_entry__.build()
    torch.cuda.set_device(0)
    N = 1024
    c = fhe.Context(N, [60] + [40] * 7 + [60], 40)
    c.keygen(0)
    graph, x = W.mini_cnn(n_slots=N // 2)
    G = fhe.Graph(graph)
    n_out, L_out = G.outputs(c)
    sizes, offs = [100, 7, 300], [0, 100, 107]
    xs = [torch.tensor(x[:, o:o + n], device="cuda") for n, o in zip(sizes, offs)]
    ys = [torch.full((n_out, n), -7.0, dtype=torch.float64, device="cuda") for n in sizes]
    G.eval_batch(c, list(zip(xs, ys)), 500)
    # the same steps one call at a time
    slots = torch.zeros((x.shape[0], N // 2), dtype=torch.float64, device="cuda")
    slots[:, :407] = torch.tensor(x[:, :407], device="cuda")
    ct = c.empty_ct(x.shape[0], c.L_top)
    c.encode_encrypt(slots, c.delta, 500, ct)
    out = c.empty_ct(n_out, L_out)
    meta = G.eval(c, [ct], out)
    m = torch.empty((n_out, N), dtype=torch.int64, device="cuda")
    c.decrypt(out, L_out, m)
    z = torch.empty((n_out, N // 2), dtype=torch.float64, device="cuda")
    c.decode(m, meta[0][1], z)
    torch.cuda.synchronize()
    for y, n, o in zip(ys, sizes, offs):
        assert torch.equal(y, z[:, o:o + n])
    ref = ckks.forward_fp64(graph, W.input_nodes(graph), [x[:, :407]])
    (node, want), = ref.items()
    got = torch.cat(ys, dim=1).cpu().numpy()
    assert np.max(np.abs(got - want)) < 1e-4
    # pinned host buffers, wider strides (only the first n columns used)
    hx = [torch.zeros((x.shape[0], n + 5), dtype=torch.float64).pin_memory() for n in sizes]
    hy = [torch.zeros((n_out, n + 3), dtype=torch.float64).pin_memory() for n in sizes]
    for h, n, o in zip(hx, sizes, offs):
        h[:, :n] = torch.tensor(x[:, o:o + n])
    G.eval_batch(c, [(a, b, n) for a, b, n in zip(hx, hy, sizes)], 500)
    torch.cuda.synchronize()
    for h, y, n in zip(hy, ys, sizes):
        assert torch.equal(h[:, :n], y.cpu())
    # more samples than slots
    big = torch.zeros((x.shape[0], N // 2 + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(fhe.FheError):
        G.eval_batch(c, [(big, torch.zeros((n_out, N // 2 + 1), dtype=torch.float64, device="cuda"))], 0)
    G.close()
    c.close()


def test_admission_cap_binds():
    """Slots beyond the admission cap are not created: with a cap below one
    slot's footprint each network keeps only its first slot."""
    nets = _nets()
    srv = serve.Server(nets, {"dense_square": 3, "cnn": 3, "mlp": 3}, 1.0, pack=True)
    assert {k: len(v) for k, v in srv.slots.items()} == {"dense_square": 1, "cnn": 1, "mlp": 1}
    assert srv.footprint > 1.0
    roomy = serve.Server(nets[:1], {"dense_square": 3}, 150e9, pack=True)
    assert len(roomy.slots["dense_square"]) == 3
