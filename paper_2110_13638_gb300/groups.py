"""Evaluation of a network graph across parameter groups (rotation nodes).

Alg. autoHE over the ingress nodes (encrypted inputs and rotations) gives the
parameter groups and their costs; Alg. parameterise gives each group its ring
and modulus chain.  A rotation (Sec. 3.1 "key-rotation stages") is a client
refresh: the ciphertexts reaching it are decrypted and decoded under the
upstream group's keys and encoded and encrypted under the rotation's own
group, so every group needs only its own depth.

Each group is evaluated by the library (fhe_eval_graph) on a subgraph: its
ingress nodes become INPUT nodes, the concern nodes where it ends (outputs
and rotations) become OUTPUT nodes.  Every step runs on the device through
the C ABI; this module only splits the graph and routes the buffers.

Ciphertext ids: input node n, ciphertext i -> first_ct_id + (n << 20) + i;
rotation node n, ciphertext i -> 2^40 + (n << 20) + i.
"""
import numpy as np

from . import fhe

REFRESH_BASE = 1 << 40


def refresh_ct_id(node, k):
    return REFRESH_BASE + (node << 20) + k


def _out_side(geo, side):
    return (geo[side] - geo["k"]) // geo["stride"] + 1


def _relayout_index(geo, n_in, m_up, m_down):
    """Gather table of the client's re-packing after a packed convolution:
    decoded filter ciphertexts [F * n_in][m_up] (filter-major) -> one row per
    feature f * OH * OW + r * OW + c, image i * images + b in column
    (m_down columns, -1 = zero)."""
    F, imgs, S, W, st = geo["filters"], geo["images"], geo["slot_stride"], geo["W"], geo["stride"]
    OH, OW = _out_side(geo, "H"), _out_side(geo, "W")
    if n_in * imgs > m_down:
        raise ValueError("%d images do not fit %d slots after the refresh" % (n_in * imgs, m_down))
    idx = np.full((F * OH * OW, m_down), -1, dtype=np.int64)
    for f in range(F):
        for r in range(OH):
            for c in range(OW):
                row = f * OH * OW + r * OW + c
                for i in range(n_in):
                    for b in range(imgs):
                        idx[row, i * imgs + b] = (f * n_in + i) * m_up + b * S + st * r * W + st * c
    return idx


def _succ(graph, n):
    return [b for a, b in graph["edges"] if a == n]


def _counts(graph):
    """Number of ciphertexts each node emits (stacked in-edges, edge order)."""
    nodes, edges = graph["nodes"], graph["edges"]
    cnt = {}
    pending = list(range(len(nodes)))
    while pending:
        progress = False
        for n in list(pending):
            ins = [a for a, b in edges if b == n]
            if any(a not in cnt for a in ins):
                continue
            k = nodes[n]["kind"]
            if k == "input":
                c = int(nodes[n]["n"])
            elif k == "linear":
                c = len(nodes[n]["row_ptr"]) - 1
            elif k == "add":
                c = cnt[ins[0]]
            elif k == "conv_packed":
                c = int(nodes[n]["filters"]) * sum(cnt[a] for a in ins)
            elif k == "rotate" and "relayout" in nodes[n]:
                g = nodes[n]["relayout"]
                c = g["filters"] * _out_side(g, "H") * _out_side(g, "W")
            else:
                c = sum(cnt[a] for a in ins)
            cnt[n] = c
            pending.remove(n)
            progress = True
        if not progress:
            raise ValueError("graph has a cycle without a concern node")
    return cnt


class GroupedNetwork:
    """A graph with rotation nodes, one context per parameter group.

    contexts: optional {group: fhe.Context} (keys generated); by default each
    group gets Context(*parameterise(cost)) with keygen(seed + group)."""

    def __init__(self, graph, seed=0, log_scale=40, special_mult=1.5, contexts=None):
        self.graph = graph
        nodes = graph["nodes"]
        self.ingress = [i for i, n in enumerate(nodes) if n["kind"] in ("input", "rotate")]
        gof, gcost = fhe.autohe(graph)
        self.group_of = dict(zip(self.ingress, gof))
        self.group_cost = gcost
        self.counts = _counts(graph)
        # ciphertexts arriving at each node (its in-edges stacked); a sink's
        # arrivals are what its group hands over
        self.arrivals = {n: sum(self.counts[a] for a, b in graph["edges"] if b == n) for n in range(len(nodes))}
        if contexts is None:
            contexts = {}
            for g, c in enumerate(gcost):
                N, bits = fhe.parameterise(c, log_scale, special_mult)
                ctx = fhe.Context(N, bits, log_scale)
                ctx.keygen(seed + g)
                contexts[g] = ctx
        self.ctx = contexts
        # nodes of each group: reached from its ingress without passing a concern node
        self.members = {g: set() for g in range(len(gcost))}
        self.sinks = {g: [] for g in range(len(gcost))}
        for i in self.ingress:
            g = self.group_of[i]
            stack = [i]
            self.members[g].add(i)
            while stack:
                n = stack.pop()
                for b in _succ(graph, n):
                    if b in self.members[g]:
                        continue
                    self.members[g].add(b)
                    if nodes[b]["kind"] in ("output", "rotate"):
                        if b not in self.sinks[g]:
                            self.sinks[g].append(b)
                    else:
                        stack.append(b)
        for g in self.sinks:
            self.sinks[g].sort()
        # order: a group runs after the groups that feed its rotations
        self.order = []
        done = set()
        while len(self.order) < len(gcost):
            moved = False
            for g in range(len(gcost)):
                if g in done:
                    continue
                feeders = {h for h in range(len(gcost)) for r in self.sinks[h]
                           if nodes[r]["kind"] == "rotate" and self.group_of.get(r) == g and h != g}
                if feeders <= done:
                    self.order.append(g)
                    done.add(g)
                    moved = True
            if not moved:
                raise ValueError("rotation groups depend on each other cyclically")
        self.sub = {g: self._subgraph(g) for g in range(len(gcost))}
        self._relayout = {}          # rotation node -> device gather table
        self.G = {g: fhe.Graph(self.sub[g][0]) for g in range(len(gcost))}
        self.last_ingress = {}
        self.last_sinks = {}

    def _subgraph(self, g):
        nodes = self.graph["nodes"]
        ing = [i for i in self.ingress if self.group_of[i] == g]
        keep = sorted(self.members[g])
        idx = {n: k for k, n in enumerate(keep)}
        sub_nodes = []
        for n in keep:
            if n in ing:
                sub_nodes.append({"kind": "input", "n": self.counts[n]})
            elif n in self.sinks[g]:
                sub_nodes.append({"kind": "output"})
            else:
                sub_nodes.append(nodes[n])
        sub_edges = [(idx[a], idx[b]) for a, b in self.graph["edges"]
                     if a in idx and b in idx and a not in self.sinks[g] and b not in ing]
        return {"nodes": sub_nodes, "edges": sub_edges}, ing

    def evaluate(self, inputs, first_ct_id=0, stream=None):
        """inputs: per INPUT node (node order), float64 device tensor
        [n_ct][N/2] of the group's ring.  Returns {output node: float64 device
        tensor [n_ct][N/2]} of decoded results."""
        import torch
        nodes = self.graph["nodes"]
        in_nodes = [i for i in self.ingress if nodes[i]["kind"] == "input"]
        slots_of = dict(zip(in_nodes, inputs))
        results = {}
        self.last_ingress, self.last_sinks = {}, {}
        for g in self.order:
            ctx, G = self.ctx[g], self.G[g]
            sub, ing = self.sub[g]
            cts = []
            for i in ing:
                z = slots_of[i]
                if z.shape[1] != ctx.N // 2:
                    if nodes[i]["kind"] == "input" or z.shape[1] > ctx.N // 2:
                        raise ValueError("node %d carries %d slots; its group's ring holds %d"
                                         % (i, z.shape[1], ctx.N // 2))
                    # smaller ring upstream: the client widens each row with zeros
                    m_up, m_dn = z.shape[1], ctx.N // 2
                    idx = np.full((z.shape[0], m_dn), -1, dtype=np.int64)
                    idx[:, :m_up] = np.arange(z.shape[0] * m_up, dtype=np.int64).reshape(z.shape[0], m_up)
                    wide = torch.empty((z.shape[0], m_dn), dtype=torch.float64, device=z.device)
                    fhe.gather_slots(z.contiguous(), torch.tensor(idx, device=z.device), z.shape[0], m_dn, wide, stream)
                    z = wide
                first = first_ct_id + (i << 20) if nodes[i]["kind"] == "input" else refresh_ct_id(i, 0)
                ct = ctx.empty_ct(z.shape[0], ctx.L_top)
                ctx.encode_encrypt(z, ctx.delta, first, ct, stream)
                cts.append(ct)
                self.last_ingress[i] = ct
            n_out, L_out = G.outputs(ctx)
            out = ctx.empty_ct(n_out, L_out)
            meta = G.eval(ctx, cts, out, stream)
            m = torch.empty((n_out, ctx.N), dtype=torch.int64, device=out.device)
            ctx.decrypt(out, L_out, m, stream)
            z = torch.empty((n_out, ctx.N // 2), dtype=torch.float64, device=out.device)
            a = 0
            while a < n_out:                        # decode each run of equal scales
                b = a + 1
                while b < n_out and meta[b][1] == meta[a][1]:
                    b += 1
                ctx.decode(m[a:b], meta[a][1], z[a:b], stream)
                a = b
            off = 0
            for s in self.sinks[g]:
                k = self.arrivals[s]
                self.last_sinks[s] = (out[off:off + k], L_out, [mm[1] for mm in meta[off:off + k]])
                if nodes[s]["kind"] == "rotate":
                    zs = z[off:off + k]              # client refresh: re-encrypted by the next group
                    if "relayout" in nodes[s]:       # client re-packs the decoded slots
                        geo = nodes[s]["relayout"]
                        down = self.ctx[self.group_of[s]]
                        rows = self.counts[s]
                        if s not in self._relayout:
                            idx = _relayout_index(geo, k // geo["filters"], zs.shape[1], down.N // 2)
                            self._relayout[s] = torch.tensor(idx, device=zs.device)
                        dst = torch.empty((rows, down.N // 2), dtype=torch.float64, device=zs.device)
                        fhe.gather_slots(zs.contiguous(), self._relayout[s], rows, down.N // 2, dst, stream)
                        zs = dst
                    slots_of[s] = zs
                else:
                    results[s] = z[off:off + k]
                off += k
        return results

    def close(self):
        for G in self.G.values():
            G.close()
