"""Continuous-batching server for encrypted inference (host loop over libfhe).

Requests of several networks arrive over time; each network belongs to a
parameter set (Alg. autoHE / parameterise of its graph) whose context holds
the relinearisation keys, resident on the device for the whole run.  Each
network gets serving slots: a fork of its parameter set's context (shared
tables and keys, own workspace), a CUDA stream, a graph handle and device /
pinned host buffers sized for one batch.  Slots are created while the total
device footprint stays under the admission cap.

Scheduling: waiting requests of a network are packed into the free slot
ranges of one batch (batch-in-slots: a request of n samples takes n
consecutive slots of the shared ciphertexts; one that does not fit a batch
is split across batches and completes with its last part).  A batch is one
native call (fhe_eval_batch: gather -> encode+encrypt -> graph -> decrypt ->
decode -> scatter) on its slot's stream; batches on different slots overlap
on the device.  New requests are admitted as
slots free up, without waiting for other batches (continuous batching).
Latency = completion time - arrival time.

The serial baseline uses one slot at a time and no packing.
"""
import time
from collections import deque

import numpy as np

from . import fhe


class Network:
    """One servable network: graph, parameter set, slot capacity."""

    def __init__(self, name, graph, data, ctx):
        self.name = name
        self.graph = graph
        self.data = data                     # [n_in][pool] float64 input pool
        self.ctx = ctx                       # parameter-set context with keys
        self.n_in = data.shape[0]
        self.capacity = ctx.slots            # samples per batch

    def inputs(self, offset, n):
        pool = self.data.shape[1]
        idx = (np.arange(n) + offset) % pool
        return self.data[:, idx]


class Slot:
    def __init__(self, net, torch):
        self.net = net
        self.ctx = net.ctx.fork()
        self.stream = torch.cuda.Stream()
        self.G = fhe.Graph(net.graph)
        n_out, L_out = self.G.outputs(self.ctx)
        self.n_out, self.L_out = n_out, L_out
        cap = net.capacity
        self.host_in = torch.zeros((net.n_in, cap), dtype=torch.float64).pin_memory()
        self.host_out = torch.zeros((n_out, cap), dtype=torch.float64).pin_memory()
        self.event = torch.cuda.Event()
        self.batch = None

    def launch(self, batch, torch, ct_base):
        """batch: list of (request, part offset in the request, slot offset, n),
        slot offsets consecutive from 0.  One fhe_eval_batch call: each part's
        columns go from pinned staging to the device and its outputs come back
        to pinned staging, all on this slot's stream."""
        hin = self.host_in.numpy()
        reqs = []
        for req, roff, soff, n in batch:
            hin[:, soff:soff + n] = req.x[:, roff:roff + n]
            reqs.append((self.host_in[:, soff:], self.host_out[:, soff:], n))
        self.batch = batch
        self.G.eval_batch(self.ctx, reqs, ct_base, stream=self.stream)
        self.event.record(self.stream)

    def done(self):
        return self.batch is not None and self.event.query()


class Request:
    __slots__ = ("rid", "net", "arrival", "n", "x", "done_parts", "issued", "finish", "y", "next_off")

    def __init__(self, rid, net, arrival, n, x):
        self.rid, self.net, self.arrival, self.n, self.x = rid, net, arrival, n, x
        self.issued = 0          # parts handed to batches
        self.done_parts = 0
        self.finish = None
        self.next_off = 0        # first sample not yet handed to a batch
        self.y = None


class Server:
    def __init__(self, nets, slots_per_net, cap_bytes, pack=True, max_inflight=None):
        import torch
        self.torch = torch
        self.nets = nets
        self.pack = pack
        self.max_inflight = max_inflight
        self.slots = {n.name: [] for n in nets}
        self.footprint = 0
        free0, _ = torch.cuda.mem_get_info()
        for n in nets:
            for _ in range(slots_per_net.get(n.name, 1)):
                before, _ = torch.cuda.mem_get_info()
                s = Slot(n, torch)
                self._warm(s)
                after, _ = torch.cuda.mem_get_info()
                cost = before - after
                if self.footprint + cost > cap_bytes and self.slots[n.name]:
                    del s
                    break
                self.footprint += cost
                self.slots[n.name].append(s)
        self.queues = {n.name: deque() for n in nets}
        self.ct_counter = 1 << 40

    def _warm(self, s):
        """one full batch so the slot's workspace, batch area and graph
        constants exist before it is counted against the cap"""
        dummy = Request(-1, s.net, 0.0, s.net.capacity, np.zeros((s.net.n_in, s.net.capacity)))
        s.launch([(dummy, 0, 0, s.net.capacity)], self.torch, 0)
        s.stream.synchronize()
        s.batch = None

    def submit(self, req):
        self.queues[req.net.name].append(req)

    def _form_batch(self, q, cap):
        batch, used = [], 0
        while q and used < cap:
            req = q[0]
            left = req.n - req.next_off
            take = min(left, cap - used)
            batch.append((req, req.next_off, used, take))
            req.next_off += take
            req.issued += 1
            used += take
            if req.next_off >= req.n:
                q.popleft()
            if not self.pack:
                break
        return batch

    def inflight(self):
        return sum(1 for v in self.slots.values() for s in v if s.batch is not None)

    def poll(self, now_fn, completed):
        for slots in self.slots.values():
            for s in slots:
                if s.done():
                    s.ctx.sync(s.stream)          # raises if a kernel of the batch gave up a device wait
                    t = now_fn()
                    out = s.host_out.numpy()
                    for req, roff, soff, n in s.batch:
                        if req.y is None:
                            req.y = np.zeros((s.n_out, req.n))
                        req.y[:, roff:roff + n] = out[:, soff:soff + n]
                        req.done_parts += 1
                        if req.next_off >= req.n and req.done_parts == req.issued:
                            req.finish = t
                            completed.append(req)
                    s.batch = None

    def dispatch(self):
        launched = 0
        # oldest waiting request first across networks
        order = sorted((q[0].arrival, name) for name, q in self.queues.items() if q)
        for _, name in order:
            for s in self.slots[name]:
                if self.max_inflight is not None and self.inflight() >= self.max_inflight:
                    return launched
                if s.batch is not None or not self.queues[name]:
                    continue
                batch = self._form_batch(self.queues[name], s.net.capacity)
                if batch:
                    s.launch(batch, self.torch, self.ct_counter)
                    self.ct_counter += s.net.n_in
                    launched += 1
        return launched

    def run(self, requests, horizon=None):
        """Replay `requests` (sorted by arrival, seconds from start) in real
        time; stop admitting after `horizon` seconds (all if None) and wait
        for the batches in flight.  Returns (completed, wall seconds, backlog)."""
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        completed = []
        i = 0
        while True:
            t = now()
            stop_admit = horizon is not None and t > horizon
            while i < len(requests) and requests[i].arrival <= t and not stop_admit:
                self.submit(requests[i])
                i += 1
            before = len(completed)
            self.poll(now, completed)
            launched = 0 if stop_admit else self.dispatch()
            arrivals_left = i < len(requests) and not stop_admit
            waiting = any(self.queues.values()) and not stop_admit
            if not arrivals_left and not waiting and self.inflight() == 0:
                break
            if launched == 0 and len(completed) == before:
                time.sleep(0.0002)
        wall = now()
        backlog = sum(len(q) for q in self.queues.values()) + (len(requests) - i)
        return completed, wall, backlog


def latency_stats(completed, wall):
    if not completed:
        return {"completed": 0}
    lat = np.array([(r.finish - r.arrival) * 1000.0 for r in completed])
    samples = sum(r.n for r in completed)
    return {"completed": len(completed), "samples": int(samples), "samples_per_s": round(samples / wall, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "mean_ms": round(float(lat.mean()), 2), "wall_s": round(wall, 2)}
