#!/usr/bin/env python3
"""Throughput of encrypted inference on one GB300 (or N replicas).

One step = one request of the encrypted CNN on 28x28x1 images with 8192
samples in the slots (RNS-CKKS, N = 16384, coefficient modulus [60, 40 x 7, 60],
scale 2^40, depth 7 from Alg. autoHE / parameterise): encode and encrypt 784
slot vectors (one fused call), evaluate the graph (conv 5x5x5 stride 2 -> degree-3 sigmoid fit ->
dense 720->100 -> sigmoid fit -> dense 100->10), decrypt and decode the 10
outputs.  Keys are generated once, outside the timed region.

Prints one JSON line.  --impl reference times the CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "encrypted samples/s per net"
UNIT = "samples/s"
DOMINANT = "keyswitch_modup_mac"
# GB300 figures (recipe: 152 SMs, 2070 MHz max SM clock; 64 INT32 multiply
# lanes per SM = 4 SMSPs x 16): the derived 32-bit multiply rate, reported
# beside the measured ceilings for context
SMS, SM_MHZ_MAX, MUL32_LANES = 152, 2070.0, 64
PEAK_KINDS = {0: "IMAD (32-bit multiply-add)", 1: "IMAD.WIDE (32x32->64 multiply-add)",
              2: "mul.hi.u64 (high half of a 64x64 product)",
              3: "Shoup butterfly, unreduced form (40-bit primes in the fused transforms)",
              4: "Shoup butterfly, Harvey form"}
BUTTERFLY = 3
# DRAM bytes (read + write) of the key-switching ModUp + key-product kernel
# per (ciphertext, target prime, digit) unit, from one ncu capture of that
# kernel (schedule 8, warp-local transforms) on 64 ciphertexts at L = 7
# (--workload relin): 245.1 MB read + 152.1 MB written over 64 * 8 * 7 units.
# Scaled by units to the bench's launches.
KS_DRAM_BYTES_PER_UNIT = (245.089024e6 + 152.088064e6) / (64 * 8 * 7)


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def replica_times(times_ms, dist, device):
    """Replicas only: every rank times its own requests; the job's time is
    the slowest rank's (all-reduce MAX over the process group, if any)."""
    import torch
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed / the job time."""
    return units_per_rank * world / (ms / 1000.0)


DATA = {
    "cnn": "synthetic (seeded U[0,1] 28x28 images, He-normal weights; Fashion-MNIST not available)",
    "cnn_relu": "synthetic (seeded U[0,1] 28x28 images, He-normal weights; Fashion-MNIST not available)",
    "mlp": "synthetic (seeded lognormal lags + Gaussian weather, Xavier weights; strawberry data not available)",
    "dense_square": "synthetic (seeded U[-1,1] inputs, N(0,0.5) weights)",
    "deep": "synthetic (seeded U[-1,1] inputs, Glorot weights)",
    "cnn_rotate": "synthetic (seeded U[0,1] 28x28 images, He-normal weights; Fashion-MNIST not available)",
    "cnn_masquerade": "synthetic (seeded U[0,1] 28x28 images, He-normal weights; Fashion-MNIST not available)",
}


def workload(name):
    from paper_2110_13638_gb300 import workloads as W
    if name == "cnn":
        g, x = W.cfg1()
        return g, x, "encrypted CNN 28x28x1, conv5x5x5/2 -> sigmoid3 -> 720x100 -> sigmoid3 -> 100x10"
    if name == "mlp":
        g, x = W.cfg2()
        return g, x, "encrypted yield MLP 64 -> 128 -> sigmoid3 -> 32 -> sigmoid3 -> 1"
    if name == "dense_square":
        g, x = W.cfg0()
        return g, x, "dense 8 -> 4 then x^2"
    if name == "cnn_relu":
        g, x = W.cnn_relu()
        return g, x, ("encrypted CNN 28x28x1, conv5x5x5/2 -> ReLU approx (Eq. relu_approximate, q=4) -> 720x100 "
                      "-> sigmoid3 -> 100x10")
    if name == "cnn_rotate":
        g, x = W.cnn_rotate()
        return g, x, ("encrypted CNN with a rotation (client refresh) after the first sigmoid: groups "
                      "conv5x5x5/2 -> sigmoid3 | 720x100 -> sigmoid3 -> 100x10")
    if name == "cnn_masquerade":
        g, x = W.cnn_masquerade(819, 8192, seed=1, side=28, filters=5, k=5, stride=2, hidden=100, classes=10)
        return g, x, ("encrypted CNN with kernel masquerading: 28x28 images packed 10 per ciphertext, conv5x5x5/2 "
                      "by rotations -> sigmoid3 | client re-pack -> 720x100 -> sigmoid3 -> 100x10")
    if name == "deep":
        g, x = W.deep_mlp(n_slots=16384, n_in=64, hidden=64, n_out=8)
        return g, x, "depth-8 MLP 64 -> 64 -> sigmoid3 -> 64 -> sigmoid3 -> 8 -> x^2 (N=32768, [60,40x8,60])"
    raise SystemExit("unknown workload " + name)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def modup_mac_shoup(N, plan):
    """Algorithmic Shoup products of the key-switching ModUp + key inner
    product kernel over one request: per ciphertext at level L, L*L forward
    transforms of (N/2) log2 N butterflies (one Shoup product each) and
    2 L (L+1) N Shoup key products."""
    import math
    lg = int(math.log2(N))
    return sum(n_ct * (L * L * (N // 2) * lg + 2 * L * (L + 1) * N) for n_ct, L in plan)


def mul_relin_rescale_shoup(N, L):
    """Shoup products of one ct-mult + relinearise + rescale at level L:
    the transforms (L digit inverses, L*L ModUp, 2 of P, 2L ModDown, 2
    rescale inverses, 2(L-1) rescale forwards) at (N/2) log2 N butterflies
    each, plus the 2 L (L+1) N key products.  The tensor product and the
    element-wise epilogue products are not counted (a lower bound)."""
    import math
    lg = int(math.log2(N))
    transforms = L + L * L + 2 + 2 * L + 2 + 2 * (L - 1)
    return transforms * (N // 2) * lg + 2 * L * (L + 1) * N


def alu_peaks(kinds=(BUTTERFLY,), target_ms=100.0):
    """Measured register-resident ceilings (fhe_peak_launch), operations/s of
    each kind, best of three launches of about target_ms each."""
    import torch
    from paper_2110_13638_gb300 import fhe
    blocks, threads = SMS * 4, 256
    sink = torch.empty(blocks * threads, dtype=torch.int64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for kind in kinds:
        iters = 256
        fhe.peak_launch(kind, blocks, threads, iters, sink)
        e0.record()
        fhe.peak_launch(kind, blocks, threads, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        iters = max(256, int(iters * target_ms / max(e0.elapsed_time(e1), 1e-3)))
        best = float("inf")
        for _ in range(3):
            e0.record()
            fhe.peak_launch(kind, blocks, threads, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[kind] = blocks * threads * iters * 32 / (best / 1000.0)
    return out


def peak_desc(rate, clk):
    mhz = clk.get("sm_mhz") if clk else None
    d = {"peak_source": "measured: bench.py int-pipe microbenchmark (fhe_peak_launch kind %d, %s), "
                        "best of 3" % (BUTTERFLY, PEAK_KINDS[BUTTERFLY])}
    if mhz:
        d["peak_per_sm_per_clock"] = round(rate / (SMS * mhz * 1e6), 3)
    d["derived_int32_mul_peak_T"] = round(SMS * MUL32_LANES * SM_MHZ_MAX * 1e6 / 1e12, 3)
    return d


def run_ours(args):
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import fhe

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()
    bfly_peak = alu_peaks()[BUTTERFLY] if rank == 0 or world == 1 else None
    g, x, desc = workload(args.workload)
    gof, gcost = fhe.autohe(g)
    N, bits = fhe.parameterise(max(gcost), 40, 1.5)
    ctx = fhe.Context(N, bits, 40)
    ctx.keygen(0)
    G = fhe.Graph(g)
    n_out, L_out = G.outputs(ctx)
    n_in = x.shape[0]
    samples = x.shape[1]
    dev = torch.device("cuda", local)
    slots = torch.tensor(x, dtype=torch.float64, device=dev)
    host_slots = torch.tensor(x, dtype=torch.float64).pin_memory()
    host_out = torch.empty((n_out, samples), dtype=torch.float64).pin_memory()
    ct = ctx.empty_ct(n_in, ctx.L_top)
    out = ctx.empty_ct(n_out, L_out)
    m = torch.empty((n_out, N), dtype=torch.int64, device=dev)
    z = torch.empty((n_out, N // 2), dtype=torch.float64, device=dev)
    meta = [None]

    def step(k, src):
        ctx.encode_encrypt(src, ctx.delta, 1_000_000 * rank + k * n_in, ct)
        meta[0] = G.eval(ctx, [ct], out)
        ctx.decrypt(out, L_out, m)
        ctx.decode(m, meta[0][0][1], z)

    for k in range(args.warmup):
        step(k, slots)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM (1.6 GB of ciphertexts per step > L2)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = fhe.launch_count()
    ctx.profile_begin(args.profile_family, 1 << 16)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(args.warmup + k, slots)
    e1.record()
    barrier()
    dev_ms = e0.elapsed_time(e1)
    prof_ms, prof_n, prof_timed = ctx.profile_end()
    launches = fhe.launch_count() - launches0
    clk = clocks.stop()
    ctx.sync()                       # raises if a kernel gave up a bounded device wait

    # ---- end to end through the C ABI's serving call with HOST buffers:
    # fhe_eval_batch copies the pinned slots in, encrypts, evaluates,
    # decrypts, decodes and copies the outputs back to pinned host memory
    G.eval_batch(ctx, [(host_slots, host_out)], 10_000_000 * (rank + 1))     # sizes the batch area
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    for k in range(args.steps):
        G.eval_batch(ctx, [(host_slots, host_out)], 10_000_000 * (rank + 1) + (k + 1) * n_in)
    e3.record()
    barrier()
    e2e_ms = e2.elapsed_time(e3)
    ctx.sync()

    dev_ms, e2e_ms = replica_times([dev_ms, e2e_ms], dist, dev)
    total_samples = samples * args.steps * world
    value = job_rate(samples * args.steps, world, dev_ms)
    e2e = job_rate(samples * args.steps, world, e2e_ms)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # roofline of the dominant kernel: key-switching ModUp + key products
    plan = []   # (ciphertexts, level) of every relinearisation in one request
    L = ctx.L_top
    for node in g["nodes"]:
        if node["kind"] == "linear":
            L -= 1
        elif node["kind"] in ("poly", "relu"):
            deg = len(node["coeffs"]) - 1 if node["kind"] == "poly" else 2
            n = n_out_prev
            if deg == 3:
                plan += [(n, L), (n, L - 1)]
            elif deg == 2:
                plan += [(n, L)]
            L -= 1 if deg == 1 else 2
        elif node["kind"] == "square":
            plan += [(n_out_prev, L)]
            L -= 1
        if node["kind"] == "linear":
            n_out_prev = node["n_out"]
        elif node["kind"] == "input":
            n_out_prev = node["n"]
    roof = None
    if args.profile_family == DOMINANT and prof_timed:
        work = modup_mac_shoup(N, plan) * args.steps
        per_launch_ms = prof_ms / prof_timed
        achieved = work / (prof_ms / 1000.0) / 1e9
        peak = bfly_peak / 1e9
        units = sum(n * (Lr + 1) * Lr for n, Lr in plan)       # (ciphertext, target, digit) transforms
        traffic = args.traffic
        if traffic is None and plan:
            traffic = round(KS_DRAM_BYTES_PER_UNIT * units / len(plan))
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 2),
                "unit": "G Shoup products/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": DOMINANT, "launches": prof_n, "avg_launch_ms": round(per_launch_ms, 4),
                "share_of_step": round(prof_ms / dev_ms, 4),
                "work_per_step": "sum over relinearisations of L*L transforms x (N/2) log2 N butterflies "
                                 "+ 2 L (L+1) N key products, one Shoup product each"}
        roof.update(peak_desc(bfly_peak, clk))
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": DATA.get(args.workload, "synthetic"),
        "config": {"workload": desc, "N": N, "coeff_modulus_bits": bits, "log_scale": 40,
                   "samples_per_request": samples, "input_ciphertexts": n_in, "output_ciphertexts": n_out,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "ntt_schedule": "%d: %s" % (ctx.ntt_variant, fhe.NTT_SCHEDULES[ctx.ntt_variant]),
                   "ntt_schedule_keyswitch": "%d: %s" % (ctx.ntt_variant_ks, fhe.NTT_SCHEDULES[ctx.ntt_variant_ks]),
                   "l2": "inputs larger than L2 (%.2f GB of input ciphertexts per step)" % (n_in * 2 * ctx.L_top * N * 8 / 1e9)},
        "e2e": {"value": round(e2e, 2), "unit": UNIT, "h2d_bytes_per_step": int(host_slots.numel() * 8),
                "d2h_bytes_per_step": int(host_out.numel() * 8),
                "path": "fhe_eval_batch with pinned host buffers (H2D of the slots, encode+encrypt, graph, "
                        "decrypt, decode, D2H of the outputs), every step"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roof,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = oracle_sample(args.workload)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(name):
    """The oracle as it stands, single-threaded, on a bounded sample of one
    request: per-unit times of every stage (encode+encrypt one input, one conv
    output, one degree-3 activation at each level, one dense output, one
    decrypt+decode), extrapolated to the request's unit counts."""
    import numpy as np
    from oracle import ckks
    g, x, desc = workload(name)
    from oracle.params import autohe, parameterise
    from paper_2110_13638_gb300 import workloads as W
    cost = max(autohe(g, W.input_nodes(g))[1])
    p = parameterise(cost)
    N, bits = p["poly_modulus_degree"], p["coeff_modulus"]
    o = ckks.Context(N, bits, 40)
    t0 = time.perf_counter()
    o.keygen(0)
    t_keygen = time.perf_counter() - t0
    rng = np.random.default_rng(0)

    def rand_ct(L, scale):
        c = np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in o.q[:L]]) for _ in range(2)])
        return ckks.Ciphertext(c, L, scale)

    total = 0.0
    parts = []
    L = o.L_top
    nodes = g["nodes"]
    n_prev = nodes[0]["n"]
    # stage: encode + encrypt (per input ciphertext)
    k = 2
    t0 = time.perf_counter()
    first = [o.encrypt(o.encode(x[i]), i) for i in range(k)]
    t = (time.perf_counter() - t0) / k
    total += t * n_prev
    parts.append("encode+encrypt %.3fs x %d" % (t, n_prev))
    for node in nodes[1:]:
        kind = node["kind"]
        if kind == "linear":
            rows = ckks.csr_rows(node)
            idx, ws = rows[0]
            need = int(max(idx)) + 1
            src = first[:need] if L == o.L_top else []
            src = src + [rand_ct(L, o.delta) for _ in range(need - len(src))]
            t0 = time.perf_counter()
            o.linear(src, [rows[0]], [0.0])
            t = time.perf_counter() - t0
            total += t * node["n_out"]
            parts.append("linear(%d terms, L=%d) %.3fs x %d" % (len(idx), L, t, node["n_out"]))
            n_prev = node["n_out"]
            L -= 1
        elif kind in ("poly", "relu"):
            a = node["coeffs"] if kind == "poly" else ckks.relu_coeffs(node["q"])
            t0 = time.perf_counter()
            o.poly(rand_ct(L, o.delta), a)
            t = time.perf_counter() - t0
            total += t * n_prev
            parts.append("poly%d(L=%d) %.3fs x %d" % (len(a) - 1, L, t, n_prev))
            L -= 1 if len(a) == 2 else 2
        elif kind == "square":
            t0 = time.perf_counter()
            o.square(rand_ct(L, o.delta))
            t = time.perf_counter() - t0
            total += t * n_prev
            parts.append("square(L=%d) %.3fs x %d" % (L, t, n_prev))
            L -= 1
    t0 = time.perf_counter()
    o.decode(o.decrypt(rand_ct(L, o.delta)), o.delta)
    t = time.perf_counter() - t0
    total += t * n_prev
    parts.append("decrypt+decode %.3fs x %d" % (t, n_prev))
    samples = x.shape[1]
    return {"value": round(samples / total, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "estimated": True,
            "method": "estimated, not a timing of a whole request: one unit of every stage timed, "
                      "extrapolated to the request's unit counts",
            "sample": "one unit of every stage, extrapolated to one request (%.1f s est.): %s; keygen %.1fs not counted"
                      % (total, "; ".join(parts), t_keygen),
            "request_s_est": round(total, 1), "host": _host_desc()}


def _host_desc():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for l in f:
                if l.lower().startswith(("model name", "cpu part", "hardware")):
                    model = l.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model}


# ---------------------------------------------------------------- batching sweep
def run_relin(args):
    """Relinearisations of --batch-cts random tensor products at --level,
    N = 16384, [60, 40 x 7, 60]: the key-switching step alone (also the small
    case the ncu captures of the key-switching kernels use)."""
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import fhe
    __graft_entry__.build()
    torch.cuda.set_device(0)
    ctx = fhe.Context(16384, [60] + [40] * 7 + [60], 40)
    ctx.keygen(0)
    n, L = args.batch_cts, args.level
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    d3 = torch.empty((n, 3, L, 16384), dtype=torch.int64, device="cuda")
    for r in range(L):
        d3[:, :, r, :] = torch.randint(0, ctx.primes[r], (n, 3, 16384), device="cuda", generator=gen)
    out = ctx.empty_ct(n, L)
    peak = alu_peaks()[BUTTERFLY]
    for _ in range(args.warmup):
        ctx.relinearise(d3, L, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    ctx.profile_begin(DOMINANT, 1 << 12)
    e0.record()
    for _ in range(args.steps):
        ctx.relinearise(d3, L, out)
    e1.record()
    torch.cuda.synchronize()
    prof_ms, prof_n, prof_timed = ctx.profile_end()
    clk = clocks.stop()
    ctx.sync()
    ms = e0.elapsed_time(e1)
    import math
    lg = int(math.log2(16384))
    # every transform of the relinearisation (L digit inverses, L*L ModUp, 2 of P, 2L ModDown) + key products
    work = n * ((L + L * L + 2 + 2 * L) * 8192 * lg + 2 * L * (L + 1) * 16384) * args.steps
    ks_work = modup_mac_shoup(16384, [(n, L)]) * args.steps
    achieved = work / (ms / 1000.0) / 1e9
    roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak / 1e9, 2),
            "unit": "G Shoup products/s", "frac": round(achieved / (peak / 1e9), 4), "traffic": None,
            "kernel": "whole relinearisation (4 launches)",
            DOMINANT: {"ms": round(prof_ms, 3), "launches": prof_n,
                       "achieved": round(ks_work / (prof_ms / 1000.0) / 1e9, 2) if prof_timed else None,
                       "frac": round(ks_work / (prof_ms / 1000.0) / peak, 4) if prof_timed else None}}
    roof.update(peak_desc(peak, clk))
    print(json.dumps({"metric": "relinearisations/s at N=16384", "value": round(n * args.steps / (ms / 1000.0), 1),
                      "unit": "ops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True, "dtype": "u64",
                      "data": "synthetic (uniform residues, seed 1)",
                      "config": {"workload": "relinearise %d tensor products at L=%d" % (n, L),
                                 "ntt_schedule_keyswitch": ctx.ntt_variant_ks},
                      "clocks": clk, "roofline": roof}), flush=True)


def run_mrr(args):
    """ct-mult + relinearise + rescale of --batch-cts random ciphertext pairs at
    --level, N = 16384, [60, 40 x 7, 60]: one level per call (the merged
    ModDown + rescale path the graph takes after an activation's square; also
    the small case of the ncu captures of the rescale-type transforms)."""
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import fhe
    __graft_entry__.build()
    torch.cuda.set_device(0)
    N = 16384
    ctx = fhe.Context(N, [60] + [40] * 7 + [60], 40)
    ctx.keygen(0)
    n, L = args.batch_cts, args.level
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    a = torch.empty((n, 2, L, N), dtype=torch.int64, device="cuda")
    b = torch.empty((n, 2, L, N), dtype=torch.int64, device="cuda")
    for r in range(L):
        a[:, :, r, :] = torch.randint(0, ctx.primes[r], (n, 2, N), device="cuda", generator=gen)
        b[:, :, r, :] = torch.randint(0, ctx.primes[r], (n, 2, N), device="cuda", generator=gen)
    out = ctx.empty_ct(n, L - 1)
    peak = alu_peaks()[BUTTERFLY]
    for _ in range(args.warmup):
        ctx.mul_relin_rescale(a, b, L, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    e0.record()
    for _ in range(args.steps):
        ctx.mul_relin_rescale(a, b, L, out)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.sync()
    ms = e0.elapsed_time(e1)
    work = n * mul_relin_rescale_shoup(N, L) * args.steps
    achieved = work / (ms / 1000.0) / 1e9
    roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak / 1e9, 2),
            "unit": "G Shoup products/s", "frac": round(achieved / (peak / 1e9), 4), "traffic": None,
            "kernel": "whole step (every launch of the call)",
            "work_per_step": "per op at level L: (L + L*L + 2 + 2L + 2 + 2(L-1)) transforms x (N/2) log2 N "
                             "butterflies + 2 L (L+1) N key products (the merged path executes 2L fewer "
                             "transforms; tensor and element-wise products not counted)"}
    roof.update(peak_desc(peak, clk))
    print(json.dumps({"metric": "ct-mult+relin+rescale/s at N=16384", "value": round(n * args.steps / (ms / 1000.0), 1),
                      "unit": "ops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True, "dtype": "u64",
                      "data": "synthetic (uniform residues, seed 1)",
                      "config": {"workload": "mul + relinearise + rescale %d ciphertext pairs at L=%d" % (n, L),
                                 "ntt_schedule": ctx.ntt_variant, "ntt_schedule_keyswitch": ctx.ntt_variant_ks},
                      "clocks": clk, "roofline": roof}), flush=True)


def run_batch(args):
    """4096 ciphertext pairs at uneven levels (L = 1 + U{1..7}, seed 3), each
    getting ct-mult + relinearise + rescale: all levels in one call (one
    persistent launch) captured in a CUDA graph, against the same call as six
    separate launches (FHE_PERSISTENT=0) and the plain path that calls
    fhe_mul_relin_rescale once per ciphertext."""
    import numpy as np
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import fhe
    __graft_entry__.build()
    torch.cuda.set_device(0)
    bits = [60] + [40] * 7 + [60]
    ctx = fhe.Context(16384, bits, 40)
    ctx.keygen(0)
    n_ct = args.batch_cts
    levels = 1 + np.random.Generator(np.random.PCG64(3)).integers(1, 8, size=n_ct)
    batches = []
    for L in range(2, 9):
        n = int((levels == L).sum())
        if n == 0:
            continue
        def rnd():
            t = torch.empty((n, 2, L, 16384), dtype=torch.int64, device="cuda")
            for r in range(L):
                t[:, :, r, :] = torch.randint(0, ctx.primes[r], (n, 2, 16384), device="cuda")
            return t
        batches.append((rnd(), rnd(), ctx.empty_ct(n, L - 1), L))
    peak = alu_peaks()[BUTTERFLY]

    def captured():
        ctx.mul_relin_rescale_levels(batches)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                ctx.mul_relin_rescale_levels(batches)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        return graph

    launches0 = fhe.launch_count()
    ctx.mul_relin_rescale_levels(batches)
    launches_per_call = fhe.launch_count() - launches0
    graph = captured()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    e0.record()
    for _ in range(args.steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ctx.sync()
    # the same call as six separate launches
    os.environ["FHE_PERSISTENT"] = "0"
    try:
        graph6 = captured()
    finally:
        os.environ.pop("FHE_PERSISTENT", None)
    e0.record()
    for _ in range(args.steps):
        graph6.replay()
    e1.record()
    torch.cuda.synchronize()
    ms6 = e0.elapsed_time(e1) / args.steps
    ctx.sync()
    work = sum(int((levels == L).sum()) * mul_relin_rescale_shoup(16384, L) for L in range(2, 9))
    achieved = work / (ms / 1000.0) / 1e9
    roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak / 1e9, 2),
            "unit": "G Shoup products/s", "frac": round(achieved / (peak / 1e9), 4), "traffic": None,
            "kernel": "whole step (every launch of the call)",
            "work_per_step": "per op at level L: (L + L*L + 2 + 2L + 2 + 2(L-1)) transforms x (N/2) log2 N "
                             "butterflies + 2 L (L+1) N key products (tensor and element-wise products not counted)"}
    roof.update(peak_desc(peak, clk))
    # plain path: one call per ciphertext
    singles = [(a[k:k + 1], b[k:k + 1], o[k:k + 1], L) for (a, b, o, L) in batches for k in range(a.shape[0])]
    for a, b, o, L in singles[:16]:
        ctx.mul_relin_rescale(a, b, L, o)
    torch.cuda.synchronize()
    e0.record()
    for a, b, o, L in singles:
        ctx.mul_relin_rescale(a, b, L, o)
    e1.record()
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    line = {"metric": "ct-mult+relin+rescale/s at N=16384", "value": round(n_ct / (ms / 1000.0), 1),
            "unit": "ops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic (uniform residues)",
            "config": {"workload": "%d ciphertext pairs at uneven levels 2..8 (seed 3), one call, one persistent "
                                   "launch, CUDA graph" % n_ct, "level_counts": {int(L): int((levels == L).sum())
                                                                                for L in range(2, 9)},
                       "kernel_launches_per_call": int(launches_per_call), "ntt_schedule": ctx.ntt_variant},
            "six_launches": {"value": round(n_ct / (ms6 / 1000.0), 1), "unit": "ops/s", "ms_per_step": round(ms6, 3),
                             "note": "the same call with FHE_PERSISTENT=0 (one launch per step), CUDA graph"},
            "one_at_a_time": {"value": round(n_ct / (ms1 / 1000.0), 1), "unit": "ops/s",
                              "ms_total": round(ms1, 2)},
            "clocks": clk, "roofline": roof}
    print(json.dumps(line), flush=True)


def run_ntt_sweep(args):
    """Forward residue-NTT throughput, N = 2^13 .. 2^16, 1 .. 30 primes of the
    40-bit chain, the autotuned schedule against the fixed one (one block per
    transform at N <= 16384, two-pass above)."""
    import math
    import os as _os
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import fhe
    __graft_entry__.build()
    torch.cuda.set_device(0)
    peak = alu_peaks()[BUTTERFLY]
    clocks = ClockSampler(0)
    clocks.start()
    rows = []
    for logN in range(13, 17):
        N = 1 << logN
        for nprime in (1, 2, 4, 8, 16, 30):
            bits = [40] * nprime + [60]
            res = {"N": N, "primes": nprime}
            for mode in ("autotuned", "fixed"):
                if mode == "fixed":
                    _os.environ["FHE_NTT_VARIANT"] = "0" if N <= 16384 else "2"
                try:
                    ctx = fhe.Context(N, bits, 40)
                finally:
                    _os.environ.pop("FHE_NTT_VARIANT", None)
                groups = max(1, (1 << 26) // (N * nprime))
                t = torch.zeros((groups, nprime, N), dtype=torch.int64, device="cuda")
                ctx.ntt(t, nprime, True)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(3):
                    ctx.ntt(t, nprime, True)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 3
                polys = groups * nprime
                gb = polys * (N // 2) * logN / ms / 1e6
                res[mode] = {"schedule": ctx.ntt_variant, "residue_ntts_per_s": round(polys / ms * 1000.0),
                             "Gbutterfly_s": round(gb, 1), "frac": round(gb / (peak / 1e9), 4)}
                ctx.close()
                del t
            rows.append(res)
    clk = clocks.stop()
    n16 = [r for r in rows if r["N"] == 16384 and r["primes"] == 8][0]["autotuned"]
    roof = {"bound": "alu", "achieved": n16["Gbutterfly_s"], "peak": round(peak / 1e9, 2),
            "unit": "G Shoup butterflies/s", "frac": n16["frac"], "traffic": None,
            "kernel": "forward transforms, N=16384, 8 primes, autotuned schedule"}
    roof.update(peak_desc(peak, clk))
    line = {"metric": "residue NTTs/s (sweep)", "value": n16["residue_ntts_per_s"], "unit": "NTT/s",
            "config": {"workload": "forward residue NTTs, N=2^13..2^16 x 1..30 primes, 2^26 words per batch; "
                                   "value = N=16384, 8 primes, autotuned"},
            "sweep": rows, "note": "autotuned vs fixed schedule per (N, primes); frac = of the measured butterfly "
                                   "ceiling", "clocks": clk, "roofline": roof}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving
def serving_setup(torch):
    from paper_2110_13638_gb300 import fhe, serve, workloads as W
    nets = []
    ctxs = {}
    for name, builder in (("dense_square", W.cfg0), ("cnn", W.cfg1), ("mlp", W.cfg2)):
        g, x = builder()
        gof, gcost = fhe.autohe(g)
        N, bits = fhe.parameterise(max(gcost), 40, 1.5)
        key = (N, tuple(bits))
        if key not in ctxs:                      # one context (and one key set) per parameter set
            c = fhe.Context(N, bits, 40)
            c.keygen(0)
            ctxs[key] = c
        nets.append(serve.Network(name, g, x, ctxs[key]))
    return nets, ctxs


def poisson_requests(nets, seconds, lam=200.0, weights=(0.5, 0.3, 0.2), seed=4):
    import numpy as np
    from paper_2110_13638_gb300 import serve
    rng = np.random.Generator(np.random.PCG64(seed))
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / lam)
        if t > seconds:
            break
        k = int(rng.choice(len(nets), p=list(weights)))
        n = int(rng.integers(1, 8193))
        off = int(rng.integers(0, 1 << 20))
        reqs.append(serve.Request(len(reqs), nets[k], t, n, nets[k].inputs(off, n)))
    return reqs


def run_grouped(args):
    """A network with rotation nodes: one context per parameter group
    (Alg. autoHE + parameterise per group), each group on the device, the
    client refresh (decrypt, decode, encode, encrypt) between groups on the
    device too.  Step = one request through every group."""
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import fhe, groups
    __graft_entry__.build()
    torch.cuda.set_device(0)
    g, x, desc = workload(args.workload)
    net = groups.GroupedNetwork(g)
    dev = torch.device("cuda", 0)
    slots = torch.tensor(x, dtype=torch.float64, device=dev)
    host_slots = torch.tensor(x, dtype=torch.float64).pin_memory()
    outs = [i for i, n in enumerate(g["nodes"]) if n["kind"] == "output"]
    res = None
    for k in range(args.warmup):
        res = net.evaluate([slots], first_ct_id=k << 24)
    torch.cuda.synchronize()
    host_out = {o: torch.empty(tuple(res[o].shape), dtype=torch.float64).pin_memory() for o in outs}
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = fhe.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for k in range(args.steps):
        net.evaluate([slots], first_ct_id=(args.warmup + k) << 24)
    e1.record()
    torch.cuda.synchronize()
    dev_ms = e0.elapsed_time(e1)
    launches = fhe.launch_count() - launches0
    clk = clocks.stop()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    for k in range(args.steps):
        slots.copy_(host_slots, non_blocking=True)
        r = net.evaluate([slots], first_ct_id=(10 * args.steps + k) << 24)
        for o in outs:
            host_out[o].copy_(r[o], non_blocking=True)
    e3.record()
    torch.cuda.synchronize()
    e2e_ms = e2.elapsed_time(e3)
    conv = [n for n in g["nodes"] if n["kind"] == "conv_packed"]
    per_req = x.shape[0] * conv[0]["images"] if conv else x.shape[1]
    samples = per_req * args.steps
    line = {
        "metric": METRIC, "value": round(samples / (dev_ms / 1000.0), 2), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": DATA.get(args.workload, "synthetic"),
        "config": {"workload": desc, "groups": [
            {"cost": c, "N": net.ctx[i].N, "L_top": net.ctx[i].L_top} for i, c in enumerate(net.group_cost)],
            "samples_per_request": int(per_req)},
        "e2e": {"value": round(samples / (e2e_ms / 1000.0), 2), "unit": UNIT,
                "h2d_bytes_per_step": int(slots.numel() * 8),
                "d2h_bytes_per_step": int(sum(res[o].numel() for o in outs) * 8)},
        "gpu_launches": int(launches), "clocks": clk, "roofline": None,
    }
    print(json.dumps(line), flush=True)
    net.close()


def run_serve(args):
    """Poisson arrivals (--serve-rate, 200 req/s by default; mix 0.5 / 0.3 / 0.2 of the dense+square
    network, the CNN and the yield MLP, 1..8192 samples each) for
    --serve-seconds, continuous batching under a 150 GB admission cap, against
    serial one-request-at-a-time evaluation on the same GPU."""
    import torch
    import __graft_entry__
    from paper_2110_13638_gb300 import serve
    __graft_entry__.build()
    torch.cuda.set_device(0)
    nets, ctxs = serving_setup(torch)
    cap = 150e9
    clocks = ClockSampler(0)
    clocks.start()
    out = {"metric": "serve samples/s, p50/p99 ms", "unit": "samples/s", "n_gpus": 1,
           "config": {"workload": "Poisson %g req/s, mix 0.5/0.3/0.2 (dense+square N=8192 / CNN / yield MLP "
                                  "N=16384), 1..8192 samples, %gs of arrivals, admission cap 150 GB"
                                  % (args.serve_rate, args.serve_seconds),
                      "parameter_sets": len(ctxs)}}
    for mode in ("continuous", "serial"):
        reqs = poisson_requests(nets, args.serve_seconds, lam=args.serve_rate)
        offered = sum(r.n for r in reqs) / args.serve_seconds
        if mode == "continuous":
            srv = serve.Server(nets, {"dense_square": 2, "cnn": 3, "mlp": 2}, cap, pack=True)
        else:
            srv = serve.Server(nets, {"dense_square": 1, "cnn": 1, "mlp": 1}, cap, pack=False, max_inflight=1)
        torch.cuda.synchronize()
        done, wall, backlog = srv.run(reqs, horizon=args.serve_seconds)
        st = serve.latency_stats(done, wall)
        st.update({"arrived": len(reqs), "backlog_at_horizon": backlog, "offered_samples_per_s": round(offered, 1),
                   "slots": {k: len(v) for k, v in srv.slots.items()},
                   "footprint_GB": round(srv.footprint / 1e9, 2)})
        for net in nets:
            d = [r for r in done if r.net is net]
            st[net.name] = serve.latency_stats(d, wall) if d else {"completed": 0}
        out[mode] = st
        del srv
        torch.cuda.synchronize()
    out["value"] = out["continuous"].get("samples_per_s")
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)


def run_int_peak(args):
    """Register-resident ceilings of the integer pipes (fhe_peak_launch):
    32-bit IMAD, IMAD.WIDE, the 64-bit high product and the two Shoup
    butterfly forms, each as operations/s and per SM per clock at the
    sampled SM clock."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    alu_peaks(tuple(PEAK_KINDS), target_ms=20.0)           # warm-up
    clocks = ClockSampler(0)
    clocks.start()
    rates = alu_peaks(tuple(PEAK_KINDS), target_ms=150.0)
    clk = clocks.stop()
    mhz = clk.get("sm_mhz") or SM_MHZ_MAX
    kinds = {PEAK_KINDS[k]: {"G_ops_per_s": round(v / 1e9, 1), "per_sm_per_clock": round(v / (SMS * mhz * 1e6), 3)}
             for k, v in rates.items()}
    print(json.dumps({"metric": "integer-pipe ceilings", "value": round(rates[BUTTERFLY] / 1e9, 1),
                      "unit": "G Shoup butterflies/s", "n_gpus": 1, "kinds": kinds,
                      "config": {"workload": "fhe_peak_launch: %d blocks x 256 threads, 32 independent chains per "
                                             "thread in registers, best of 3 launches of ~150 ms" % (SMS * 4)},
                      "derived_int32_mul_peak_T": round(SMS * MUL32_LANES * SM_MHZ_MAX * 1e6 / 1e12, 3),
                      "clocks": clk}), flush=True)


def _oracle_worker(name):
    return oracle_sample(name)


def run_reference(args):
    """The oracle as it stands on every host core: each step runs one bounded
    sample of the request (one unit of every stage, extrapolated) in each of
    os.cpu_count() spawned processes at once; the step's rate is the sum of
    their rates.  Same metric and configuration as the GPU arm; rank 0 only."""
    rank, world, local = _env_rank()
    if rank != 0:
        return
    if args.workload not in ("cnn", "mlp", "dense_square", "cnn_relu", "deep"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the graph workloads "
                                                              "(cnn, mlp, dense_square, cnn_relu, deep)"}))
        return
    import multiprocessing as mp
    procs = max(1, os.cpu_count() or 1)
    vals, last = [], None
    with mp.get_context("spawn").Pool(procs) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_worker, [args.workload] * procs)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            res = pool.map(_oracle_worker, [args.workload] * procs)
            vals.append(sum(r["value"] for r in res))
            last = res[0]
        wall = time.perf_counter() - t0
    value = statistics.median(vals)
    step_ms = wall / max(1, args.steps) * 1000.0
    g, x, desc = workload(args.workload)
    from oracle.params import autohe, parameterise
    from paper_2110_13638_gb300 import workloads as W
    p = parameterise(max(autohe(g, W.input_nodes(g))[1]))
    outs = sum(len(n["row_ptr"]) - 1 for n in g["nodes"][-2:-1] if n["kind"] == "linear") or None
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(step_ms, 1), "higher_is_better": True,
            "estimated": True,
            "method": "estimated, not a timing of a whole request: each step times one unit of every stage in "
                      "every process (ms_per_step is that measured wall time); value = the sum over processes of "
                      "samples per request / the request time extrapolated from those units",
            "ms_per_request_est": round(x.shape[1] / value * 1000.0 * procs, 1),
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": DATA.get(args.workload, "synthetic"),
            "config": {"workload": desc, "N": p["poly_modulus_degree"], "coeff_modulus_bits": p["coeff_modulus"],
                       "log_scale": 40, "samples_per_request": int(x.shape[1]), "input_ciphertexts": int(x.shape[0]),
                       "output_ciphertexts": outs, "parallelism": "host, %d processes" % procs},
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": procs, "kind": "oracle",
                             "estimated": True,
                             "sample": "%d concurrent processes, each: %s" % (procs, last["sample"]),
                             "host": last["host"]},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cnn", choices=["cnn", "mlp", "dense_square", "cnn_relu", "deep", "cnn_rotate",
                                                          "cnn_masquerade", "batch", "relin", "ntt_sweep", "serve",
                                                          "int_peak", "mrr"])
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--batch-cts", type=int, default=4096)
    ap.add_argument("--level", type=int, default=7, help="level of --workload relin")
    ap.add_argument("--profile-family", default=DOMINANT)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel (from profiles/)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "relin":
        run_relin(args)
    elif args.workload == "mrr":
        run_mrr(args)
    elif args.workload == "ntt_sweep":
        run_ntt_sweep(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "int_peak":
        run_int_peak(args)
    elif args.workload in ("cnn_rotate", "cnn_masquerade"):
        run_grouped(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
