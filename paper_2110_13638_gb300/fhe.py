"""Python binding of libfhe (include/fhe.h): argument marshalling only.

Every step of the encrypted path runs in the sm_103a CUDA library; this module
converts PyTorch tensors to device pointers and host arrays to C arrays, and
raises FheError on a non-zero return code.  There is no fallback: if the
library is not built, the first call raises.

Device buffers are torch tensors (dtype int64 holding raw 64-bit residues, or
float64 slots) on the current CUDA device; work is enqueued on the current
torch stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "csrc", "_build", "libfhe.so")

(FHE_NODE_INPUT, FHE_NODE_LINEAR, FHE_NODE_POLY, FHE_NODE_SQUARE, FHE_NODE_ADD, FHE_NODE_OUTPUT,
 FHE_NODE_RELU, FHE_NODE_ROTATE, FHE_NODE_CONV_PACKED) = range(9)
_KINDS = {"input": FHE_NODE_INPUT, "linear": FHE_NODE_LINEAR, "poly": FHE_NODE_POLY,
          "square": FHE_NODE_SQUARE, "add": FHE_NODE_ADD, "output": FHE_NODE_OUTPUT, "relu": FHE_NODE_RELU,
          "rotate": FHE_NODE_ROTATE, "conv_packed": FHE_NODE_CONV_PACKED}

ERRORS = {-1: "FHE_EINVAL", -2: "FHE_ENOMEM", -3: "FHE_ELEVEL", -4: "FHE_ESCALE", -5: "FHE_ECUDA",
          -6: "FHE_ETIMEOUT", -7: "FHE_EUNSUPPORTED", -8: "FHE_ENOKEY"}


class FheError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class CtxInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("slots", ctypes.c_uint32), ("L_top", ctypes.c_uint32),
                ("log_scale", ctypes.c_uint32), ("primes", ctypes.c_uint64 * 64), ("key_bytes", ctypes.c_uint64),
                ("ntt_variant", ctypes.c_uint32), ("ntt_variant_us", ctypes.c_float * 16),
                ("ntt_variant_ks", ctypes.c_uint32), ("ntt_variant_ks_us", ctypes.c_float * 16),
                ("workspace_bytes", ctypes.c_uint64)]


class CtMeta(ctypes.Structure):
    _fields_ = [("level", ctypes.c_uint32), ("scale", ctypes.c_double)]


class LevelBatch(ctypes.Structure):
    _fields_ = [("d_a", ctypes.c_void_p), ("d_b", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("n_ct", ctypes.c_uint32), ("level", ctypes.c_uint32)]


class NodeDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("n_out", ctypes.c_uint32),
                ("row_ptr", ctypes.POINTER(ctypes.c_uint32)), ("col_idx", ctypes.POINTER(ctypes.c_uint32)),
                ("weight", ctypes.POINTER(ctypes.c_double)), ("bias", ctypes.POINTER(ctypes.c_double)),
                ("coeffs", ctypes.c_double * 4), ("degree", ctypes.c_uint32), ("conv", ctypes.c_uint32 * 6),
                ("coeffs_hi", ctypes.POINTER(ctypes.c_double))]


class Request(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("n_samples", ctypes.c_uint32), ("x_stride", ctypes.c_uint32),
                ("y", ctypes.c_void_p), ("y_stride", ctypes.c_uint32)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint32), ("nodes", ctypes.POINTER(NodeDesc)),
                ("n_edges", ctypes.c_uint32), ("edge_src", ctypes.POINTER(ctypes.c_uint32)),
                ("edge_dst", ctypes.POINTER(ctypes.c_uint32))]


# exported symbols and their signatures (mirrors include/fhe.h)
_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_I = ctypes.c_int
SIGNATURES = {
    "fhe_parameterise": [_U32, _U32, ctypes.c_double, _P, _P, _U32, _P],
    "fhe_autohe": [_P, _P, _U32, _P, _U32, _P],
    "fhe_autoparam": [_P, _U32, ctypes.c_double, _P, _P, _U32, _P],
    "fhe_prime_chain": [_U32, _P, _U32, _P],
    "fhe_gauss_table": [_P],
    "fhe_ctx_create": [_U32, _P, _U32, _U32, _P],
    "fhe_ctx_fork": [_P, _P],
    "fhe_ctx_destroy": [_P],
    "fhe_ctx_query": [_P, _P],
    "fhe_keygen": [_P, _U64, _P],
    "fhe_export_secret": [_P, _P, _P],
    "fhe_encode": [_P, _P, _U32, _U32, ctypes.c_double, _P, _P],
    "fhe_encrypt": [_P, _P, _U32, _U64, _P, _P],
    "fhe_encode_encrypt": [_P, _P, _U32, ctypes.c_double, _U64, _P, _P],
    "fhe_decrypt": [_P, _P, _U32, _U32, _P, _P],
    "fhe_decode": [_P, _P, _U32, ctypes.c_double, _P, _P],
    "fhe_ntt": [_P, _P, _U32, _U32, _I, _P],
    "fhe_ct_convert": [_P, _P, _U32, _U32, _I, _P, _P],
    "fhe_add": [_P, _P, _P, _U32, _U32, _P, _P],
    "fhe_tensor": [_P, _P, _P, _U32, _U32, _P, _P],
    "fhe_relinearise": [_P, _P, _U32, _U32, _P, _P],
    "fhe_relinearise_noalloc": [_P, _P, _U32, _U32, _P, _P],
    "fhe_rescale": [_P, _P, _U32, _U32, _U32, _P, _P],
    "fhe_mul_relin_rescale": [_P, _P, _P, _U32, _U32, _P, _P],
    "fhe_mul_relin_rescale_levels": [_P, _P, _U32, _P],
    "fhe_mul_const": [_P, _P, _P, _U32, _U32, _P, _P],
    "fhe_add_const": [_P, _P, _P, _U32, _U32, _P],
    "fhe_graph_create": [_P, _P],
    "fhe_graph_destroy": [_P],
    "fhe_graph_outputs": [_P, _P, _P, _P],
    "fhe_eval_graph": [_P, _P, _P, _U32, _P, _P, _U32, _P],
    "fhe_eval_batch": [_P, _P, _P, _U32, _U64, _P],
    "fhe_galois_keygen": [_P, _P, _U32, _P],
    "fhe_gather_slots": [_P, _P, _U32, _U32, _P, _P],
    "fhe_rotate": [_P, _P, _U32, _U32, ctypes.c_int32, _P, _P],
    "fhe_profile_begin": [_P, ctypes.c_char_p, _U32],
    "fhe_profile_end": [_P, _P, _P, _P],
    "fhe_profile_families": [],
    "fhe_launch_count": [_P],
    "fhe_device_faults": [_P],
    "fhe_ctx_sync": [_P, _P],
    "fhe_peak_launch": [_U32, _U32, _U32, _U32, _P, _P],
    "fhe_inject_fault": [_P, _U32],
    "fhe_last_error": [],
}

_lib = None


def lib():
    """Load libfhe.so; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise FheError(-7, "libfhe.so is not built (%s); run __graft_entry__.build()" % SO_PATH)
        L = ctypes.CDLL(SO_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("fhe_last_error", "fhe_profile_families") else ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise FheError(rc, lib().fhe_last_error().decode(errors="replace"))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _arr(values, ctype):
    a = (ctype * len(values))()
    for i, v in enumerate(values):
        a[i] = v
    return a


# ---------------------------------------------------------------- host-only
def parameterise(cost, log_scale=40, special_mult=1.5):
    N = ctypes.c_uint32()
    bits = (ctypes.c_uint32 * 64)()
    nb = ctypes.c_uint32()
    _check(lib().fhe_parameterise(cost, log_scale, special_mult, ctypes.byref(N), bits, 64, ctypes.byref(nb)))
    return N.value, [bits[i] for i in range(nb.value)]


def launch_count():
    out = ctypes.c_uint64()
    _check(lib().fhe_launch_count(ctypes.byref(out)))
    return out.value


def device_faults():
    """Device fault flags (bit 0: a tensor-core MAC wait gave up), cleared by the read."""
    out = ctypes.c_uint32()
    _check(lib().fhe_device_faults(ctypes.byref(out)))
    return out.value


def peak_launch(kind, blocks, threads, iters, sink, stream=None):
    """Enqueue the integer-pipe ceiling microbenchmark (include/fhe.h):
    blocks * threads * iters * 32 operations of `kind`; sink: int64 device
    tensor of at least blocks * threads words."""
    if sink.numel() < blocks * threads or sink.dtype.itemsize != 8 or not sink.is_cuda:
        raise ValueError("sink must be a device tensor of blocks * threads 8-byte words")
    _check(lib().fhe_peak_launch(kind, blocks, threads, iters, _ptr(sink), _stream(stream)))


def profile_families():
    return lib().fhe_profile_families().decode().split(",")


def prime_chain(N, bits):
    out = (ctypes.c_uint64 * len(bits))()
    _check(lib().fhe_prime_chain(N, _arr(bits, ctypes.c_uint32), len(bits), out))
    return [int(v) for v in out]


def gauss_table():
    out = (ctypes.c_uint64 * 38)()
    _check(lib().fhe_gauss_table(out))
    return [int(v) for v in out]


def gather_slots(src, index, rows, cols, dst, stream=None):
    """dst[r][c] = src.flatten()[index[r * cols + c]] (0 where index < 0);
    float64 device tensors, int64 device index."""
    _check(lib().fhe_gather_slots(_ptr(src), _ptr(index), rows, cols, _ptr(dst), _stream(stream)))


class _GraphArrays:
    """Keeps the C arrays of a graph description alive while it is used."""

    def __init__(self, graph):
        nodes = graph["nodes"]
        self.keep = []
        self.nodes = (NodeDesc * len(nodes))()
        for i, n in enumerate(nodes):
            d = self.nodes[i]
            d.kind = _KINDS[n["kind"]]
            if n["kind"] == "linear":
                rp = np.ascontiguousarray(n["row_ptr"], dtype=np.uint32)
                ci = np.ascontiguousarray(n["col_idx"], dtype=np.uint32)
                w = np.ascontiguousarray(n["weight"], dtype=np.float64)
                b = np.ascontiguousarray(n["bias"], dtype=np.float64)
                self.keep += [rp, ci, w, b]
                d.n_out = len(rp) - 1
                d.row_ptr = rp.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
                d.col_idx = ci.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
                d.weight = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                d.bias = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            elif n["kind"] == "input":
                d.n_out = int(n.get("n", 0))
            elif n["kind"] == "conv_packed":
                w = np.ascontiguousarray(np.asarray(n["weight"], dtype=np.float64).reshape(-1))
                b = np.ascontiguousarray(n["bias"], dtype=np.float64)
                self.keep += [w, b]
                d.n_out = int(n["filters"])
                d.weight = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                d.bias = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                for k, key in enumerate(("H", "W", "k", "stride", "images", "slot_stride")):
                    d.conv[k] = int(n[key])
            if n["kind"] == "poly":
                a = [float(v) for v in n["coeffs"]]
                if not 2 <= len(a) <= 32:
                    raise ValueError("polynomial nodes take 2 to 32 coefficients (degree 1..31)")
                d.degree = len(a) - 1
                for k in range(min(4, len(a))):
                    d.coeffs[k] = a[k]
                if len(a) > 4:
                    hi = np.ascontiguousarray(a, dtype=np.float64)
                    self.keep.append(hi)
                    d.coeffs_hi = hi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            elif n["kind"] == "relu":
                d.coeffs[0] = float(n["q"])
        src = np.array([e[0] for e in graph["edges"]], dtype=np.uint32)
        dst = np.array([e[1] for e in graph["edges"]], dtype=np.uint32)
        self.keep += [src, dst]
        self.desc = GraphDesc(len(nodes), self.nodes, len(src),
                              src.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                              dst.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))


def autohe(graph):
    """(group of each ingress node -- INPUT and ROTATE -- in node order, cost of
    each group)."""
    ga = _GraphArrays(graph)
    n_in = sum(1 for n in graph["nodes"] if n["kind"] in ("input", "rotate"))
    gof = (ctypes.c_uint32 * max(1, n_in))()
    gcost = (ctypes.c_uint32 * max(1, n_in))()
    ng = ctypes.c_uint32()
    _check(lib().fhe_autohe(ctypes.byref(ga.desc), gof, n_in, gcost, n_in, ctypes.byref(ng)))
    return [gof[i] for i in range(n_in)], [gcost[i] for i in range(ng.value)]


# ---------------------------------------------------------------- context
# names of the NTT schedules the autotuner chooses between (index = ntt_variant)
NTT_SCHEDULES = (
    "radix-16 passes, 512 threads, one block per transform",
    "radix-8 passes, 1024 threads, one block per transform",
    "two-pass column/row tiles, radix-16",
    "two-pass column/row tiles, radix-8",
    "radix-8, 1024 threads, global loads/stores fused into the first/last pass",
    "radix-16, 512 threads, global loads/stores fused into the first/last pass",
    "key-switching digit transforms split over two blocks per polynomial (one per output half), 256 threads",
    "key-switching digit transforms on a cluster of four blocks (one per coefficient quarter), accumulators in "
    "shared memory",
    "warp-local: the first log2 N - 10 stages block-wide, then one 1024-point sub-transform per warp, 32 values "
    "per lane",
)


class Context:
    """An RNS-CKKS context on the current CUDA device (tables and keys in HBM)."""

    def __init__(self, N, bits, log_scale=40, _fork_of=None):
        h = ctypes.c_void_p()
        if _fork_of is not None:
            _check(lib().fhe_ctx_fork(_fork_of.h, ctypes.byref(h)))
            self._parent = _fork_of          # keeps the parent alive
        else:
            _check(lib().fhe_ctx_create(N, _arr(bits, ctypes.c_uint32), len(bits), log_scale, ctypes.byref(h)))
        self.h = h
        info = CtxInfo()
        _check(lib().fhe_ctx_query(self.h, ctypes.byref(info)))
        self.N = info.N
        self.slots = info.slots
        self.L_top = info.L_top
        self.log_scale = info.log_scale
        self.primes = [int(info.primes[i]) for i in range(info.L_top + 1)]
        self.key_bytes = int(info.key_bytes)
        self.ntt_variant = int(info.ntt_variant)
        self.ntt_variant_us = [float(info.ntt_variant_us[i]) for i in range(len(NTT_SCHEDULES))]
        self.ntt_variant_ks = int(info.ntt_variant_ks)
        self.ntt_variant_ks_us = [float(info.ntt_variant_ks_us[i]) for i in range(len(NTT_SCHEDULES))]
        self.delta = float(2 ** log_scale)

    def fork(self):
        """A context sharing these tables and keys with its own workspace."""
        return Context(self.N, None, self.log_scale, _fork_of=self)

    def close(self):
        if getattr(self, "h", None):
            lib().fhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- measurement -------------------------------------------------------------
    def profile_begin(self, family, max_launches=65536):
        _check(lib().fhe_profile_begin(self.h, family.encode(), max_launches))

    def profile_end(self):
        """-> (total device ms, launches, timed launches) of the profiled family"""
        ms = ctypes.c_double()
        n = ctypes.c_uint64()
        t = ctypes.c_uint64()
        _check(lib().fhe_profile_end(self.h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(t)))
        return ms.value, n.value, t.value

    # -- allocation helpers (torch device memory) --------------------------
    def empty_ct(self, n, level, comps=2):
        import torch
        return torch.empty((n, comps, level, self.N), dtype=torch.int64, device="cuda")

    def empty_pt(self, n, level):
        import torch
        return torch.empty((n, level, self.N), dtype=torch.int64, device="cuda")

    def workspace_bytes(self):
        """Device bytes of this context's call workspace and batch area."""
        info = CtxInfo()
        _check(lib().fhe_ctx_query(self.h, ctypes.byref(info)))
        return int(info.workspace_bytes)

    # -- health ---------------------------------------------------------------
    def sync(self, stream=None):
        """Wait for the stream; raises FheError (FHE_ETIMEOUT) if a kernel of a
        call on this context gave up a bounded device wait."""
        _check(lib().fhe_ctx_sync(self.h, _stream(stream)))

    def inject_fault(self, kind=1):
        """Test hook: kind 1 = the next tensor-core layer MAC withholds its
        matrix products, so its bounded waits run out (FHE_ETIMEOUT)."""
        _check(lib().fhe_inject_fault(self.h, kind))

    # -- argument checks (a wrong-sized buffer would be read or written out of bounds)
    def _ct(self, t, n, comps, level, name):
        _dev(t, (n, comps, level, self.N), "int64", name)

    def _lv(self, level, lo=1):
        """True if the library accepts `level`; otherwise it refuses the call
        with FHE_ELEVEL before touching any buffer, so shapes are not checked."""
        return lo <= level <= self.L_top

    # -- keys / encode / encrypt / decrypt / decode ------------------------
    def keygen(self, seed, stream=None):
        _check(lib().fhe_keygen(self.h, seed, _stream(stream)))

    def export_secret(self, out, stream=None):
        _dev(out, (self.L_top + 1, self.N), "int64", "out")
        _check(lib().fhe_export_secret(self.h, _ptr(out), _stream(stream)))

    def encode(self, slots, level, scale, out, stream=None):
        n = _rows(slots)
        _dev(slots, (n, self.N // 2), "float64", "slots")
        if self._lv(level):
            _dev(out, (n, level, self.N), "int64", "out")
        _check(lib().fhe_encode(self.h, _ptr(slots), n, level, scale, _ptr(out), _stream(stream)))

    def encrypt(self, pt, first_ct_id, out, stream=None):
        n = _rows(pt)
        _dev(pt, (n, self.L_top, self.N), "int64", "pt")
        self._ct(out, n, 2, self.L_top, "out")
        _check(lib().fhe_encrypt(self.h, _ptr(pt), n, first_ct_id, _ptr(out), _stream(stream)))

    def encode_encrypt(self, slots, scale, first_ct_id, out, stream=None):
        n = _rows(slots)
        _dev(slots, (n, self.N // 2), "float64", "slots")
        self._ct(out, n, 2, self.L_top, "out")
        _check(lib().fhe_encode_encrypt(self.h, _ptr(slots), n, scale, first_ct_id, _ptr(out),
                                        _stream(stream)))

    def decrypt(self, ct, level, out, stream=None):
        n = _rows(ct)
        if self._lv(level):
            self._ct(ct, n, 2, level, "ct")
        _dev(out, (n, self.N), "int64", "out")
        _check(lib().fhe_decrypt(self.h, _ptr(ct), n, level, _ptr(out), _stream(stream)))

    def decode(self, m, scale, out, stream=None):
        n = _rows(m)
        _dev(m, (n, self.N), "int64", "m")
        _dev(out, (n, self.N // 2), "float64", "out")
        _check(lib().fhe_decode(self.h, _ptr(m), n, scale, _ptr(out), _stream(stream)))

    # -- layout ---------------------------------------------------------------
    def ntt(self, polys, rows, forward, stream=None):
        n = _rows(polys)
        if 1 <= rows <= self.L_top + 1:            # otherwise the library refuses the call
            _dev(polys, (n, rows, self.N), "int64", "polys")
        _check(lib().fhe_ntt(self.h, _ptr(polys), n, rows, 1 if forward else 0, _stream(stream)))

    def ct_convert(self, ct, level, to_coeff, out, stream=None):
        n = _rows(ct)
        if self._lv(level):
            self._ct(ct, n, 2, level, "ct")
            self._ct(out, n, 2, level, "out")
        _check(lib().fhe_ct_convert(self.h, _ptr(ct), n, level, 1 if to_coeff else 0, _ptr(out),
                                    _stream(stream)))

    # -- operations -----------------------------------------------------------
    def add(self, a, b, level, out, stream=None):
        n = _rows(a)
        if self._lv(level):
            for t, nm in ((a, "a"), (b, "b"), (out, "out")):
                self._ct(t, n, 2, level, nm)
        _check(lib().fhe_add(self.h, _ptr(a), _ptr(b), n, level, _ptr(out), _stream(stream)))

    def tensor(self, a, b, level, out, stream=None):
        n = _rows(a)
        if self._lv(level):
            self._ct(a, n, 2, level, "a")
            self._ct(b, n, 2, level, "b")
            self._ct(out, n, 3, level, "out")
        _check(lib().fhe_tensor(self.h, _ptr(a), _ptr(b), n, level, _ptr(out), _stream(stream)))

    def galois_keygen(self, steps, stream=None):
        """Rotation keys for the given slot steps (parent context)."""
        arr = _arr([int(v) for v in steps], ctypes.c_int32)
        _check(lib().fhe_galois_keygen(self.h, arr, len(steps), _stream(stream)))

    def rotate(self, ct, level, step, out, stream=None):
        n = _rows(ct)
        if self._lv(level):
            self._ct(ct, n, 2, level, "ct")
            self._ct(out, n, 2, level, "out")
        _check(lib().fhe_rotate(self.h, _ptr(ct), n, level, int(step), _ptr(out), _stream(stream)))

    def relinearise(self, d3, level, out, stream=None):
        n = _rows(d3)
        if self._lv(level):
            self._ct(d3, n, 3, level, "d3")
            self._ct(out, n, 2, level, "out")
        _check(lib().fhe_relinearise(self.h, _ptr(d3), n, level, _ptr(out), _stream(stream)))

    def relinearise_noalloc(self, d3, level, out, stream=None):
        """fhe_relinearise without allocating: scratch from the library's fixed
        16 MiB device array (see include/fhe.h)."""
        n = _rows(d3)
        if self._lv(level):
            self._ct(d3, n, 3, level, "d3")
            self._ct(out, n, 2, level, "out")
        _check(lib().fhe_relinearise_noalloc(self.h, _ptr(d3), n, level, _ptr(out), _stream(stream)))

    def rescale(self, x, comps, level, out, stream=None):
        n = _rows(x)
        if self._lv(level, 2):
            self._ct(x, n, comps, level, "x")
            self._ct(out, n, comps, level - 1, "out")
        _check(lib().fhe_rescale(self.h, _ptr(x), n, comps, level, _ptr(out), _stream(stream)))

    def mul_relin_rescale(self, a, b, level, out, stream=None):
        n = _rows(a)
        if self._lv(level, 2):
            self._ct(a, n, 2, level, "a")
            self._ct(b, n, 2, level, "b")
            self._ct(out, n, 2, level - 1, "out")
        _check(lib().fhe_mul_relin_rescale(self.h, _ptr(a), _ptr(b), n, level, _ptr(out),
                                           _stream(stream)))

    def mul_relin_rescale_levels(self, batches, stream=None):
        """batches: list of (a, b, out, level) tensors; every step is one
        launch over all batches."""
        arr = (LevelBatch * max(1, len(batches)))()
        for k, (a, b, out, level) in enumerate(batches):
            n = _rows(a)
            if self._lv(level, 2):
                self._ct(a, n, 2, level, "a")
                self._ct(b, n, 2, level, "b")
                self._ct(out, n, 2, level - 1, "out")
            arr[k] = LevelBatch(a.data_ptr(), b.data_ptr(), out.data_ptr(), n, level)
        _check(lib().fhe_mul_relin_rescale_levels(self.h, arr, len(batches), _stream(stream)))

    def mul_const(self, x, consts, level, out, stream=None):
        n = _rows(x)
        if self._lv(level):
            self._ct(x, n, 2, level, "x")
            self._ct(out, n, 2, level, "out")
        c = np.ascontiguousarray(consts, dtype=np.int64)
        if c.shape != (n,):
            raise ValueError("one constant per ciphertext expected")
        _check(lib().fhe_mul_const(self.h, _ptr(x), c.ctypes.data_as(ctypes.c_void_p), n, level,
                                   _ptr(out), _stream(stream)))

    def add_const(self, x, consts, level, stream=None):
        n = _rows(x)
        if self._lv(level):
            self._ct(x, n, 2, level, "x")
        c = np.ascontiguousarray(consts, dtype=np.int64)
        if c.shape != (n,):
            raise ValueError("one constant per ciphertext expected")
        _check(lib().fhe_add_const(self.h, _ptr(x), c.ctypes.data_as(ctypes.c_void_p), n, level,
                                   _stream(stream)))


def _rows(t):
    if getattr(t, "dim", None) is None or t.dim() < 1:
        raise ValueError("a batched tensor is expected")
    return int(t.shape[0])


def _dev(t, shape, dtype, name):
    """t must be a contiguous CUDA tensor of `dtype` and `shape` on the current device."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.dtype != getattr(torch, dtype):
        raise ValueError("%s: dtype %s, expected %s" % (name, t.dtype, dtype))
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError("%s must live on the current CUDA device" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s: shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


class Graph:
    """A network graph (workload dict) copied into the library."""

    def __init__(self, graph):
        self._arrays = _GraphArrays(graph)
        h = ctypes.c_void_p()
        _check(lib().fhe_graph_create(ctypes.byref(self._arrays.desc), ctypes.byref(h)))
        self.h = h
        self.in_sizes = [int(n.get("n", 0)) for n in graph["nodes"] if n["kind"] == "input"]
        self.n_inputs = len(self.in_sizes)
        self._out_shape = {}

    def close(self):
        if getattr(self, "h", None):
            lib().fhe_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, ctx):
        n = ctypes.c_uint32()
        L = ctypes.c_uint32()
        _check(lib().fhe_graph_outputs(ctx.h, self.h, ctypes.byref(n), ctypes.byref(L)))
        return n.value, L.value

    def _outs(self, ctx):
        key = (ctx.N, tuple(ctx.primes))
        if key not in self._out_shape:
            self._out_shape[key] = self.outputs(ctx)
        return self._out_shape[key]

    def eval(self, ctx, inputs, out, stream=None):
        """inputs: list of ciphertext tensors, one per input node; out: tensor
        [n_out][2][out_level][N].  Returns a list of (level, scale)."""
        if len(inputs) != self.n_inputs:
            raise ValueError("%d input tensors for %d input nodes" % (len(inputs), self.n_inputs))
        for k, (t, n) in enumerate(zip(inputs, self.in_sizes)):
            ctx._ct(t, n, 2, ctx.L_top, "inputs[%d]" % k)
        n_out, L_out = self._outs(ctx)
        ctx._ct(out, n_out, 2, L_out, "out")
        arr = (ctypes.c_void_p * len(inputs))(*[t.data_ptr() for t in inputs])
        cap = out.shape[0]
        meta = (CtMeta * max(1, cap))()
        _check(lib().fhe_eval_graph(ctx.h, self.h, arr, len(inputs), _ptr(out), meta, cap, _stream(stream)))
        return [(meta[i].level, meta[i].scale) for i in range(cap)]

    def autoparam(self, log_scale=40, special_mult=1.5):
        """(N, coefficient-modulus bits) of one parameter set for the whole graph."""
        N = ctypes.c_uint32()
        bits = (ctypes.c_uint32 * 64)()
        nb = ctypes.c_uint32()
        _check(lib().fhe_autoparam(self.h, log_scale, special_mult, ctypes.byref(N), bits, 64, ctypes.byref(nb)))
        return N.value, [bits[i] for i in range(nb.value)]

    def eval_batch(self, ctx, requests, first_ct_id, stream=None):
        """requests: list of (x, y) float64 tensors (device or pinned host),
        x [n_in][>= n] and y [n_out][>= n] with unit column stride, or
        (x, y, n) to use only the first n columns.  Packs them into the slots,
        encrypts, evaluates, decrypts and decodes in one call."""
        import torch
        if self.n_inputs != 1:
            raise ValueError("eval_batch needs a graph with exactly one input node")
        n_out, _ = self._outs(ctx)
        arr = (Request * max(1, len(requests)))()
        for k, rq in enumerate(requests):
            x, y = rq[0], rq[1]
            n = rq[2] if len(rq) > 2 else x.shape[1]
            if x.dim() != 2 or y.dim() != 2 or x.shape[0] != self.in_sizes[0] or y.shape[0] != n_out:
                raise ValueError("request %d: x must be [%d][>= n], y [%d][>= n]" % (k, self.in_sizes[0], n_out))
            if x.dtype != torch.float64 or y.dtype != torch.float64 or x.stride(1) != 1 or y.stride(1) != 1:
                raise ValueError("requests take float64 tensors with unit column stride")
            if not 0 < n <= min(x.shape[1], y.shape[1]):
                raise ValueError("request %d: %d samples do not fit its buffers" % (k, n))
            arr[k] = Request(x.data_ptr(), n, x.stride(0), y.data_ptr(), y.stride(0))
        _check(lib().fhe_eval_batch(ctx.h, self.h, arr, len(requests), first_ct_id, _stream(stream)))


def raw_u64(t):
    """Device int64 tensor of raw residues -> host numpy uint64 array."""
    return t.detach().cpu().numpy().view(np.uint64)
