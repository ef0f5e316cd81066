"""ctypes loader for the oracle's C arithmetic core (oracle/ckks_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle is imported by tests/, by
__graft_entry__.smoke() and by the CPU-baseline leg of bench.py, never by the
product path.  It shares no code with the CUDA library.
"""
import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force=False):
    """Compile the C core with gcc (plain -O2, no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = os.path.join(_BUILD, "STAMP")
    want = platform.machine()
    same_machine = os.path.exists(stamp) and open(stamp).read().strip() == want
    if (not force and same_machine and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    libs = ["-lquadmath"] if platform.machine() == "x86_64" else ["-lm"]
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-ffp-contract=off",
           _SRC, "-o", tmp] + libs
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    with open(stamp, "w") as f:
        f.write(want + "\n")
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u64, i64, u32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
        P = ctypes.c_void_p
        sig = {
            "o_mulmod": (u64, [u64, u64, u64]),
            "o_powmod": (u64, [u64, u64, u64]),
            "o_vec_mul_scalar": (None, [P, ctypes.c_size_t, u64, u64]),
            "o_vec_mul": (None, [P, P, P, ctypes.c_size_t, u64]),
            "o_vec_mac_scalar": (None, [P, P, ctypes.c_size_t, u64, u64]),
            "o_ntt": (None, [P, u32, u64, u64]),
            "o_intt": (None, [P, u32, u64, u64]),
            "o_polymul": (None, [P, P, P, u32, u64, u64]),
            "o_polymul_schoolbook": (None, [P, P, P, u32, u64]),
            "o_splitmix_out": (u64, [u64, u64]),
            "o_stream": (u64, [u64, u64, u64]),
            "o_sample_uniform": (None, [u64, u32, u64, u32, P]),
            "o_sample_ternary": (None, [u64, u32, P]),
            "o_sample_gauss": (None, [u64, u32, P, u32, P]),
            "o_encode": (ctypes.c_int, [P, u32, dbl, P, P]),
            "o_decode": (None, [P, u32, dbl, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a


# ---- thin numpy wrappers ---------------------------------------------------

def mulmod(a, b, q):
    return int(lib().o_mulmod(int(a), int(b), int(q)))


def vec_mul_scalar(a, c, q):
    """Return a * c mod q elementwise (a: uint64 array)."""
    out = _u64(a).copy()
    lib().o_vec_mul_scalar(_ptr(out), out.size, int(c) % int(q), int(q))
    return out


def vec_mul(a, b, q):
    a = _u64(a)
    b = _u64(b)
    out = np.empty_like(a)
    lib().o_vec_mul(_ptr(a), _ptr(b), _ptr(out), a.size, int(q))
    return out


def vec_mac_scalar(acc, a, c, q):
    """In place: acc = acc + a * c mod q."""
    a = _u64(a)
    assert acc.dtype == np.uint64 and acc.flags.c_contiguous
    lib().o_vec_mac_scalar(_ptr(acc), _ptr(a), a.size, int(c) % int(q), int(q))


def ntt(a, q, psi):
    out = _u64(a).copy()
    lib().o_ntt(_ptr(out), out.size, int(q), int(psi))
    return out


def intt(a, q, psi):
    out = _u64(a).copy()
    lib().o_intt(_ptr(out), out.size, int(q), int(psi))
    return out


def polymul(a, b, q, psi):
    a = _u64(a)
    b = _u64(b)
    out = np.empty_like(a)
    lib().o_polymul(_ptr(a), _ptr(b), _ptr(out), a.size, int(q), int(psi))
    return out


def polymul_schoolbook(a, b, q):
    a = _u64(a)
    b = _u64(b)
    out = np.empty_like(a)
    lib().o_polymul_schoolbook(_ptr(a), _ptr(b), _ptr(out), a.size, int(q))
    return out


def stream(seed, domain, obj):
    return int(lib().o_stream(int(seed) & (2**64 - 1), int(domain), int(obj) & (2**64 - 1)))


def splitmix_out(state, i):
    return int(lib().o_splitmix_out(int(state), int(i)))


def sample_uniform(s0, residue, q, N):
    out = np.empty(N, dtype=np.uint64)
    lib().o_sample_uniform(int(s0), int(residue), int(q), int(N), _ptr(out))
    return out


def sample_ternary(s0, N):
    out = np.empty(N, dtype=np.int64)
    lib().o_sample_ternary(int(s0), int(N), _ptr(out))
    return out


def sample_gauss(s0, N, cdt):
    cdt = np.ascontiguousarray(cdt, dtype=np.uint64)
    kmax = cdt.size // 2
    out = np.empty(N, dtype=np.int64)
    lib().o_sample_gauss(int(s0), int(N), _ptr(cdt), kmax, _ptr(out))
    return out


def encode(z, N, scale, want_frac=False):
    z = np.ascontiguousarray(z, dtype=np.float64)
    assert z.size == N // 2
    m = np.empty(N, dtype=np.int64)
    frac = np.empty(N, dtype=np.float64) if want_frac else None
    rc = lib().o_encode(_ptr(z), int(N), float(scale), _ptr(m),
                        _ptr(frac) if want_frac else None)
    if rc != 0:
        raise OverflowError("encoded coefficient does not fit in int64")
    return (m, frac) if want_frac else m


def decode(m, N, scale):
    m = np.ascontiguousarray(m, dtype=np.int64)
    re = np.empty(N // 2, dtype=np.float64)
    im = np.empty(N // 2, dtype=np.float64)
    lib().o_decode(_ptr(m), int(N), float(scale), _ptr(re), _ptr(im))
    return re, im
