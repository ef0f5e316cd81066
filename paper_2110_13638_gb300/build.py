"""Build libfhe.so (the sm_103a CUDA library behind include/fhe.h) in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2110_13638_gb300/csrc/_build/libfhe.so.  Host code is compiled with
-ffp-contract=off so FP64 constant encodings round identically on every host.
"""
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(CSRC, "_build")
SO = os.path.join(BUILD, "libfhe.so")
ROOT = os.path.dirname(HERE)

# the transform-heavy units first, so the parallel build starts them earliest
SOURCES = ["k_relin_modup.cu", "k_relin_tensor.cu", "k_persist.cu", "k_modup_cluster.cu", "k_keys.cu", "k_encrypt.cu", "k_groups_ks.cu", "k_groups.cu", "k_groups_fwd.cu", "k_relin.cu",
           "k_rescale.cu", "k_common.cu", "k_encode.cu", "k_mac.cu", "k_mac_tc.cu", "capi.cu", "graph.cu", "batch.cu", "noalloc.cu", "k_peak.cu",
           "host_math.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                   "-I" + os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "fhe.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def _stamp_ok():
    """Objects built on another machine (architecture) are never reused."""
    stamp = os.path.join(BUILD, "STAMP")
    want = platform.machine() + " " + " ".join(ARCH)
    ok = os.path.exists(stamp) and open(stamp).read().strip() == want
    return ok, stamp, want


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    ok, stamp, want = _stamp_ok()
    force = force or not ok
    cc = nvcc()
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, os.path.splitext(s)[0] + ".o")
        if force or _stale(obj, src):
            cmd = [cc] + _flags() + ["-x", "cu" if s.endswith(".cu") else "c++", "-c", src, "-o", obj]
            if s.endswith(".cpp"):
                cmd = [cc] + _flags() + ["-c", src, "-o", obj]
            jobs.append((s, cmd))

    def run(job):
        name, cmd = job
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (name, p.stdout, p.stderr))
        return p.stderr

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out:
                print(out, file=sys.stderr)
    objs = [os.path.join(BUILD, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    if force or jobs or not os.path.exists(SO):
        tmp = SO + ".tmp%d" % os.getpid()
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (p.stdout, p.stderr))
        os.replace(tmp, SO)
    with open(stamp, "w") as f:
        f.write(want + "\n")
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
