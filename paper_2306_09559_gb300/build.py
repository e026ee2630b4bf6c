"""Build libmpmc.so (sm_103a) in-tree with nvcc; no torch, no cmake.

Each .cu translation unit compiles in parallel to an object under
``paper_2306_09559_gb300/_build/`` and the objects link into
``paper_2306_09559_gb300/libmpmc.so``.  A unit is rebuilt only when its
source, a header, or the flags changed.
"""

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmpmc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libmpmc.so")
    return path


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_digest():
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                h.update(f.encode())
                h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def _compile(src, extra, hdr):
    obj = os.path.join(BUILD, src[:-3] + ".o")
    stamp = obj + ".key"
    key = hashlib.sha256((open(os.path.join(CSRC, src), "rb").read().hex() + hdr
                          + " ".join(ARCH + FLAGS + extra)).encode()).hexdigest()
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == key:
        return obj, None
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, r.stdout + r.stderr
    open(stamp, "w").write(key)
    return obj, (r.stderr or None)


def build(verbose=False, ptxas_info=False):
    """Compile every CUDA source and link libmpmc.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    hdr = _headers_digest()
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, hdr), srcs))
    errors = [(s, msg) for s, (o, msg) in zip(srcs, results) if msg and ("error" in msg.lower())]
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {s}\n{m}" for s, m in errors))
    if verbose:
        for s, (o, msg) in zip(srcs, results):
            if msg:
                print(f"--- {s}\n{msg}", file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
