"""In-tree build of the msp CUDA library (sm_103a) with nvcc + g++.

Produces paper_2412_08981_gb300/_build/libmsp.so.  Translation units are
compiled in parallel; only the sources that changed are rebuilt.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmsp.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
            "--expt-relaxed-constexpr",
            "-I" + INCLUDE, "-I" + CSRC] + ARCH
# no FMA contraction in host set-up code: the same weights on x86 and on Arm
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-ffp-contract=off",
             "-I" + INCLUDE, "-I" + CSRC,
             "-I/usr/local/cuda/include"]


def _sources():
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))
    return [os.path.join(CSRC, f) for f in srcs]


def _headers_digest():
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _obj_for(src, digest):
    with open(src, "rb") as fh:
        tag = hashlib.sha256(fh.read()).hexdigest()[:16]
    base = os.path.basename(src).replace(".", "_")
    return os.path.join(OUT_DIR, f"{base}.{tag}.{digest}.o")


def _compile(src, obj, verbose):
    if os.path.exists(obj):
        return obj
    if src.endswith(".cu"):
        cmd = [NVCC] + CU_FLAGS + ["-c", src, "-o", obj + ".tmp"]
    else:
        cmd = ["g++"] + CXX_FLAGS + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libmsp.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    digest = _headers_digest()
    srcs = _sources()
    objs = [_obj_for(s, digest) for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        list(ex.map(lambda so: _compile(so[0], so[1], verbose), zip(srcs, objs)))
    stamp = LIB + ".inputs"
    want = "\n".join(objs)
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == want:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(want)
    # drop stale objects
    keep = set(objs)
    for f in os.listdir(OUT_DIR):
        p = os.path.join(OUT_DIR, f)
        if f.endswith(".o") and p not in keep:
            os.remove(p)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
