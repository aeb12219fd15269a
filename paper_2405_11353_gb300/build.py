"""Build libnttgb.so in place: nvcc for sm_103a, one object per .cu, in parallel.

Usage: python -m paper_2405_11353_gb300.build [--force] [--jobs N]
"""
import argparse
import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnttgb.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp"))
                  + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _digest(extra=""):
    h = hashlib.sha256()
    for p in _sources() + _headers():
        h.update(os.path.relpath(p, ROOT).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode() + extra.encode())
    return h.hexdigest()


# Sources of the fused forward transform with 4-byte words and Shoup
# twiddles (the two launches of the two-pass split the benchmark times).
FORWARD_U32_SOURCES = ("fused.cuh", "stream.cuh", "fused_launch.cuh", "modarith.cuh", "fused_u32_shoup.cu")


def kernel_digest(files=None):
    """Digest of kernel sources and headers (relative paths + contents):
    identifies the code an ncu capture was taken on.  `files`: names under
    csrc/ to cover (default: all of them)."""
    h = hashlib.sha256()
    paths = _sources() + _headers() if files is None else [os.path.join(CSRC, f) for f in files]
    for p in sorted(paths):
        h.update(os.path.relpath(p, ROOT).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _compile(src):
    obj = os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC] + ARCH + FLAGS + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj


def build(force=False, jobs=None, verbose=False):
    """Compile every kernel source for sm_103a and link libnttgb.so."""
    os.makedirs(OBJ, exist_ok=True)
    stamp = os.path.join(OBJ, "digest")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    jobs = jobs or min(len(_sources()), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(_compile, _sources()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcuda"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    a = ap.parse_args()
    build(force=a.force, jobs=a.jobs, verbose=True)
    sys.exit(0)
