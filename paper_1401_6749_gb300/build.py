"""Build the tmloops C-ABI library (libtmloops.so) in-tree for sm_103a.

Each translation unit in csrc/ is compiled by nvcc in parallel, then linked
into one shared library next to this file.  Rebuilds only when the contents
of a source, a header or the flags differ from those the library was built
from (a hash in _build/flags.txt; file times play no part).  Concurrent
callers (e.g. the ranks of a torchrun job) serialise on a lock file: the
first builds, the others find the library up to date.
"""
import contextlib
import fcntl
import glob
import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtmloops.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress=177",
              "-I", INCLUDE, "-I", CSRC] + ARCH


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the tmloops CUDA library cannot be built")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


STAMP = os.path.join(BUILD, "flags.txt")


def _extra_flags():
    """Extra nvcc flags from TMLOOPS_EXTRA_NVCC (tuning builds, e.g. -DTM_DSLASH_MINBLOCKS=8)."""
    return os.environ.get("TMLOOPS_EXTRA_NVCC", "").split()


def _fingerprint():
    """Hash of the flags and of every source and header the library is built from."""
    h = hashlib.sha256(" ".join(NVCC_FLAGS + _extra_flags()).encode())
    for d in sorted(_deps()):
        h.update(os.path.relpath(d, ROOT).encode())
        with open(d, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return False
    with open(STAMP) as f:
        return f.read().strip() == _fingerprint()


@contextlib.contextmanager
def build_lock():
    """Exclusive lock of the build directory (blocks until it is free)."""
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as fh:
        fcntl.flock(fh, fcntl.LOCK_EX)
        try:
            yield
        finally:
            fcntl.flock(fh, fcntl.LOCK_UN)


def build(force=False, verbose=False, jobs=None):
    """Compile csrc/*.cu and link libtmloops.so; returns the library path."""
    if not force and up_to_date():
        return LIB
    with build_lock():
        if not force and up_to_date():  # another process built it meanwhile
            return LIB
        return _build(verbose, jobs)


def _build(verbose, jobs):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    fp = _fingerprint()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + _extra_flags() + ["-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, res.stdout, res.stderr))
        if verbose and (res.stdout or res.stderr):
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath", "-Xlinker", "/usr/local/cuda/lib64"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (res.stdout, res.stderr))
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(fp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
