"""Build libmgrit.so in-tree for sm_103a with nvcc (one -gencode, parallel TUs)."""
import os
import shutil
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmgrit.so")
# MGRIT_DEBUG variant: bounds checks on every shared/global index (prints and
# skips a bad access instead of faulting)
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libmgrit_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "mgrit.h"))
    return max(os.path.getmtime(h) for h in hs)


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmgrit.so")
    return exe


def build(force=False, verbose=False, extra=(), debug=False):
    """Compile every .cu under csrc/ and link libmgrit.so (static cudart);
    debug=True builds libmgrit_debug.so with -DMGRIT_DEBUG."""
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if debug:
        extra = tuple(extra) + ("-DMGRIT_DEBUG",)
    os.makedirs(bdir, exist_ok=True)
    srcs = sources()
    hdr = _headers_mtime()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append([nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o])

    times = {}

    def run(cmd):
        t0 = time.time()
        r = subprocess.run(cmd, capture_output=True, text=True)
        times[os.path.basename(cmd[-3]) if cmd[-4] == "-c" else "link"] = time.time() - t0
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed for " + cmd[-3])
        return r.stdout + r.stderr

    # the kernel-table units instantiate the templates and take longest:
    # start them first so that the short units fill in around them
    jobs.sort(key=lambda cmd: (not os.path.basename(cmd[-3]).startswith("table_"), cmd[-3]))
    t_start = time.time()
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            outs = list(ex.map(run, jobs))
    else:
        outs = []
    if jobs or not os.path.exists(lib):
        tmp = lib + ".tmp.%d" % os.getpid()
        run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib)
    if times:
        slow = sorted(times.items(), key=lambda kv: -kv[1])[:4]
        sys.stderr.write("[build] %s: %d jobs in %.0f s; slowest %s\n" % (
            os.path.basename(lib), len(times), time.time() - t_start,
            ", ".join("%s %.0f s" % kv for kv in slow)))
    return "".join(outs)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else (),
                debug="--debug" in sys.argv))
