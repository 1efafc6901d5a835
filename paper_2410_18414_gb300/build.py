"""Build libgpic.so (the CUDA library behind include/pic.h) in-tree for sm_103a.

Each .cu under csrc/ is compiled to an object in parallel, then linked into
paper_2410_18414_gb300/libgpic.so.  Objects go to paper_2410_18414_gb300/_build/.
A translation unit is rebuilt when it or any header it may include is newer than
its object.

    python -m paper_2410_18414_gb300.build [--force] [--debug] [--sanitize]

--sanitize builds libgpic_asan.so (objects in _build_asan/) with the host code under
AddressSanitizer and UndefinedBehaviorSanitizer, for the host-side tests of the C ABI
(load it with the gcc runtime preloaded: LD_PRELOAD=$(gcc -print-file-name=libasan.so)).
"""
import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgpic.so")
BUILD_ASAN = os.path.join(HERE, "_build_asan")
LIB_ASAN = os.path.join(HERE, "libgpic_asan.so")
# host-side sanitizers (device code is unaffected); one flag per -Xcompiler, as nvcc
# splits its argument at commas
SANITIZE = ["-Xcompiler=-fsanitize=address", "-Xcompiler=-fsanitize=undefined",
            "-Xcompiler=-fno-omit-frame-pointer"]
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libgpic)")


def _flags(debug):
    f = ARCH + ["-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    f += ["-O0", "-G"] if debug else ["-O3"]
    return f


def _stale(obj, src, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + headers)


def build(force=False, debug=False, verbose=False, sanitize=False):
    nvcc = nvcc_path()
    build_dir, lib = (BUILD_ASAN, LIB_ASAN) if sanitize else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                     + glob.glob(os.path.join(INCLUDE, "*.h")))
    flags = _flags(debug) + (SANITIZE if sanitize else [])
    jobs = []
    for src in sources:
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, src, headers):
            jobs.append([nvcc, "-c", src, "-o", obj] + flags)
    objs = [os.path.join(build_dir, os.path.basename(s)[:-3] + ".o") for s in sources]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed on " + cmd[2])
    if force or jobs or not os.path.exists(lib) or any(
            os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        cmd = [nvcc, "-shared", "-o", lib] + objs + ARCH + ["-lcudart_static", "-lrt", "-ldl",
                                                              "-lpthread"]
        if sanitize:
            cmd += SANITIZE
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link of " + os.path.basename(lib) + " failed")
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--debug", action="store_true")
    ap.add_argument("--sanitize", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, debug=a.debug, verbose=a.verbose, sanitize=a.sanitize))
