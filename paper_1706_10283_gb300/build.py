"""Build libbolt.so (the C-ABI CUDA library) in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo``, then linked into
``paper_1706_10283_gb300/libbolt.so`` with the static CUDA runtime.

``build(stamps=True)`` makes the diagnostic variant ``libbolt_stamps.so``
(``-DBOLT_PHASE_STAMPS``: the top-k kernels record per-CTA phase times,
read by ``phases.py``); the library itself never contains the stamps.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbolt.so")
BUILD_STAMPS = os.path.join(HERE, "_build_stamps")
LIB_STAMPS = os.path.join(HERE, "libbolt_stamps.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _flags(verbose):
    f = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wall", "-Xcompiler", "-ffp-contract=off"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(HERE, "..", "include", "*.h"))


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False, jobs=None, stamps=False):
    lib, bdir = (LIB_STAMPS, BUILD_STAMPS) if stamps else (LIB, BUILD)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    extra = ["-DBOLT_PHASE_STAMPS"] if stamps else []

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc()] + _flags(verbose) + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, zip(srcs, objs)))
    failed = [(s, out) for s, rc, out in results if rc != 0]
    for s, rc, out in results:
        if out.strip() and (verbose or rc != 0):
            sys.stderr.write("== %s\n%s\n" % (os.path.basename(s), out))
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(s) for s, _ in failed))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, stamps="--stamps" in sys.argv))
