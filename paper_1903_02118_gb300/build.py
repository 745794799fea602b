"""Build the CUDA library libfdph.so in-tree for sm_103a (no torch extension machinery).

Each translation unit is compiled in parallel by nvcc, then linked into
``paper_1903_02118_gb300/libfdph.so``.  Host code is compiled with
``-ffp-contract=off`` so that the plan's tree and integer decisions are
reproducible bit for bit.

``build(check=True)`` builds the bounded-index debug library ``libfdph_check.so`` instead: the
device translation units are compiled with ``-DFDPH_CHECK`` (index checks on every ring, state,
partial-sum and near-slice access of the step kernels, canaries after every plan allocation);
the host units are shared with the normal build.  The binding loads it when the environment
variable ``FDPH_LIB`` is ``check``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfdph.so")
LIB_CHECK = os.path.join(HERE, "libfdph_check.so")
SOURCES = ["fdph.cu", "noalloc.cu", "tree.cpp", "lra.cpp", "plan.cpp"]
DEVICE_SOURCES = ["fdph.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfdph.so")
    return exe


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-I", os.path.join(HERE, "..", "include"),
            "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off,-O2", "--expt-relaxed-constexpr"]


def build(verbose=False, force=False, check=False):
    os.makedirs(BUILD, exist_ok=True)
    lib = LIB_CHECK if check else LIB
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "fdph.h"))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in deps):
        return lib
    cc = nvcc()

    def compile_one(src):
        checked = check and os.path.basename(src) in DEVICE_SOURCES
        obj = os.path.join(BUILD, os.path.basename(src) + (".check.o" if checked else ".o"))
        if check and not checked and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
            return obj, ""   # host units are the normal build's
        cmd = [cc, *_flags(), *(["-DFDPH_CHECK"] if checked else []), "-c", src, "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        else:
            cmd = [cc, *_flags(), "-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for obj, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, check="--check" in sys.argv))
