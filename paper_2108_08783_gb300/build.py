"""Build ``liblbm.so`` (the C-ABI library of ``include/lbm.h``) in place for sm_103a.

The four translation units are compiled in parallel with nvcc (one
``-gencode`` for sm_103a, ``-lineinfo`` for profiling) and linked into a
shared object next to this file, with the CUDA runtime linked statically.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblbm.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["lattice_build.cpp", "kernels.cu", "capi.cu", "mlp.cu"]
HEADERS = ["lbm_internal.h", "d3q19.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(HERE, "..", "include", "lbm.h"))
    files.append(os.path.join(HERE, "..", "include", "lbm_mlp.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src, extra, bdir):
    obj = os.path.join(bdir, src + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xptxas", "-warn-spills", *extra, "-c", path, "-o", obj]
    else:
        cmd = [NVCC, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-c", path,
               "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=(), out=None):
    """Compile and link ``liblbm.so`` if any source is newer; return its path.

    ``extra`` adds nvcc flags (e.g. ``-DLBM_MINB_F32=4``); ``out`` writes the
    shared object elsewhere (with its own object directory) instead of the
    package's ``liblbm.so``."""
    lib = LIB if out is None else os.path.abspath(out)
    if out is None and not force and not _stale():
        return LIB
    bdir = BUILD if out is None else lib + ".objs"
    os.makedirs(bdir, exist_ok=True)
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra), bdir), SOURCES))
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, "-shared", *ARCH, "-o", tmp, *[o for o, _ in results], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
