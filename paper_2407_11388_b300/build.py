"""Build librac.so (the CUDA library behind include/rac.h) for sm_103a.

    python -m paper_2407_11388_b300.build [--force] [--verbose]

nvcc cross-compiles without a GPU.  The library links the CUDA runtime
statically, so it only needs the driver at run time."""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "librac.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object in parallel (one nvcc per file), then
    link the shared library; returns its path."""
    if not force and not _stale():
        return LIB
    import shutil
    import tempfile
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
             "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC,
             "--expt-relaxed-constexpr"]
    if verbose:
        flags = ["-Xptxas", "-v", *flags]
    objdir = tempfile.mkdtemp(prefix="racbuild")
    try:
        srcs = sources()
        objs = [os.path.join(objdir, os.path.basename(p) + ".o") for p in srcs]
        # the slowest files first, so that the pool ends with the quick ones
        jobs = sorted(zip(srcs, objs), key=lambda so: -os.path.getsize(so[0]))
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as pool:
            for f in [pool.submit(subprocess.check_call, [nvcc, *flags, "-c", src, "-o", obj])
                      for src, obj in jobs]:
                f.result()
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
