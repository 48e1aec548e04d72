"""Build step for the CUDA library libidx.so (sm_103a), placed beside this file.

nvcc cross-compiles for sm_103a without a GPU.  The library exports exactly the
C ABI of include/idx.h.

A second library, libidx_strict.so, is the same source compiled as a test build
(IDX_STRICT_ROUNDING, no FMA contraction): its FP64 kernels evaluate the method's
formulas in their plain written order with correctly rounded divisions.  Tests use it
to separate rounding order from the method; the product path loads libidx.so only.
"""
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libidx.so")
LIB_STRICT = os.path.join(HERE, "libidx_strict.so")
SOURCES = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
DEPS = SOURCES + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + [os.path.join(ROOT, "include", "idx.h")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-warn-spills"]
VARIANTS = {
    "default": (LIB, []),
    # the strict FP64 update returns early, which leaves the production path unreachable there
    "strict": (LIB_STRICT, ["-fmad=false", "-DIDX_STRICT_ROUNDING", "-diag-suppress", "128"]),
}


def _stale(path):
    newest = max(os.path.getmtime(p) for p in DEPS)
    return not os.path.exists(path) or os.path.getmtime(path) < newest


def _command(variant, verbose, tmp):
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    extra = VARIANTS[variant][1]
    return [nvcc] + NVCC_FLAGS + extra + (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp] + SOURCES


def build(force: bool = False, verbose: bool = False, variant: str = "default") -> str:
    """Compile one library variant if a source is newer than it (or force); returns its path."""
    path = VARIANTS[variant][0]
    if not force and not _stale(path):
        return path
    tmp = path + ".%d.tmp" % os.getpid()
    subprocess.run(_command(variant, verbose, tmp), check=True)
    os.replace(tmp, path)
    return path


def build_all(force: bool = False) -> list:
    """Compile every library variant, the stale ones side by side."""
    todo = [v for v, (path, _) in VARIANTS.items() if force or _stale(path)]
    procs = []
    for v in todo:
        path = VARIANTS[v][0]
        tmp = path + ".%d.tmp" % os.getpid()
        procs.append((v, path, tmp, subprocess.Popen(_command(v, False, tmp))))
    failed = []
    for v, path, tmp, p in procs:
        if p.wait() != 0:
            failed.append(v)
        else:
            os.replace(tmp, path)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    return [VARIANTS[v][0] for v in VARIANTS]


if __name__ == "__main__":
    import sys
    if "--all" in sys.argv:
        print(build_all(force=True))
    else:
        print(build(force=True, verbose="-v" in sys.argv,
                    variant="strict" if "--strict" in sys.argv else "default"))
