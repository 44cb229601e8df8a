"""Build the CUDA library libptahmc.so in-tree for sm_103a (B300), and its check build
libptahmc_check.so (nvcc -DPTA_CHECK: every instrumented tile index, unit offset, bulk-copy and
TMA coordinate is tested before use; a failure skips the access and the call returns
PTA_ECHECK naming it).  Python loads the check build when PTA_CHECK_BUILD=1."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libptahmc.so")
LIB_CHECK = os.path.join(HERE, "libptahmc_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(HERE, "..", "include", "ptahmc.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(verbose: bool = False, force: bool = False, extra=(), check: bool = False) -> str:
    lib = LIB_CHECK if check else LIB
    if not force and not needs_build(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(HERE, "_build_check" if check else "_build")
    if check:
        extra = list(extra) + ["-DPTA_CHECK"]
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
                    "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3"] + list(extra)
    from concurrent.futures import ThreadPoolExecutor

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        r = subprocess.run([nvcc, "-c", src, "-o", obj] + flags, capture_output=True, text=True)
        return src, obj, r

    objs = []
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for src, obj, r in ex.map(compile_one, sources()):
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            objs.append(obj)
    cmd = [nvcc, "-shared", "-o", lib] + objs + ARCH + ["-Xcompiler", "-fopenmp", "-lcudart", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, check="--check" in sys.argv))
