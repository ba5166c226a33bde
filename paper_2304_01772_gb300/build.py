"""Build libspinmc.so in-tree for sm_103a (nvcc for the kernels, g++ for the host ABI).

    python -m paper_2304_01772_gb300.build [--force] [--variant check|san]

Translation units compile in parallel; the shared library lands next to this
file and is what the Python binding loads.  Two test variants build beside it
(the binding loads one when SPINMC_LIBRARY names its path):

* check -> libspinmc_check.so: kernels compiled with -DSPIN_CHECK, so every
  work-list entry, shared-memory ring index and table address is checked
  before use; a failed check records an error code in a device word (the
  access is skipped, nothing traps) that spin_check_status reports.
* san -> libspinmc_san.so: host code built with AddressSanitizer and
  UndefinedBehaviorSanitizer (run with libasan preloaded).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
            f"-I{INCLUDE}", f"-I{CSRC}"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", f"-I{INCLUDE}", f"-I{CSRC}",
             f"-I{os.path.join(CUDA, 'include')}"]
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]
VARIANTS = {
    # name: (library file, extra nvcc flags, extra g++ flags, extra link flags)
    "": ("libspinmc.so", [], [], []),
    "check": ("libspinmc_check.so", ["-DSPIN_CHECK"], ["-DSPIN_CHECK"], []),
    "san": ("libspinmc_san.so", ["-Xcompiler", ",".join(SAN)], SAN, ["-Xcompiler", ",".join(SAN[:2])]),
}
OUT = os.path.join(HERE, VARIANTS[""][0])


def library_path(variant: str = "") -> str:
    return os.path.join(HERE, VARIANTS[variant][0])


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _newest_input():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "spinmc.h")]
    return max(os.path.getmtime(f) for f in files)


def _compile(args):
    src, variant = args
    _, cu_extra, cxx_extra, _ = VARIANTS[variant]
    path = os.path.join(CSRC, src)
    obj = os.path.join(ROOT, "_build", variant or "default", src + ".o")
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, *CU_FLAGS, *cu_extra, "-c", path, "-o", obj]
    else:
        cmd = ["g++", *CXX_FLAGS, *cxx_extra, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, variant: str = "") -> str:
    out = library_path(variant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_input():
        return out
    os.makedirs(os.path.join(ROOT, "_build", variant or "default"), exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(_compile, [(f, variant) for f in sources()]))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", *VARIANTS[variant][3], "-o", tmp,
           *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    v = sys.argv[sys.argv.index("--variant") + 1] if "--variant" in sys.argv else ""
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, variant=v))
