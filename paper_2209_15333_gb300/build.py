"""Build the CUDA library ``_build/libcfd_gb300.so`` for sm_103a with nvcc.

One translation unit, one -gencode, static CUDA runtime; no torch headers.
``checked=True`` builds ``_build/libcfd_gb300_checked.so`` with index-bounds
checks in the kernels (CFD_BOUNDS_CHECK): an out-of-range node index sets an
error word and skips the access instead of trapping.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcfd_gb300.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libcfd_gb300_checked.so")
SOURCES = [os.path.join(CSRC, "cfd_api.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(ROOT, "include", "cfd.h"), __file__]

FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC", "-shared", "-cudart", "static", "--expt-relaxed-constexpr"]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib):
        if os.path.getmtime(lib) >= max(os.path.getmtime(p) for p in DEPS if os.path.exists(p)):
            return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *FLAGS, *(["-DCFD_BOUNDS_CHECK"] if checked else []), *(["-Xptxas", "-v"] if verbose else []),
           *SOURCES, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stderr[-20000:])
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
