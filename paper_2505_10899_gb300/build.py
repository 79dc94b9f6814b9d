"""Build the CUDA library liblbm_gb300.so in-tree with nvcc for sm_103a.

The translation units (2-D and 3-D kernels per precision, host runtimes + C ABI)
are compiled in parallel and linked into one shared library under
``paper_2505_10899_gb300/_lib``.  Usage: ``python -m paper_2505_10899_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
SO_NAME = "liblbm_gb300.so"
SO_PATH = os.path.join(LIBDIR, SO_NAME)
SOURCES = ["kern_f32.cu", "kern_f64.cu", "lbm_api.cu", "lbm_adjoint.cu", "lbm_noalloc.cu",
           "kern3_f64.cu", "kern3_f32.cu", "kern3_f16.cu", "lbm3_api.cu", "lbm_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm_gb300.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                   "--expt-relaxed-constexpr", *extra]


def _newest_input() -> float:
    t = 0.0
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return max(t, os.path.getmtime(__file__))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    """Compile and link; returns the path of the shared library.  checked:
    the debug build with index checks in the step kernels (LBM_CHECK_BOUNDS),
    liblbm_gb300_checked.so beside the normal library."""
    so_path = SO_PATH.replace(".so", "_checked.so") if checked else SO_PATH
    objdir = OBJDIR + ("_checked" if checked else "")
    if (not force and os.path.exists(so_path)
            and os.path.getmtime(so_path) >= _newest_input()):
        return so_path
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if checked:
        extra = extra + ["-DLBM_CHECK_BOUNDS"]

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [cc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, err in results:
            sys.stderr.write(err)
    tmp = so_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, so_path)
    return so_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_info="--ptxas-info" in sys.argv, checked="--checked" in sys.argv))
