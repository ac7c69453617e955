"""Build ``libsnn.so`` (the sm_103a CUDA library behind ``include/snn.h``)
and its bounds-checked variant ``libsnn_check.so`` (the same sources with
``-DSNN_CHECK=1``; the binding loads it when ``SNN_CHECKED=1`` is set).

The translation units of both are compiled in parallel with nvcc for
``arch=compute_103a,code=sm_103a`` and linked into shared libraries inside
the package directory (kept in-tree, next to the binding that loads them).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsnn.so")
LIB_CHECKED = os.path.join(PKG, "libsnn_check.so")
SOURCES = ["snn_kernels.cu", "snn_build.cu", "snn_api.cu", "snn_serve.cu",
           "snn_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2", f"-I{os.path.join(ROOT, 'include')}"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build "
                       "libsnn")


def _inputs_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "snn.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def lib_path() -> str:
    """The library the binding loads: the bounds-checked variant when the
    environment sets SNN_CHECKED=1, else the production one."""
    return LIB_CHECKED if os.environ.get("SNN_CHECKED") == "1" else LIB


def _fresh(lib: str) -> bool:
    return os.path.exists(lib) and os.path.getmtime(lib) >= _inputs_mtime()


def build(force: bool = False, verbose: bool = False) -> str:
    """Build both variants (the stale ones); returns the loaded variant's
    path."""
    todo = [(lib, chk) for lib, chk in ((LIB, False), (LIB_CHECKED, True))
            if force or not _fresh(lib)]
    if not todo:
        return lib_path()
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(job):
        src, chk = job
        out = OUT_DIR + ("_check" if chk else "")
        os.makedirs(out, exist_ok=True)
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *(["-DSNN_CHECK=1"] if chk else []), *extra,
               "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    jobs = [(src, chk) for _, chk in todo for src in SOURCES]
    with ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, _) in enumerate(todo):
        tmp = lib + ".tmp%d" % os.getpid()
        mine = objs[k * len(SOURCES):(k + 1) * len(SOURCES)]
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *mine],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib_path()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
