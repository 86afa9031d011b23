"""Build libtpx.so in-tree for sm_103a with nvcc (no cmake, no torch)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtpx.so")
# the checked build (-DTPX_CHECKED: the fused kernel tests every data-dependent
# index and reports a violation in the status word instead of touching memory)
CHECKED_LIB = os.path.join(OUT_DIR, "libtpx_checked.so")
# the phase-timing build (-DTPX_PHASE_TIMING: per-phase clock64 counters in
# the fused kernel, read with tpx_debug_phase_times)
PHASES_LIB = os.path.join(OUT_DIR, "libtpx_phases.so")
SOURCES = ["tpx_fused.cu", "tpx_prepass.cu", "tpx_runtime.cu", "tpx_noalloc.cu", "tpx_general.cu", "tpx_stream.cu",
           "tpx_refine.cu", "tpx_cnn.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "-I" + CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtpx")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "tpx.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False, phases: bool = False) -> str:
    lib = CHECKED_LIB if checked else PHASES_LIB if phases else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    extra = ["-DTPX_CHECKED"] if checked else ["-DTPX_PHASE_TIMING"] if phases else []
    tag = "chk." if checked else "ph." if phases else ""

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", f".{tag}{os.getpid()}.o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
