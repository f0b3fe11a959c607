"""Build the CUDA library liblabs_gb300.so in-tree for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process in parallel, then
linked into one shared library with a plain C ABI (include/labs.h).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "liblabs_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + os.path.join(ROOT, "include")]

SOURCES = ["walk_kernels.cu", "walk_class.cu", "labs_api.cu", "noalloc.cu", "batch_kernels.cu", "batch_class.cu",
           "batch_api.cu", "serve.cu", "model.cu"]
PER_CLASS = ("walk_class.cu", "batch_class.cu")  # compiled once per lag-word class W
HEADERS = sorted(f for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))  # every header of the sources
LAG_WORD_CLASSES = range(1, 9)  # the per-class sources are compiled once per class W (m <= 32 W lags)


def _units():
    """(source, object, extra flags) of every translation unit."""
    units = []
    for src in SOURCES:
        if src in PER_CLASS:
            for w in LAG_WORD_CLASSES:
                units.append((src, src.replace(".cu", "_w%d.o" % w), ["-DPSAW_W=%d" % w]))
        else:
            units.append((src, src.replace(".cu", ".o"), []))
    return units


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "labs.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale(LIB_PATH):
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src, obj_name, extra in _units():
        obj = os.path.join(BUILD_DIR, obj_name)
        objs.append(obj)
        cmd = [nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append((obj_name, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
