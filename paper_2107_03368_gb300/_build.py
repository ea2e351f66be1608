"""In-tree build of the package's native libraries.

``libsynth.so`` (host C, the input generator) is built with gcc and
``libdt.so`` (the CUDA search library behind ``include/dt.h``) with nvcc for
sm_103a only.  Both land next to this file and are rebuilt when a source is
newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

SYNTH_SO = os.path.join(HERE, "libsynth.so")
DT_SO = os.path.join(HERE, "libdt.so")
OBJ_DIR = os.path.join(HERE, "_build")

CUDA_SOURCES = [
    "api.cu",
    "autotune.cu",
    "bf_popc.cu",
    "bf_tc.cu",
    "dt_build.cu",
    "dt_insert.cu",
    "index_io.cu",
    "quicci.cu",
    "dt_search.cu",
    "encoder.cu",
    "enc_tc.cu",
    "ivf.cu",
    "objects.cu",
    "votes.cu",
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r


def build_synth(force=False):
    src = os.path.join(CSRC, "synth.c")
    if force or _stale(SYNTH_SO, [src]):
        tmp = SYNTH_SO + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
              "-o", tmp, src, "-lm"])
        os.replace(tmp, SYNTH_SO)
    return SYNTH_SO


def build_dt(force=False, verbose_ptxas=False):
    srcs = [os.path.join(CSRC, s) for s in CUDA_SOURCES]
    deps = srcs + _headers()
    if not (force or _stale(DT_SO, deps)):
        return DT_SO
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I" + INCLUDE, "-I" + CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]

    def compile_one(s):
        obj = os.path.join(OBJ_DIR, os.path.basename(s) + ".o")
        _run([nvcc] + flags + ["-c", s, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = DT_SO + ".tmp%d" % os.getpid()
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, DT_SO)
    return DT_SO


def build_all(force=False):
    build_synth(force)
    build_dt(force)
