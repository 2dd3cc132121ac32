"""Build libsipg.so in-tree for sm_103a (GB300) with nvcc.

Each translation unit compiles in its own nvcc process (in parallel); the
objects are linked into paper_1607_01323_gb300/libsipg.so.  Usable as
``python -m paper_1607_01323_gb300.build``.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libsipg.so")
BUILD = os.path.join(ROOT, "_build")
SOURCES = ["apply_f64.cu", "apply_f32.cu", "misc.cu", "cg.cu", "mg.cu", "projection.cu", "convective.cu", "stepper.cu", "general.cu", "tables.cpp", "api.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
           "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
    if src.endswith(".cu"):
        cmd += ["--expt-relaxed-constexpr"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose_ptxas=False, force=False):
    """Compile and link; returns the path of libsipg.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in os.listdir(CSRC)
                                                          if h.endswith((".h", ".cuh"))]
    srcs.append(os.path.join(INCLUDE, "sipg.h"))
    if not force and os.path.exists(OUT) and not verbose_ptxas:
        t_out = os.path.getmtime(OUT)
        if all(os.path.getmtime(s) < t_out for s in srcs):
            return OUT
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    if verbose_ptxas:
        for (obj, err), src in zip(results, SOURCES):
            if err.strip():
                sys.stderr.write("== %s\n%s" % (src, err))
    tmp = OUT + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-lcudart_static", "-ldl", "-lrt",
                                                                               "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force=True))
