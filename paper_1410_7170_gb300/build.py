"""Builds libovl.so in-tree for sm_103a (nvcc + g++, translation units in parallel).

    python -m paper_1410_7170_gb300.build [--force]
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libovl.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["dslash.cu", "blas.cu", "multishift.cu", "solver.cu", "api.cu", "sap.cu", "multirhs.cu", "deflate.cu",
              "krylov.cu", "noalloc.cu", "server.cu", "peak.cu",
              "mg.cu", "mg_ctl.cu"]
CXX_SOURCES = ["zolotarev.cpp", "eig_host.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libovl.so")


def _sources():
    cu = [s for s in CU_SOURCES if os.path.exists(os.path.join(CSRC, s))]
    cxx = [s for s in CXX_SOURCES if os.path.exists(os.path.join(CSRC, s))]
    return cu, cxx


def _stale(obj, deps, cmd=None):
    """True if obj is missing, older than a dependency, or was compiled with another command
    (the command of the last successful compile is kept beside the object)."""
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    if any(os.path.getmtime(d) > t for d in deps):
        return True
    if cmd is not None:
        try:
            with open(obj + ".cmd") as f:
                return f.read() != " ".join(cmd)
        except OSError:
            return True
    return False


def build(force=False, verbose=False):
    """Compile every translation unit and link libovl.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    cu, cxx = _sources()
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "ovl.h"))
    jobs = []
    for s in cu:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT_DIR, s + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas=-v" if verbose else "-w",
               "--expt-relaxed-constexpr", "-c", src, "-o", obj]
        jobs.append((obj, src, cmd))
    for s in cxx:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT_DIR, s + ".o")
        cmd = ["g++", "-O2", "-fcx-limited-range", "-std=c++17", "-fPIC", "-c", src, "-o", obj]
        jobs.append((obj, src, cmd))
    todo = [(o, c) for o, s, c in jobs if force or _stale(o, [s] + headers, c)]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for (obj, _), (cmd, r) in zip(todo, ex.map(lambda oc: run(oc[1]), todo)):
            if r.returncode != 0:
                raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            with open(obj + ".cmd", "w") as f:
                f.write(" ".join(cmd))
    objs = [o for o, _, _ in jobs]
    if force or todo or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
