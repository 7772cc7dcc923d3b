"""Build liblbm.so in-tree from csrc/ with nvcc for sm_103a.

Translation units compile in parallel; the result is
``paper_1412_5170_gb300/liblbm.so`` (git-ignored).  Run as
``python -m paper_1412_5170_gb300.build`` or via ``__graft_entry__.build()``.
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["lbm_api.cu", "lbm_observe.cu", "lbm_strip.cu", "lbm_strip_f32.cu", "lbm_pipe_f32.cu", "lbm_strip_f64.cu", "lbm_noalloc.cu", "lbm_batch.cu", "lbm_batch_strip.cu", "lbm_mlp.cu", "lbm_peak.cu", "lbm_host.cpp"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def flags(verbose_ptxas: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(objs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(INCLUDE, s) for s in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale(None):
        return LIB
    with tempfile.TemporaryDirectory(prefix="lbm_build_") as tmp:
        procs, objs = [], []
        for s in SOURCES:
            o = os.path.join(tmp, s + ".o")
            objs.append(o)
            cmd = [nvcc()] + flags(verbose) + ["-c", os.path.join(CSRC, s), "-o", o]
            procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        failed = False
        for s, p in procs:
            out, _ = p.communicate()
            if out and (verbose or p.returncode):
                sys.stderr.write("== %s\n%s" % (s, out))
            failed |= p.returncode != 0
        if failed:
            raise RuntimeError("liblbm build failed")
        tmp_lib = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp_lib] + objs)
        os.replace(tmp_lib, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
