"""Build libnh.so (the C-ABI library) for sm_103a with nvcc, in-tree.

    python -m paper_2204_01722_b300.build [--verbose] [--ptxas-info] [--force]

Objects go to paper_2204_01722_b300/_build/, the library to
paper_2204_01722_b300/libnh.so.  Sources are compiled in parallel; the operator
kernels are compiled once per P (nodes per direction, 2..5).
"""
import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libnh.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def units():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        if f == "nh_operator.cu":
            for p in (2, 3, 4, 5):
                out.append((f, [f"-DNH_P_INST={p}"], f"nh_operator_P{p}.o"))
        else:
            out.append((f, [], f[:-3] + ".o"))
    return out


def _compile(src, defs, obj, extra):
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, *defs, "-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return cmd, r


def build(verbose=False, ptxas_info=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "nh.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    jobs = []
    for src, defs, obj in units():
        op = os.path.join(BUILD, obj)
        if force or ptxas_info or not os.path.exists(op) or os.path.getmtime(op) < newest:
            jobs.append((src, defs, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            for cmd, r in ex.map(lambda j: _compile(*j, extra), jobs):
                if verbose or ptxas_info:
                    print(" ".join(cmd))
                    sys.stdout.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                    raise RuntimeError("nvcc failed: " + " ".join(cmd))
    objs = [os.path.join(BUILD, o) for _, _, o in units()]
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args()
    print(build(a.verbose, a.ptxas_info, a.force))
