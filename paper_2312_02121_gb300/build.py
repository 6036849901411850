"""Builds the CUDA library ``libgsplat103.so`` in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and the
objects are linked into ``paper_2312_02121_gb300/libgsplat103.so`` (git-ignored).
A rebuild happens only when a source or ``include/gsplat103.h`` is newer than
the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libgsplat103.so")
SOURCES = ["gs_abi.cu", "gs_autotune.cu", "gs_project.cu", "gs_sort.cu", "gs_sort_static.cu", "gs_raster.cu",
           "gs_raster_bwd2.cu",
           "gs_raster_nc.cu", "gs_train.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgsplat103.so")


def _inputs():
    deps = [os.path.join(CSRC, s) for s in SOURCES]
    deps += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    deps.append(os.path.join(INCLUDE, "gsplat103.h"))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(d) <= t for d in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library; returns its path."""
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(OBJ_DIR, exist_ok=True)
    cc = nvcc()
    tag = f"{os.getpid()}"

    def compile_one(src: str) -> str:
        obj = os.path.join(OBJ_DIR, src.replace(".cu", f".{tag}.o"))
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".{tag}.tmp"
    r = subprocess.run([cc, *ARCH, "-shared", *objs, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH


def resources() -> list:
    """Per kernel, what ptxas reports when compiling every source for sm_103a:
    (translation unit, demangled kernel, registers, spill store bytes, spill
    load bytes, static shared memory bytes).  Nothing is linked or written."""
    import re
    cc = nvcc()
    rows = []

    def one(src: str):
        cmd = [cc, *ARCH, *FLAGS, "-Xptxas=-v", "-c", os.path.join(CSRC, src), "-o", os.devnull]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return src, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        outs = list(ex.map(one, SOURCES))
    for src, text in outs:
        cur = None
        for ln in text.splitlines():
            m = re.search(r"Compiling entry function '([^']+)'", ln)
            if m:
                cur = dict(tu=src, name=m.group(1), regs=0, spill_st=0, spill_ld=0, smem=0)
                rows.append(cur)
                continue
            if cur is None:
                continue
            m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", ln)
            if m:
                cur["spill_st"], cur["spill_ld"] = int(m.group(1)), int(m.group(2))
            m = re.search(r"Used (\d+) registers", ln)
            if m:
                cur["regs"] = int(m.group(1))
                m2 = re.search(r"(\d+) bytes smem", ln)
                cur["smem"] = int(m2.group(1)) if m2 else 0
    filt = shutil.which("c++filt")
    if filt and rows:
        names = subprocess.run([filt], input="\n".join(r["name"] for r in rows), capture_output=True,
                               text=True).stdout.splitlines()
        if len(names) == len(rows):
            for r, n in zip(rows, names):
                r["name"] = n
    return rows


if __name__ == "__main__":  # pragma: no cover
    import sys
    if "--resources" in sys.argv:
        print("| source | kernel | registers | spill st / ld (B) | static smem (B) |")
        print("|---|---|---|---|---|")
        for r in resources():
            name = r["name"].split("(")[0].replace("void ", "")  # the kernel and its template arguments
            print(f"| {r['tu']} | `{name}` | {r['regs']} | {r['spill_st']} / {r['spill_ld']} | {r['smem']} |")
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
