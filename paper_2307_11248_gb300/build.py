"""Build the CUDA library ``libqap.so`` in-tree for sm_103a with nvcc.

The translation units compile in parallel; the library is rebuilt only when
a source, header or flag changed (a content hash is stored beside it).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libqap.so")

UNITS = ["qap_api.cu", "qap_walk_i32_f8.cu", "qap_walk_i32_f8m.cu", "qap_walk_i32_f16.cu",
         "qap_walk_i64_f16.cu", "qap_batch_i32_f8.cu", "qap_batch_i32_f8m.cu",
         "qap_batch_i32_f16.cu", "qap_batch_i64_f16.cu", "qap_walk_i64_f64.cu",
         "qap_walk_i64_f64p.cu", "qap_batch_i64_f64.cu", "qap_batch_i64_f64p.cu", "qap_server.cu",
         "qap_walk_i32_f16m.cu", "qap_walk_i64_f16m.cu", "qap_batch_i32_f16m.cu",
         "qap_batch_i64_f16m.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-pthread", "-I", INCLUDE]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _digest():
    h = hashlib.sha256()
    h.update(" ".join(ARCH + FLAGS).encode())
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h", ".py")) and name != "__init__.py":
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode())
                    h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile ``libqap.so`` if it is missing or stale; return its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libqap.sha256")
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    objs = [os.path.join(BUILD, u.replace(".cu", ".o")) for u in UNITS]

    def compile_one(unit, obj):
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{res.stdout}\n{res.stderr}")
        return res.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        logs = list(ex.map(compile_one, UNITS, objs))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs],
                   check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    if verbose:
        for log in logs:
            print(log)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
