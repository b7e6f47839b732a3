"""Build libatm.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel to objects under _build/ and are
linked into paper_2107_09596_gb300/libatm.so."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libatm.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "atm.h")
OBJ_DIR = os.path.join(ROOT, "_build")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
]


def sources():
    return [os.path.join(SRC_DIR, f) for f in ("atm_api.cu", "atm_noalloc.cu", "atm_nn.cu", "atm_fused.cu", "atm_df.cu")]


def _newest_input() -> float:
    files = [HEADER] + [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ_DIR, exist_ok=True)
    objs, procs = [], []
    for src in sources():
        obj = os.path.join(OBJ_DIR, os.path.basename(src) + ".%d.o" % os.getpid())
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc] + NVCC_FLAGS + ["-c", "-o", obj, src],
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    logs = []
    for p in procs:
        out, _ = p.communicate()
        logs.append(out)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + out)
    tmp = LIB + ".tmp%d" % os.getpid()
    res = subprocess.run([nvcc, "-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    for o in objs:
        os.remove(o)
    if verbose:
        print("".join(logs) + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
