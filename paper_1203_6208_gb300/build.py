"""Build libbdgb.so in-tree with nvcc for sm_103a (GB300).

Each .cu file under csrc/ compiles to an object in _build/ (in parallel), and
the objects link into paper_1203_6208_gb300/libbdgb.so with the static CUDA
runtime.  Rebuilds only what changed.  Usage: python -m paper_1203_6208_gb300.build
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbdgb.so")
PROBE_SRC = os.path.join(HERE, "probe", "peaks.cu")
PROBE_LIB = os.path.join(HERE, "libbdpeaks.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps_mtime() -> float:
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(INCLUDE, "bd.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def _arch_stamp_ok() -> bool:
    """Objects from another host architecture (a copy made on x86 and run
    on the Arm GPU host, or the reverse) must never be linked."""
    stamp = os.path.join(OBJ, ".host_arch")
    cur = platform.machine()
    ok = os.path.exists(stamp) and open(stamp).read().strip() == cur
    if not ok:
        os.makedirs(OBJ, exist_ok=True)
        with open(stamp, "w") as f:
            f.write(cur)
    return ok


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    if not _arch_stamp_ok():
        force = True
    nvcc = _nvcc()
    hdr_t = _deps_mtime()
    procs = []
    objs = []
    for src in sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src[:-3] + ".o")
        objs.append(o)
        if (not force and os.path.exists(o) and os.path.getmtime(o) >= os.path.getmtime(s)
                and os.path.getmtime(o) >= hdr_t):
            continue
        cmd = [nvcc, *ARCH, *FLAGS, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if force or procs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    if force or not os.path.exists(PROBE_LIB) or (
            os.path.getmtime(PROBE_LIB) < os.path.getmtime(PROBE_SRC)):
        tmp = PROBE_LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc, *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", PROBE_SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, PROBE_LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
