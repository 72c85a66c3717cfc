"""Build librmp.so (the CUDA library behind include/rmp.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
import sysconfig

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librmp.so")
# CPython marshalling of the synchronous calls (csrc/rmp_pyfast.c), linked against LIB
FAST = os.path.join(PKG, "_rmp_fast" + (sysconfig.get_config_var("EXT_SUFFIX") or ".so"))
FAST_SRC = os.path.join(CSRC, "rmp_pyfast.c")
SOURCES = ["rmp_kernels.cu", "rmp_api.cu", "rmp_server.cu", "rmp_static.cu", "rmp_stream.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I" + INCLUDE, "-I" + CSRC]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "rmp.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build_fast(verbose: bool = False) -> bool:
    """Compile the CPython extension of the synchronous calls.  Optional: without it (no
    Python headers, no C compiler) the binding calls the same C functions through ctypes."""
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-I" + sysconfig.get_paths()["include"],
           "-I" + INCLUDE, FAST_SRC, "-L" + PKG, "-lrmp", "-Wl,-rpath,$ORIGIN",
           "-o", FAST + ".%d.tmp" % os.getpid()]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        sys.stderr.write("note: %s not built (the ctypes path is used):\n%s"
                         % (os.path.basename(FAST), r.stdout.decode(errors="replace")))
        return False
    os.replace(cmd[-1], FAST)
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    return True


def fast_up_to_date() -> bool:
    return os.path.exists(FAST) and os.path.getmtime(FAST) >= max(os.path.getmtime(LIB),
                                                                    os.path.getmtime(FAST_SRC))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        if not fast_up_to_date():
            build_fast(verbose)
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = ["nvcc", *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    build_fast(verbose)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
