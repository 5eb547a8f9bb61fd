"""Build the CUDA library libhvx.so in-tree with nvcc for sm_103a.

Every translation unit under csrc/ is compiled in parallel into _build/, then
linked into paper_2008_11476_gb300/libhvx.so (CUDA runtime linked statically).
A build is skipped when the library is newer than every source file.

The headers that kernels generated at run time include (csrc/codegen.cpp
compiles them with NVRTC) are embedded into the library as string constants:
_build/jit_headers.inc is written from them before compiling.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhvx.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE,
          "-I", BUILD]

# (C++ identifier, header under csrc/) embedded for the run-time compiler
JIT_HEADERS = [("kJitPointMath", "point_math.cuh"), ("kJitPhaseTable", "phase_table.h"),
               ("kJitParams", "jit_params.h"), ("kJitReduceMath", "reduce_math.cuh")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhvx.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    deps += glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(f) > t for f in deps)


def write_jit_headers() -> None:
    parts = ["// Written by _build.py: headers of the kernels generated at run time.\n"]
    for name, fn in JIT_HEADERS:
        with open(os.path.join(CSRC, fn)) as f:
            text = f.read()
        if ")HVXJIT\"" in text:
            raise RuntimeError(f"{fn} contains the raw-string delimiter")
        parts.append(f'static const char {name}[] = R"HVXJIT({text})HVXJIT";\n')
    out = os.path.join(BUILD, "jit_headers.inc")
    tmp = out + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write("".join(parts))
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    write_jit_headers()
    cc = nvcc()
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [cc, *ARCH, *COMMON, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
