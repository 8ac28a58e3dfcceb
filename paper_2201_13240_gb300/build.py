"""Build the in-tree CUDA library libwos.so (sm_103a) and its host check library.

    python -m paper_2201_13240_gb300.build

nvcc compiles the translation units in parallel (-gencode arch=compute_103a,
code=sm_103a, -O3, -lineinfo) and links a shared library next to this file.
The host check library is the same step math compiled by g++ for CPU tests.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libwos.so")
HOSTCHECK = os.path.join(HERE, "libwos_hostcheck.so")

CU_SOURCES = ["wos_capi.cu", "wos_walk_f32.cu", "wos_walk_f64.cu", "wos_nf_f32.cu", "wos_nf_f64.cu",
              "wos_adjoint.cu", "wos_render.cu", "wos_jit.cu", "wos_mesh.cpp", "wos_handles.cu", "wos_peaks.cu"]
HEADERS = ["wos_math.cuh", "wos_problem.cuh", "wos_walk_impl.cuh", "wos_nf_impl.cuh", "wos_adjoint_impl.cuh",
           "wos_internal.h", "wos_mesh.h", "wos_jit.h", "wos_capi_state.h"]
# headers of the walk kernel, embedded in the library for the runtime-compiled (problem-
# specialised) kernels
JIT_HEADERS = ["wos_internal.h", "wos_math.cuh", "wos_problem.cuh", "wos_walk_impl.cuh", "wos_adjoint_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-I", BUILD_DIR]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwos.so")
    return cand


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _write_jit_sources() -> None:
    """_build/wos_jit_sources.inc: the walk kernel's headers as C++ raw string literals."""
    delim = "WOSJIT"
    names, texts = [], []
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h), encoding="utf-8") as f:
            text = f.read()
        if ")" + delim + '"' in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        names.append(f'"{h}"')
        texts.append(f'R"{delim}({text}){delim}"')
    body = ("// generated by build.py: headers of the walk kernel for runtime compilation\n"
            f"static const int kJitHeaderCount = {len(JIT_HEADERS)};\n"
            f"static const char* const kJitHeaderNames[] = {{{', '.join(names)}}};\n"
            "static const char* const kJitHeaderTexts[] = {\n" + ",\n".join(texts) + "};\n")
    out = os.path.join(BUILD_DIR, "wos_jit_sources.inc")
    old = None
    if os.path.exists(out):
        with open(out, encoding="utf-8") as f:
            old = f.read()
    if old != body:
        with open(out, "w", encoding="utf-8") as f:
            f.write(body)


def build_lib(force: bool = False, verbose: bool = False) -> str:
    deps = [os.path.join(CSRC, s) for s in CU_SOURCES + HEADERS] + [os.path.join(INCLUDE, "wos.h")]
    if not force and not _stale(LIB, deps):
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    _write_jit_sources()
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose:
            sys.stdout.write(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s} ---\n{o}" for s, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"], check=True)
    os.replace(tmp, LIB)
    return LIB


def build_hostcheck(force: bool = False) -> str:
    src = os.path.join(CSRC, "wos_hostcheck.cpp")
    deps = [src, os.path.join(CSRC, "wos_math.cuh")]
    if not force and not _stale(HOSTCHECK, deps):
        return HOSTCHECK
    tmp = HOSTCHECK + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-Wno-unknown-pragmas", "-o", tmp, src],
                   check=True)
    os.replace(tmp, HOSTCHECK)
    return HOSTCHECK


def build(force: bool = False, verbose: bool = False) -> None:
    build_lib(force=force, verbose=verbose)
    build_hostcheck(force=force)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
