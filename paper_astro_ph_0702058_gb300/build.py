"""Builds libnbody.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel into ``_build/`` and linked into
``paper_astro_ph_0702058_gb300/libnbody.so`` (CUDA runtime linked statically,
so the library does not depend on the PyTorch wheel's CUDA runtime).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libnbody.so")
SOURCES = ["api.cu", "force.cu", "force_plain.cu", "force_comp.cu", "force_check.cu", "force_sorted.cu", "force_ds.cu", "energy_ds.cu", "integrator.cu", "cluster_step.cu", "grid_step.cu", "noalloc.cu", "ensemble.cu", "adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Per-source nvcc flags (none at present).
SOURCE_FLAGS: dict[str, list[str]] = {}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out: str | None = None, build_dir: str | None = None) -> str:
    """Compiles the library if a source changed (or ``force``); returns its path.

    ``extra`` adds nvcc flags (e.g. -D tuning macros); ``out`` and ``build_dir``
    place a variant build elsewhere than the default library.
    """
    lib = out or LIB
    bdir = build_dir or BUILD
    if not force and out is None and up_to_date():
        return LIB
    os.makedirs(bdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                    "--expt-relaxed-constexpr"] + (extra or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags + SOURCE_FLAGS.get(src, [])
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"nvcc failed on {src}")
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))


def build_probe(out: str | None = None) -> str:
    """Compiles the standalone pipe-throughput probe (csrc/pipe_probe.cu); returns its path."""
    exe = out or os.path.join(BUILD, "pipe_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    cmd = [nvcc(), os.path.join(CSRC, "pipe_probe.cu"), "-o", exe, "-O3", "-std=c++17"] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed on pipe_probe.cu")
    return exe
