"""Builds the in-tree CUDA library ``_build/libdsp.so`` for sm_103a.

The translation units (the FP32-mixed evolve kernel on contiguous tiles; the
row-strip kernel, compiled once per scheme and strip height; the other kernels;
the host API; the allocation-free density) are compiled in parallel with nvcc,
then linked into one shared library with the CUDA runtime linked statically.  Host code is compiled without floating-point
contraction, so the host-side arithmetic (pulse tables, projection nodes) rounds
the same way on every host architecture.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdsp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdsp.so")


def sources() -> list[str]:
    return [os.path.join(CSRC, f) for f in ("dsp_mixed.cu", "dsp_strip.cu", "dsp_kernels.cu",
                                            "dsp_api.cpp", "dsp_noalloc.cu")]


# dsp_strip.cu is compiled once per scheme (EXACT, STRANG_XY, MAGNUS4) and strip height
# (2 packs per thread: 4-row strips; 1: 2-row strips): (object suffix, defines).
STRIP_VARIANTS = [(f"_s{s}_np{n}", [f"-DDSP_STRIP_SCHEME={s}", f"-DDSP_STRIP_NP={n}"])
                  for s in (0, 1, 2) for n in (2, 1)]


def units() -> list[tuple[str, str, list[str]]]:
    """(source, object base name, extra defines) of every translation unit."""
    out = []
    for src in sources():
        base = os.path.basename(src)
        if base == "dsp_strip.cu":
            out += [(src, base + suffix, defs) for suffix, defs in STRIP_VARIANTS]
        else:
            out.append((src, base, []))
    return out


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + [os.path.join(CSRC, h) for h in ("dsp_internal.h", "dsp_df.cuh",
                                                        "dsp_device.cuh")] + [
                        os.path.join(INCLUDE, "dsp.h"),
                        os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


BOUNDS_LIB = os.path.join(BUILD, "bounds_check", "libdsp.so")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          bounds_check: bool = False) -> str:
    """Compile and link libdsp.so if any source is newer than it; returns its path.

    bounds_check=True builds the variant with -DDSP_BOUNDS_CHECK (device index
    checks that flag DSP_E_BOUNDS instead of accessing) into _build/bounds_check/."""
    lib = BOUNDS_LIB if bounds_check else LIB
    if not force and not _stale(lib):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    nvcc = _nvcc()
    objs, procs = [], []
    for src, name, defs in units():
        obj = os.path.join(os.path.dirname(lib), name + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + COMMON + defs + (["-DDSP_BOUNDS_CHECK"] if bounds_check else [])
        cmd += ["-Xcompiler", "-ffp-contract=off"]
        if src.endswith(".cu"):
            cmd += ARCH + ["-lineinfo"]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0 or ptxas_info:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed = True
            sys.stderr.write("failed: " + " ".join(cmd) + "\n")
    if failed:
        raise RuntimeError("building libdsp.so failed")
    tmp = lib + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    subprocess.run(link, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
