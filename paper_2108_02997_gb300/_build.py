"""Build steps for the native parts of the package (no cmake, no setuptools).

* ``libprgraphgen.so`` — the seeded graph generators (plain C, gcc).
* ``libpagerank.so``  — the C-ABI PageRank library (CUDA, nvcc, sm_103a only).
* ``libprceiling.so`` — the gather-rate probes bench.py reports beside its
  roofline (CUDA; measurement only, not part of the library).

Each library is rebuilt when a source file is newer than it, or when the
extra compiler definitions in the environment variable PR_NVCC_FLAGS (tuning
constants such as -DPR_HUB_BYTES=...) differ from the last build's. The CUDA
translation units compile in parallel to keep the build within a minute.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
ROOT = PKG.parent
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"

GRAPHGEN_SO = PKG / "libprgraphgen.so"
PAGERANK_SO = PKG / "libpagerank.so"
CEILING_SO = PKG / "libprceiling.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]

CU_SOURCES = ["pr_api.cu", "pr_graph.cu", "pr_solve.cu", "pr_learn.cu", "pr_noalloc.cu", "pr_plan.cu"]
CU_HEADERS = ["pr_internal.cuh", "pr_host.h", "pr_kernels.cuh", "df64.cuh"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpagerank.so")


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).exists() and Path(d).stat().st_mtime > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(map(str, cmd)) + "\n" + r.stdout + r.stderr)
    return r


def build_graphgen(force: bool = False) -> Path:
    src = CSRC / "graphgen.c"
    if force or _stale(GRAPHGEN_SO, [src]):
        tmp = GRAPHGEN_SO.with_suffix(".so.tmp")
        _run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", str(tmp), str(src), "-lm"])
        os.replace(tmp, GRAPHGEN_SO)
    return GRAPHGEN_SO


def build_pagerank(force: bool = False, verbose_ptxas: bool = False) -> Path:
    srcs = [CSRC / s for s in CU_SOURCES]
    hdrs = [CSRC / h for h in CU_HEADERS] + sorted(INCLUDE.glob("*.h"))
    extra = os.environ.get("PR_NVCC_FLAGS", "").split()
    stamp = BUILD / "flags.txt"
    flags_changed = (stamp.read_text() if stamp.exists() else "") != " ".join(extra)
    if flags_changed:
        force = True
    if not (force or _stale(PAGERANK_SO, srcs + hdrs + [Path(__file__)])):
        return PAGERANK_SO
    nvcc = _nvcc()
    BUILD.mkdir(exist_ok=True)
    flags = ARCH + NVCC_FLAGS + extra + ["-I", str(INCLUDE), "-I", str(CSRC)]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]

    def compile_one(src: Path) -> Path:
        obj = BUILD / (src.stem + ".o")
        if force or _stale(obj, [src] + hdrs + [Path(__file__)]):
            r = _run([nvcc, *flags, "-c", str(src), "-o", str(obj)])
            if verbose_ptxas:
                (BUILD / (src.stem + ".ptxas.txt")).write_text(r.stdout + r.stderr)
        return obj

    with _cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = PAGERANK_SO.with_suffix(".so.tmp")
    _run([nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart", "-lcuda"])
    os.replace(tmp, PAGERANK_SO)
    stamp.write_text(" ".join(extra))
    return PAGERANK_SO


def build_ceiling(force: bool = False) -> Path:
    src = CSRC / "gather_ceiling.cu"
    if force or _stale(CEILING_SO, [src, Path(__file__)]):
        tmp = CEILING_SO.with_suffix(".so.tmp")
        _run([_nvcc(), *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", str(tmp), str(src),
              "-lcudart"])
        os.replace(tmp, CEILING_SO)
    return CEILING_SO


def build_all(force: bool = False) -> None:
    build_graphgen(force)
    with _cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build_pagerank, force), ex.submit(build_ceiling, force)]
        for f in futs:
            f.result()
