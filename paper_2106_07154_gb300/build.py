"""Compiles liblts.so in-tree for sm_103a (nvcc for the CUDA kernels, g++ for
the host runtime), in parallel, without cmake.

Usage: ``python -m paper_2106_07154_gb300.build [--force]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG / "_build"
LIB = PKG / "liblts.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> Path:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and (Path(cand) / "bin" / "nvcc").exists():
            return Path(cand)
    nvcc = shutil.which("nvcc")
    if nvcc:
        return Path(nvcc).resolve().parent.parent
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    return sorted(CSRC.glob("*.cpp")) + sorted(CSRC.glob("*.cu"))


def _headers():
    return sorted(CSRC.glob("*.h")) + sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def _compile_cmd(src: Path, obj: Path, cuda: Path):
    if src.suffix == ".cu":
        return [str(cuda / "bin" / "nvcc"), *ARCH, "-lineinfo", "-O3", "-std=c++17",
                "-Xcompiler", "-fPIC", "-Xptxas", "-v", f"-I{INCLUDE}", f"-I{CSRC}",
                "-c", str(src), "-o", str(obj)]
    return ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-Wall", "-Wno-unused-function",
            f"-I{INCLUDE}", f"-I{CSRC}", f"-I{cuda / 'include'}", "-c", str(src), "-o", str(obj)]


def build(force: bool = False, verbose: bool = False) -> Path:
    cuda = cuda_home()
    BUILD.mkdir(exist_ok=True)
    srcs = _sources()
    newest_header = max((h.stat().st_mtime for h in _headers()), default=0.0)
    jobs = []
    for src in srcs:
        obj = BUILD / (src.name + ".o")
        stale = (force or not obj.exists() or obj.stat().st_mtime < src.stat().st_mtime
                 or obj.stat().st_mtime < newest_header)
        if stale:
            jobs.append((src, obj, _compile_cmd(src, obj, cuda)))

    def run(job):
        src, obj, cmd = job
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        log = BUILD / (src.name + ".log")
        log.write_text(res.stdout + res.stderr)
        return src

    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        for src in ex.map(run, jobs):
            if verbose:
                print("compiled", src.name)
    objs = [BUILD / (s.name + ".o") for s in srcs]
    if force or jobs or not LIB.exists():
        tmp = LIB.with_suffix(".so.tmp")
        cmd = ["g++", "-shared", "-fopenmp", "-o", str(tmp), *map(str, objs),
               f"-L{cuda / 'lib64'}", "-lcudart", f"-Wl,-rpath,{cuda / 'lib64'}"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
