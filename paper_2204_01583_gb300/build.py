"""Build the sm_103a shared library in-tree (nvcc, one -gencode, parallel compiles).

    python -m paper_2204_01583_gb300.build

writes ``paper_2204_01583_gb300/_lib/libov_gb300.so``.  Sources are compiled to
objects in parallel and linked once; an up-to-date library is not rebuilt.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libov_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _sources():
    return sorted(list(SRC.glob("*.cu")) + list(SRC.glob("*.cpp")))


def _deps():
    return _sources() + sorted(SRC.glob("*.h")) + sorted(SRC.glob("*.cuh")) + [ROOT / "include" / "ov.h", Path(__file__)]


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include"), "-I", str(SRC)]


def _compile(src: Path, obj: Path, verbose: bool):
    cmd = [NVCC] + ARCH + _flags() + ["-c", str(src), "-o", str(obj)]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> Path:
    if LIB.exists() and not force:
        t = LIB.stat().st_mtime
        if all(p.stat().st_mtime <= t for p in _deps()):
            return LIB
    OUT_DIR.mkdir(exist_ok=True)
    objs = []
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        futs = {}
        for src in _sources():
            obj = OUT_DIR / (src.stem + src.suffix.replace(".", "_") + ".o")
            objs.append(obj)
            futs[ex.submit(_compile, src, obj, verbose)] = src
        for f in cf.as_completed(futs):
            logs.append(f"== {futs[f].name}\n{f.result()}")
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = [NVCC] + ARCH + ["-shared", "-o", str(tmp)] + [str(o) for o in objs] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    p = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(p)
