"""In-tree build of the native libraries.

* ``libgtadoc.so``  - the CUDA engine behind the ``gt_*`` C ABI (sm_103a only).
* ``corpus/libgtcorpus.so`` - the host-side Sequitur compressor that prepares
  inputs.

Both are compiled next to their sources with plain ``nvcc`` / ``g++`` calls so
that the same commands work on x86 and on an Arm (Grace) host.  A library is
rebuilt only when one of its sources is newer than the ``.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = ROOT / "_build"

GTADOC_SO = PKG / "libgtadoc.so"
CORPUS_SO = PKG / "corpus" / "libgtcorpus.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fvisibility=hidden"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(cand).exists():
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libgtadoc.so")
    return cand


def _stale(target: Path, sources) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(s).stat().st_mtime > t for s in sources)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(map(str, cmd)) + "\n" + r.stdout)
    return r.stdout


_corpus_lock = threading.Lock()


def build_corpus(force: bool = False) -> Path:
    """Build the Sequitur library; threads of one process build it once (the
    lock), processes each write their own temporary file."""
    src = PKG / "corpus" / "sequitur.cpp"
    with _corpus_lock:
        if force or _stale(CORPUS_SO, [src]):
            tmp = CORPUS_SO.with_suffix(f".so.tmp{os.getpid()}_{threading.get_ident()}")
            _run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", str(src), "-o", str(tmp)])
            os.replace(tmp, CORPUS_SO)
    return CORPUS_SO


def gtadoc_sources():
    return sorted(CSRC.glob("*.cu"))


def build_gtadoc(force: bool = False, verbose_ptxas: bool = False) -> Path:
    srcs = gtadoc_sources()
    headers = sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))
    if not (force or _stale(GTADOC_SO, srcs + headers)):
        return GTADOC_SO
    BUILD.mkdir(exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def compile_one(src: Path):
        obj = BUILD / (src.stem + ".o")
        out = _run([nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", str(INCLUDE), "-I", str(CSRC),
                    "-c", str(src), "-o", str(obj)])
        return obj, out

    with ThreadPoolExecutor(max_workers=min(8, len(srcs) or 1)) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    tmp = GTADOC_SO.with_suffix(f".so.tmp{os.getpid()}")
    _run([nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"])
    os.replace(tmp, GTADOC_SO)
    if verbose_ptxas:
        return GTADOC_SO, "\n".join(o for _, o in results)
    return GTADOC_SO


def build_all(force: bool = False) -> None:
    build_corpus(force)
    build_gtadoc(force)
