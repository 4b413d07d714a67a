"""Build the CUDA library libspvgpu.so in-tree for sm_103a (nvcc).

An object is rebuilt when the hash of what it is made from (its source, every
header of the library, the compiler flags) differs from the hash recorded
beside it; the library is relinked when its objects' hashes differ from the
ones recorded beside it. Hashes rather than file times: a copied tree (file
times reset or preserved either way) never reuses a stale build.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libspvgpu.so")
SOURCES = ["spv_asm.cu", "spv_batch.cu", "spv_build.cu", "spv_dis.cu", "spv_info.cu", "spv_layout.cu", "spv_pipe.cu", "spv_prof.cu", "spv_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _read(path: str) -> bytes:
    with open(path, "rb") as f:
        return f.read()


def _headers() -> list:
    hs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    return hs + [os.path.join(ROOT, "include", "spv.h")]


def _source_hash(src: str, extra) -> str:
    h = hashlib.sha256()
    # the flags as written here, the include path relative to the repository
    # (a copy of the tree elsewhere keeps its hashes)
    h.update(" ".join(ARCH + FLAGS + list(extra)).replace(ROOT, "<root>").encode())
    h.update(_read(os.path.join(CSRC, src)))
    for hp in _headers():
        h.update(os.path.basename(hp).encode())
        h.update(_read(hp))
    return h.hexdigest()


def _recorded(path: str) -> str:
    try:
        with open(path + ".hash") as f:
            return f.read().strip()
    except OSError:
        return ""


def _record(path: str, digest: str) -> None:
    with open(path + ".hash", "w") as f:
        f.write(digest + "\n")


def _compile(src: str, extra, digest: str, force: bool) -> str:
    obj = os.path.join(OBJ, src.replace(".cu", ".o"))
    if not force and os.path.exists(obj) and _recorded(obj) == digest:
        return obj
    cmd = ["nvcc", *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    _record(obj, digest)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    digests = {s: _source_hash(s, extra) for s in SOURCES}
    lib_digest = hashlib.sha256("".join(digests[s] for s in SOURCES).encode()).hexdigest()
    if not force and os.path.exists(LIB) and _recorded(LIB) == lib_digest:
        return LIB
    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, digests[s], force), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run(["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    _record(LIB, lib_digest)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
