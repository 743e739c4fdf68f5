"""Build liboblivgm.so in-tree with nvcc for sm_103a (no CMake, parallel TUs)."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboblivgm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["oblivgm.cu", "plain.cu", "onehot.cu", "fetch.cu", "keygen_dev.cu", "fresh.cu", "shuffle.cu", "aes_layouts.cu", "host_crypto.cpp", "serve.cpp"]
HEADERS = ["aes_bitsliced_sbox.cuh", "device_fss.cuh", "gen_device.cuh", "host_crypto.h", "ptx_async.cuh", "runtime.h"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "oblivgm.h")]
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]

    def compile_one(src: str) -> str:
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src + ".o")
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc] + common + (["-lineinfo"] if src.endswith(".cu") else []) + ["-c", path, "-o", obj + ".tmp"]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.check_call(cmd)
            os.replace(obj + ".tmp", obj)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
