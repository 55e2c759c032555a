"""Random-gather probe used by bench.py beside the random planet query (a measurement aid, not part
of libshm.so or its C ABI).

``build()`` compiles gather_probe.cu for sm_103a into bench_probe/_build/libgather_probe.so (nvcc,
in-tree, rebuilt when the source changes); ``gather_probe`` runs it on torch tensors: per item q it
reads in[q] (12 B), gathers one aligned block of ``block_bytes`` from ``table`` at a hashed
position and writes out[q] (28 B), so its time is the memory system's rate for an uncorrelated
footprint read with the query's I/O and none of its arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gather_probe.cu")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgather_probe.so")
_lib = None


def build() -> str:
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
           "-fPIC", "-shared", SRC, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on gather_probe.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} not built: call bench_probe.build()")
        L = C.CDLL(LIB)
        L.gather_probe.restype = C.c_int
        L.gather_probe.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def gather_probe(table: torch.Tensor, block_bytes: int, inp: torch.Tensor, out: torch.Tensor = None, stream=None):
    """Items = rows of ``inp`` (float32 [Q][3]); ``out`` float32 [Q][7] (values meaningless)."""
    Q = inp.shape[0]
    if out is None:
        out = torch.empty((Q, 7), dtype=torch.float32, device=inp.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = _load().gather_probe(C.c_void_p(table.data_ptr()), table.numel() * table.element_size(), int(block_bytes), Q,
                              C.c_void_p(inp.data_ptr()), C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream))
    if st != 0:
        raise RuntimeError(f"gather_probe failed (status {st})")
    return out
