"""Build and load the oracle's plain C parts -- TEST AND CPU-BASELINE
INFRASTRUCTURE ONLY.

``memcpy_threads.c`` is the all-cores CPU memcpy baseline (see its header).
It is compiled with the host C compiler into ``oracle/_build`` (git-ignored)
on the machine that runs it; nothing here touches the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "memcpy_threads.c")
LIB = os.path.join(OUT, "libmemcpy_threads.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([cc, "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", SRC, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.mt_memcpy_epochs.restype = ctypes.c_int
        lib.mt_memcpy_epochs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_void_p]
        _lib = lib
    return _lib


class ThreadedMemcpy:
    """Holds the pointer table, the op table and the epoch boundaries of one
    workload over numpy slot buffers, and applies all epochs per call."""

    def __init__(self, slot_arrays, ops: np.ndarray, epochs):
        self.lib = load()
        self.slot_arrays = slot_arrays
        self.ptrs = np.array([a.ctypes.data for a in slot_arrays], dtype=np.uint64)
        self.ops = np.ascontiguousarray(ops)
        assert self.ops.dtype.itemsize == 32
        self.bounds = np.array([a for a, _ in epochs] + [epochs[-1][1]], dtype=np.uint64)
        assert all(b == a2 for (_, b), (a2, _) in zip(epochs[:-1], epochs[1:])), "epochs must be contiguous"
        self.scratch = np.zeros(max(b - a for a, b in epochs) + 1, dtype=np.uint64)

    def run(self, threads: int) -> int:
        return self.lib.mt_memcpy_epochs(self.ptrs.ctypes.data, self.ops.ctypes.data, self.bounds.ctypes.data,
                                         len(self.bounds) - 1, threads, self.scratch.ctypes.data)
