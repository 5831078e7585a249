"""The oracle's Jacobi PCG on all host cores (oracle; test infrastructure only).

Binding of ``cpu_pcg.c``: the textbook PCG of ``pcg.py`` (Sec. 3; Saad,
Alg. 9.1) on the assembled CSR matrix, with the rows and vector updates split
over POSIX threads.  Only the tests and the benchmark's CPU baseline use it.
``build()`` compiles the C file with gcc (``__graft_entry__.build()`` calls it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_DIR, "cpu_pcg.c")
LIB = os.path.join(_DIR, "libcpupcg.so")
_lib = None


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-ffp-contract=off", "-fPIC",
                        "-shared", "-pthread", SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        lib.oracle_pcg_threads.restype = ctypes.c_int
        lib.oracle_pcg_threads.argtypes = [ctypes.c_int64, P, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P]
        _lib = lib
    return _lib


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def pcg_threads(A, b: np.ndarray, diag: np.ndarray, iters: int, nthreads: int | None = None):
    """x after exactly ``iters`` PCG iterations from x0 = 0 and the residual norms
    [||r_0||, ..., ||r_iters||]; A a scipy CSR matrix."""
    lib = _load()
    nthreads = host_threads() if nthreads is None else int(nthreads)
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int32)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    diag = np.ascontiguousarray(diag, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    hist = np.zeros(iters + 1)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    done = lib.oracle_pcg_threads(n, ptr(indptr), ptr(indices), ptr(data), ptr(diag), ptr(b), ptr(x), iters,
                                  nthreads, ptr(hist))
    if done < 0:
        raise MemoryError("oracle_pcg_threads: allocation or thread creation failed")
    if done < iters:
        raise FloatingPointError(f"CG breakdown after {done} iterations")
    return x, hist
