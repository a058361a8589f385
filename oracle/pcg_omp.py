"""ctypes wrapper of ``pcg_omp.c``: the oracle's Jacobi-PCG on all host cores (oracle).

TEST INFRASTRUCTURE ONLY (the "fair CPU" timing of the benchmark and its test).  The C file
is compiled with gcc and OpenMP into ``oracle/_build/liboracle_pcg.so`` by ``compile()``
(which ``__graft_entry__.build()`` runs with the same command).
"""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcg_omp.c")
LIB = os.path.join(HERE, "_build", "liboracle_pcg.so")
CMD = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB, "-lm"]


def compile(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    subprocess.run(CMD, check=True, capture_output=True, text=True)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(compile())
        f = lib.oracle_pcg_csr
        f.restype = C.c_int
        f.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                      C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int)]
        _lib = lib
    return _lib


def pcg(K, b, rtol=1e-8, maxit=200000, x0=None):
    """Solve K x = b (K SPD, scipy CSR) by Jacobi-PCG on the host cores.

    Returns (x, iterations, relative residual ||b - K x|| / ||b|| of the recurrence, threads)."""
    K = K.tocsr()
    ip = np.ascontiguousarray(K.indptr, dtype=np.int64)
    ix = np.ascontiguousarray(K.indices, dtype=np.int32)
    a = np.ascontiguousarray(K.data, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(bb) if x0 is None else np.array(x0, dtype=np.float64)
    it, rr, nt = C.c_int(0), C.c_double(0), C.c_int(0)
    st = _load().oracle_pcg_csr(K.shape[0], ip.ctypes.data, ix.ctypes.data, a.ctypes.data, bb.ctypes.data,
                                x.ctypes.data, rtol, maxit, C.byref(it), C.byref(rr), C.byref(nt))
    if st < 0:
        raise RuntimeError("oracle_pcg_csr: bad argument or out of memory")
    return x, it.value, rr.value, nt.value
