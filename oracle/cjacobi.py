"""ctypes loader for the plain-C Jacobi SVD (test infrastructure only).

``build()`` compiles ``jacobi_svd.c`` with gcc into ``oracle/_build/``;
``jacobi_svd(A)`` returns (U, s, V) for a tiny FP64 matrix of any shape.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_svd.c")
_OUT = os.path.join(_HERE, "_build", "libjacobi_svd.so")
_lib = None


def build(force=False):
    """Compile the C Jacobi SVD (gcc -O2 -fPIC -shared); returns the .so path."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", _OUT, _SRC, "-lm"])
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        _lib.jacobi_svd.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d, d,
                                    ctypes.c_double, ctypes.c_int]
        _lib.jacobi_svd.restype = ctypes.c_int
    return _lib


def jacobi_svd(A, tol=1e-15, max_sweeps=100):
    """SVD of a small matrix by one-sided Jacobi in C: A = U diag(s) V^T."""
    A = np.asarray(A, dtype=np.float64)
    trans = A.shape[0] < A.shape[1]
    if trans:
        A = A.T
    m, n = A.shape
    Af = np.asfortranarray(A)
    s = np.zeros(n)
    U = np.zeros((m, n), order="F")
    V = np.zeros((n, n), order="F")
    d = ctypes.POINTER(ctypes.c_double)
    rc = _load().jacobi_svd(m, n, Af.ctypes.data_as(d), s.ctypes.data_as(d),
                            U.ctypes.data_as(d), V.ctypes.data_as(d), tol, max_sweeps)
    if rc < 0:
        raise RuntimeError("jacobi_svd failed (%d)" % rc)
    if trans:
        U, V = V, U
    return np.ascontiguousarray(U), s, np.ascontiguousarray(V)
