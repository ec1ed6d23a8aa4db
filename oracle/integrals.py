"""ctypes binding of the McMurchie-Davidson integral code -- TEST INFRASTRUCTURE ONLY.

Compiles ``md_integrals.c`` with gcc into ``oracle/_build/libmdint.so`` when the
library is missing or older than its source.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_integrals.c")
_LIB = os.path.join(_HERE, "_build", "libmdint.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C integrals (gcc, OpenMP) and return the .so path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            _lib.oracle_boys.restype = ctypes.c_double
            _lib.oracle_boys.argtypes = [I, ctypes.c_double]
            _lib.oracle_one_electron.argtypes = [I, I, P, P, P, P, P, P, P, I, P, P, I, I, P]
            _lib.oracle_eri3.argtypes = [I, P, P, P, P, P, P, P, I, P, P, P, P, P, P, P, I, I, P]
            _lib.oracle_eri2.argtypes = [I, P, P, P, P, P, P, P, I, I, P]
            _lib.oracle_eri4.argtypes = [I, P, P, P, P, P, P, P, P]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class CBasis:
    """Flat arrays describing a list of contracted Cartesian shells for the C code."""

    def __init__(self, l, atom, xyz, nprim, exps, coefs):
        self.l = np.ascontiguousarray(l, dtype=np.int32)
        self.atom = np.ascontiguousarray(atom, dtype=np.int32)
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.nprim = np.ascontiguousarray(nprim, dtype=np.int32)
        self.pstart = np.ascontiguousarray(np.concatenate([[0], np.cumsum(self.nprim)[:-1]]), dtype=np.int32)
        self.exps = np.ascontiguousarray(exps, dtype=np.float64)
        self.coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        self.ncart = int(sum((li + 1) * (li + 2) // 2 for li in self.l))

    def args(self):
        return [len(self.l), _ptr(self.l), _ptr(self.atom), _ptr(self.xyz), _ptr(self.nprim), _ptr(self.pstart),
                _ptr(self.exps), _ptr(self.coefs)]


def boys(n: int, T: float) -> float:
    return lib().oracle_boys(int(n), float(T))


def one_electron(kind: int, cb: CBasis, Z=None, axyz=None, datom=-1, ddim=0):
    """kind 0: S, 1: T, 2: V = sum_C -Z_C <a|1/r_C|b>; optional derivative."""
    n = cb.ncart
    out = np.zeros((n, n))
    Zc = np.ascontiguousarray(Z if Z is not None else np.zeros(0), dtype=np.int32)
    Xc = np.ascontiguousarray(axyz if axyz is not None else np.zeros((0, 3)), dtype=np.float64)
    lib().oracle_one_electron(int(kind), *cb.args(), int(len(Zc)), _ptr(Zc), _ptr(Xc), int(datom), int(ddim),
                              _ptr(out))
    return out


def eri2(ca: CBasis, datom=-1, ddim=0):
    out = np.zeros((ca.ncart, ca.ncart))
    lib().oracle_eri2(*ca.args(), int(datom), int(ddim), _ptr(out))
    return out


def eri3(cb: CBasis, ca: CBasis, datom=-1, ddim=0):
    """(mu nu|P) over Cartesian functions, shape (ncart, ncart, naux_cart)."""
    out = np.zeros((cb.ncart, cb.ncart, ca.ncart))
    lib().oracle_eri3(*cb.args(), *ca.args(), int(datom), int(ddim), _ptr(out))
    return out


def eri4(cb: CBasis):
    n = cb.ncart
    out = np.zeros((n, n, n, n))
    lib().oracle_eri4(*cb.args(), _ptr(out))
    return out
