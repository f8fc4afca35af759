"""Plain sum-factorised FP64 tangent application on the host cores (oracle; test
infrastructure and the timed CPU baseline only).

ctypes binding of oracle/sumfact.c (Algorithm 1 element by element, with sum factorisation,
Section 2.4; OpenMP over the elements of each of the eight colour classes).  It computes the
operator of `oracle.fem.Operator.apply` (homogeneous material) and is pinned to it by
tests/test_oracle_sumfact.py; its purpose is to be timed beside the GPU library.  The shared
library is compiled with gcc on first use (or by the repository's build step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .tables import element_tables

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sumfact.c")
LIB = os.path.join(HERE, "liboracle_sumfact.so")

_lib = None


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.sf_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               dp, dp, dp, dp, dp, dp, dp]
        L.sf_apply.restype = ctypes.c_int
        L.sf_cache.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.sf_cache.restype = ctypes.c_int
        L.sf_threads.argtypes = []
        L.sf_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """Host threads the OpenMP loops use (OMP_NUM_THREADS, else one per core)."""
    return int(lib().sf_threads())


class SumFactOperator:
    """A(u) du on N^3 Q_p elements of the unit cube with Lame parameters (mu, lam) and
    boundary preset bc (0 none, 1 clamp x = 0, 2 compression), FP64."""

    def __init__(self, n_el: int, degree: int, mu: float, lam: float, bc: int = 0):
        self.N, self.p, self.mu, self.lam, self.bc = n_el, degree, float(mu), float(lam), bc
        _, _, w, B, D = element_tables(degree)
        self.B = np.ascontiguousarray(B, dtype=np.float64)
        self.D = np.ascontiguousarray(D, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.n_dofs = 3 * (degree * n_el + 1) ** 3
        self.cache = None

    def set_cache(self, u):
        """Point table of the cached strategy at u: F^-1 and ln J per Gauss point."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        self.cache = np.empty(self.N ** 3 * (self.p + 1) ** 3 * 10)
        if lib().sf_cache(self.N, self.p, _p(self.B), _p(self.D), _p(u), _p(self.cache)) != 0:
            raise ValueError("det F <= 0 at a Gauss point")

    def apply(self, u, du, cached: bool = False, out=None):
        du = np.ascontiguousarray(du, dtype=np.float64)
        v = np.empty(self.n_dofs) if out is None else out
        if cached and self.cache is None:
            raise ValueError("set_cache first")
        uu = None if cached else np.ascontiguousarray(u, dtype=np.float64)
        rc = lib().sf_apply(self.N, self.p, self.mu, self.lam, self.bc, _p(self.B), _p(self.D), _p(self.w),
                            _p(uu), _p(du), _p(self.cache if cached else None), _p(v))
        if rc != 0:
            raise ValueError("det F <= 0 at a Gauss point" if rc == 1 else "bad arguments")
        return v
