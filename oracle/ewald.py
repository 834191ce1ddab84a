"""Plain FP64 Ewald oracle for periodic Laplace lattice sums (test infrastructure).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module.  The product library never does, and this
module imports nothing from the product package.

It computes the definition of the paper's Eq. (1.1) with the Green's function of
Eq. (1.2) (3D ``1/(4 pi r)``, 2D ``-log(r)/(2 pi)``), the self term excluded, under the
tin-foil convention of Sec. 1 (the k = 0 Fourier mode is zero), by classical Ewald
summation in ``ewald_oracle.c``.  For non-neutral charges the result is the zero-mean
periodic potential (uniform neutralising background).  Ewald's splitting parameter
``alpha`` only moves work between the two sums; the result is independent of it to
the truncation tolerance, which the tests check.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald_oracle.c")
_LIB = os.path.join(_HERE, "libewald_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C code (gcc, -O2, OpenMP) next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(ctypes.c_double)
        PI = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_ewald.argtypes = [ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_int64, P, PI,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P,
                                     ctypes.c_int]
        lib.oracle_ewald.restype = ctypes.c_int
        lib.oracle_ewald_bloch.argtypes = [ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_int64, P, PI, P,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P, P,
                                           ctypes.c_int]
        lib.oracle_ewald_bloch.restype = ctypes.c_int
        lib.oracle_e1.argtypes = [ctypes.c_double]
        lib.oracle_e1.restype = ctypes.c_double
        _lib = lib
    return _lib


def e1(x: float) -> float:
    """The oracle's own exponential integral E1 (used by the 2D short-range kernel)."""
    return _load().oracle_e1(float(x))


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_alpha(d: int, V: float, n: int, m: int) -> float:
    """Balance real-space pair work (~ m n / alpha^d) against mode work (~ (n+m) alpha^d)."""
    n = max(n, 1)
    m = max(m, 1)
    ratio = 4.0  # cost of one real-space pair relative to one mode term
    X = math.sqrt(2.0 * m * n * ratio * math.pi ** d / (V * V * (n + m)))
    return X ** (1.0 / d)


def ewald(L, y, q, x=None, self_idx=None, *, tol: float = 1e-15, alpha: float | None = None,
          grad: bool = True, nthreads: int | None = None):
    """Periodic potential (and gradient) at targets ``x``.

    L: (d, d) lattice matrix, column j = lattice vector a_j.
    y: (n, d) source positions; q: (n,) charges.
    x: (m, d) targets, or None for "at the sources" (self pairs excluded by index).
    self_idx: (m,) index of the source coinciding with each target, or -1 (only used
        when x is given).
    Returns (pot (m,), grad (m, d) or None).
    """
    L = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
    d = L.shape[0]
    assert L.shape == (d, d) and d in (2, 3)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(-1, d))
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
    n = y.shape[0]
    assert q.shape[0] == n
    if x is None:
        x = y
        sidx = np.arange(n, dtype=np.int64)
    else:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, d))
        sidx = (np.full(x.shape[0], -1, dtype=np.int64) if self_idx is None
                else np.ascontiguousarray(np.asarray(self_idx, dtype=np.int64)))
    m = x.shape[0]
    V = abs(np.linalg.det(L))
    if alpha is None:
        alpha = default_alpha(d, V, n, m)
    s = math.sqrt(-math.log(tol))
    rcut = s / alpha
    kcut = 2.0 * alpha * s
    Lc = np.ascontiguousarray(L.T)  # column-major storage of L
    pot = np.zeros(m, dtype=np.float64)
    g = np.zeros((m, d), dtype=np.float64) if grad else None
    rc = _load().oracle_ewald(
        d, _ptr(Lc), n, _ptr(y), _ptr(q), m, _ptr(x),
        sidx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(alpha), rcut, kcut,
        _ptr(pot), _ptr(g) if grad else ctypes.POINTER(ctypes.c_double)(),
        int(nthreads or 0))
    if rc != 0:
        raise RuntimeError(f"oracle_ewald failed ({rc})")
    return pot, g


def ewald_bloch(L, y, q, beta, x=None, self_idx=None, *, tol: float = 1e-15, alpha: float | None = None,
                nthreads: int | None = None):
    """Quasi-periodic (Bloch) potential and gradient at targets ``x``:
    Phi(x) = sum_n sum_j' q_j e^{i beta.L n} G(x - y_j - L n), so that
    Phi(x + L n) = e^{i beta.L n} Phi(x) (paper Sec. 3.7).  No neutrality is needed; beta
    must not be a reciprocal-lattice vector.  Direct loops: for small N.
    Returns (pot (m,) complex, grad (m, d) complex)."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
    d = L.shape[0]
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(-1, d))
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
    beta = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(d))
    n = y.shape[0]
    if x is None:
        x = y
        sidx = np.arange(n, dtype=np.int64)
    else:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, d))
        sidx = (np.full(x.shape[0], -1, dtype=np.int64) if self_idx is None
                else np.ascontiguousarray(np.asarray(self_idx, dtype=np.int64)))
    m = x.shape[0]
    V = abs(np.linalg.det(L))
    if alpha is None:
        alpha = default_alpha(d, V, n, m)
    s = math.sqrt(-math.log(tol))
    rcut = s / alpha
    kcut = 2.0 * alpha * s
    Lc = np.ascontiguousarray(L.T)
    pr, pi = np.zeros(m), np.zeros(m)
    gr, gi = np.zeros((m, d)), np.zeros((m, d))
    rc = _load().oracle_ewald_bloch(
        d, _ptr(Lc), n, _ptr(y), _ptr(q), m, _ptr(x),
        sidx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(beta), float(alpha), rcut, kcut,
        _ptr(pr), _ptr(pi), _ptr(gr), _ptr(gi), int(nthreads or 0))
    if rc == -2:
        raise ValueError("beta is a reciprocal-lattice vector (the periodic case)")
    if rc != 0:
        raise RuntimeError(f"oracle_ewald_bloch failed ({rc})")
    return pr + 1j * pi, gr + 1j * gi


def nthreads_default() -> int:
    return os.cpu_count() or 1
