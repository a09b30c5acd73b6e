"""FP64 CPU oracle for grids too large to assemble (Sec. 2.1.1, Eq. (2)).

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU-baseline leg,
never by the library.

The assembled K of oracle.fem is applied without forming it, by the plain C
element loop of oracle/fullsize.c (compiled here with gcc, OpenMP over the
host's cores):

  apply(grid, E, k0, u)          K(E) u over all DOFs (no boundary condition)
  residual(grid, E, k0, f, fixed, u)   f - K u on the free DOFs and its norm
  element_energies(grid, k0, u)  u_e^T k0 u_e for every element
  cg(grid, E, k0, f, fixed, rtol)      Jacobi-preconditioned CG on K_ff, FP64,
                                 to a true relative residual rtol (or the
                                 attainable FP64 floor)

k0 (Sec. 2.1.2) and E (Eq. (1)) come from oracle.fem, whose assembled K the
tests compare this with on small grids.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fullsize.c")
LIB = os.path.join(HERE, "_fullsize.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/fullsize.c into oracle/_fullsize.so (gcc, OpenMP when the
    compiler has it)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: the same loops, one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("gcc failed on oracle/fullsize.c:\n" + r.stdout + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        i, d, p, lg = C.c_int, C.c_double, C.c_void_p, C.c_long
        L.oracle_apply.argtypes = [i, i, i, p, p, p, p]
        L.oracle_apply.restype = None
        L.oracle_residual.argtypes = [i, i, i, p, p, p, p, p, p]
        L.oracle_residual.restype = d
        L.oracle_element_energies.argtypes = [i, i, i, p, p, p]
        L.oracle_element_energies.restype = None
        L.oracle_cg.argtypes = [i, i, i, p, p, p, p, d, lg, p, C.POINTER(d)]
        L.oracle_cg.restype = lg
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(grid):
    return int(grid.nx), int(grid.ny), int(grid.nz)


def _check(grid, E=None, u=None):
    if E is not None and E.size != grid.n_elem:
        raise ValueError("E must hold one value per element")
    if u is not None and u.size != grid.n_dof:
        raise ValueError("vectors must hold one value per DOF")


def apply(grid, E, k0, u) -> np.ndarray:
    """K(E) u over all DOFs, no boundary condition (the assembled fem.assemble
    matrix times u)."""
    E, k0, u = _f64(E), _f64(k0), _f64(u)
    _check(grid, E, u)
    y = np.empty(grid.n_dof)
    lib().oracle_apply(*_dims(grid), E.ctypes.data, k0.ctypes.data, u.ctypes.data, y.ctypes.data)
    return y


def residual(grid, E, k0, f, fixed, u):
    """(r, ||r||_2) with r = f - K u on free DOFs and 0 on fixed ones."""
    E, k0, f, u = _f64(E), _f64(k0), _f64(f), _f64(u)
    _check(grid, E, u)
    fx = np.ascontiguousarray(fixed, dtype=np.uint8)
    r = np.empty(grid.n_dof)
    nr = lib().oracle_residual(*_dims(grid), E.ctypes.data, k0.ctypes.data, f.ctypes.data,
                               fx.ctypes.data, u.ctypes.data, r.ctypes.data)
    return r, float(nr)


def rel_residual(grid, E, k0, f, fixed, u) -> float:
    """||f - K u||_2 / ||f||_2 over the free DOFs, every DOF included."""
    f = _f64(f)
    return residual(grid, E, k0, f, fixed, u)[1] / float(np.linalg.norm(f[~np.asarray(fixed)]))


def element_energies(grid, k0, u) -> np.ndarray:
    """u_e^T k0 u_e for every element."""
    k0, u = _f64(k0), _f64(u)
    _check(grid, None, u)
    w = np.empty(grid.n_elem)
    lib().oracle_element_energies(*_dims(grid), k0.ctypes.data, u.ctypes.data, w.ctypes.data)
    return w


def cg(grid, E, k0, f, fixed, rtol: float = 1e-12, maxiter: int = 1_000_000):
    """Jacobi-PCG in FP64 on K_ff u_f = f_f from u = 0.  Returns
    (u, iterations, final true relative residual); the residual may stay
    above rtol where FP64 cannot go lower."""
    E, k0, f = _f64(E), _f64(k0), _f64(f)
    _check(grid, E, f)
    fx = np.ascontiguousarray(fixed, dtype=np.uint8)
    f = f.copy()
    f[fx.astype(bool)] = 0.0
    x = np.zeros(grid.n_dof)
    rel = C.c_double(0.0)
    it = lib().oracle_cg(*_dims(grid), E.ctypes.data, k0.ctypes.data, f.ctypes.data,
                         fx.ctypes.data, float(rtol), int(maxiter), x.ctypes.data, C.byref(rel))
    return x, int(it), float(rel.value)
