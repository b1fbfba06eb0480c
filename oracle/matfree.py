"""ctypes front end of the matrix-free C oracle (oracle/matfree.c) -- TEST
INFRASTRUCTURE ONLY. ``build()`` compiles it with gcc (-O2 -fopenmp) into
oracle/_build/libholstein_oracle.so; nothing here touches the CUDA library."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "matfree.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libholstein_oracle.so")


class _Model(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("T", ctypes.c_int), ("dtau", ctypes.c_double),
                ("t", ctypes.c_double), ("mu", ctypes.c_double),
                ("alpha", ctypes.c_double), ("omega0", ctypes.c_double),
                ("kinetic", ctypes.c_int)]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               SRC, "-o", LIB, "-lm"])
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        mp = ctypes.POINTER(_Model)
        _lib.orc_M.argtypes = [mp, dp, dp, dp]
        _lib.orc_MT.argtypes = [mp, dp, dp, dp]
        _lib.orc_expV.argtypes = [mp, dp, dp]
        _lib.orc_kinetic.argtypes = [mp, dp, ctypes.c_int]
        _lib.orc_cg.argtypes = [mp, dp, dp, dp, ctypes.c_double, ctypes.c_int, dp]
        _lib.orc_cg.restype = ctypes.c_int
        _lib.orc_force_fermion.argtypes = [mp, dp, dp, dp, dp]
        _lib.orc_force_boson.argtypes = [mp, dp, dp]
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _m(model) -> _Model:
    """A workload or a dense-oracle Model (its `kinetic`, "checkerboard" by
    default, selects the propagator)."""
    exact = getattr(model, "kinetic", "checkerboard") == "exact"
    return _Model(model.L, model.Ltau, model.dtau, model.t, model.mu, model.alpha, model.omega0,
                  1 if exact else 0)


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def expV(model, x):
    x = _c(x)
    out = np.empty_like(x)
    lib().orc_expV(ctypes.byref(_m(model)), _p(x), _p(out))
    return out


def M_apply(model, x, v):
    d = expV(model, x)
    v = _c(v)
    out = np.empty_like(v)
    lib().orc_M(ctypes.byref(_m(model)), _p(d), _p(v), _p(out))
    return out


def MT_apply(model, x, v):
    d = expV(model, x)
    v = _c(v)
    out = np.empty_like(v)
    lib().orc_MT(ctypes.byref(_m(model)), _p(d), _p(v), _p(out))
    return out


def MTM_apply(model, x, v):
    return MT_apply(model, x, M_apply(model, x, v))


def cg(model, x, b, tol=1e-13, max_iter=20000):
    """Returns (v, iterations or -1, true relative residual)."""
    x, b = _c(x), _c(b)
    v = np.empty_like(b)
    res = ctypes.c_double(0.0)
    it = lib().orc_cg(ctypes.byref(_m(model)), _p(x), _p(b), _p(v), tol, max_iter,
                      ctypes.byref(res))
    return v, it, res.value


def rel_residual(model, x, b, v) -> float:
    r = _c(b) - MTM_apply(model, x, v)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def force_fermion(model, x, v, b):
    x, v, b = _c(x), _c(v), _c(b)
    F = np.zeros_like(x)
    lib().orc_force_fermion(ctypes.byref(_m(model)), _p(x), _p(v), _p(b), _p(F))
    return F


def force_boson(model, x):
    x = _c(x)
    F = np.zeros_like(x)
    lib().orc_force_boson(ctypes.byref(_m(model)), _p(x), _p(F))
    return F
