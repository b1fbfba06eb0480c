"""ctypes declarations of the C ABI in include/holstein.h (marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

HOL_OK = 0
HOL_EINVAL = -1
HOL_ENOTCONV = -2
HOL_ENUMERIC = -3
HOL_ETIMEOUT = -4
HOL_ECUDA = -5
HOL_ENOMEM = -6

HOL_REFLECT = 0
HOL_SWAP = 1
HOL_OP_M = 0
HOL_OP_MT = 1
HOL_OP_MTM = 2

HOL_F64 = 0
HOL_F32 = 1

HOL_PINV = 0
HOL_PINVT = 1
HOL_PINV_PINVT = 2

HOL_KINETIC_CHECKERBOARD = 0
HOL_KINETIC_EXACT = 1


class hol_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("Ltau", ctypes.c_int), ("dtau", ctypes.c_double),
                ("t", ctypes.c_double), ("mu", ctypes.c_double), ("alpha", ctypes.c_double),
                ("omega0", ctypes.c_double), ("max_rhs", ctypes.c_int),
                ("kinetic", ctypes.c_int)]


class hol_cg_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precond", ctypes.c_int),
                ("prec", ctypes.c_int), ("reliable_every", ctypes.c_int),
                ("check_every", ctypes.c_int)]


class hol_md_opts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("n_steps", ctypes.c_int), ("n_sub", ctypes.c_int),
                ("m_reg", ctypes.c_double), ("cg_force", hol_cg_opts),
                ("cg_action", hol_cg_opts)]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); every entry point declared in include/holstein.h
SIGNATURES = {
    "hol_create": (_I, [ctypes.POINTER(hol_params), ctypes.POINTER(_VP)]),
    "hol_destroy": (_I, [_VP]),
    "hol_last_error": (ctypes.c_char_p, []),
    "hol_set_field": (_I, [_VP, _VP, _VP]),
    "fermion_matvec": (_I, [_VP, _I, _I, _VP, _VP, _I, _VP]),
    "cg_solve": (_I, [_VP, _VP, _VP, _I, ctypes.POINTER(hol_cg_opts),
                      ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    "cg_solve_graph": (_I, [_VP, _VP, _VP, _I, ctypes.POINTER(hol_cg_opts),
                            ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    "force": (_I, [_VP, _VP, _VP, _I, _VP, _I, _VP, _VP]),
    "precond_apply": (_I, [_VP, _I, _I, _VP, _VP, _I, _VP]),
    "mass_apply": (_I, [_VP, _I, _D, _VP, _VP, _VP]),
    "md_integrate": (_I, [_VP, _VP, _VP, _VP, _I, ctypes.POINTER(hol_md_opts), _VP]),
    "fourier_accel_leapfrog": (_I, [_VP, _VP, _VP, _VP, _I, ctypes.POINTER(hol_md_opts), _D,
                                    ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                    _VP]),
    "measure_observables": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    "global_update": (_I, [_VP, _VP, _VP, _I, _I, _I, _I, ctypes.c_double,
                           ctypes.POINTER(hol_cg_opts), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), _VP]),
    "stochastic_measure": (_I, [_VP, _VP, _I, ctypes.POINTER(hol_cg_opts), _VP, _VP, _VP, _I,
                                ctypes.POINTER(_I), _VP]),
    "pseudofermion_phi": (_I, [_VP, _VP, _VP, _I, _VP]),
    "phi_to_rhs": (_I, [_VP, _VP, _VP, _I, _VP]),
    "fermion_matvec_static": (_I, [ctypes.POINTER(hol_params), _VP, _I, _VP, _VP, _I, _VP]),
    "hmc_batch": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                       ctypes.POINTER(_VP), _I, ctypes.POINTER(hol_md_opts),
                       ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D), _I]),
    "hmc_batch_graph": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                             ctypes.POINTER(_VP), _I, ctypes.POINTER(hol_md_opts),
                             ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D), _VP]),
    "measure_batch_graph": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), _I,
                                 ctypes.POINTER(hol_cg_opts), ctypes.POINTER(_VP),
                                 ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _I, _VP]),
    "measure_batch": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), _I,
                           ctypes.POINTER(hol_cg_opts), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                           ctypes.POINTER(_VP), _I, _I]),
    "hol_set_option": (_I, [_VP, ctypes.c_char_p, _I]),
    "hol_get_option": (_I, [_VP, ctypes.c_char_p, ctypes.POINTER(_I)]),
    "hol_arnoldi_bounds": (_I, [_VP, _VP, _I, _D, _I, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                ctypes.POINTER(_I), _VP]),
    "hol_get_bounds": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP]),
    "hol_hessenberg_eigenvalues": (_I, [_I, _VP, _VP, _VP]),
    "hol_exact_taps": (_I, [_I, _D, _D, _VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hol_tune": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                      ctypes.POINTER(_D), _VP]),
    "hol_launch_count": (ctypes.c_ulonglong, []),
    "hol_fma_peak": (_I, [_I, ctypes.POINTER(_D), _VP]),
    "hol_timer_enable": (_I, [_VP, _I]),
    "hol_timer_read": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: run paper_2203_01291_gb300.build.build()"
                           " (or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
