"""GB300 (sm_103a) library for the hot path of hybrid Monte Carlo for the
Holstein model (Cohen-Stead et al., arXiv:2203.01291).

Every computation runs in the CUDA library built from csrc/ and exposed
through the C ABI of include/holstein.h; this module only marshals
arguments (torch tensors -> device pointers, current CUDA stream). There is
no CPU fallback: without the built library, or without a GPU, the calls
raise.

    ctx = Context(L=32, Ltau=200, dtau=0.1, t=1.0, mu=0.0, alpha=1.0,
                  omega0=0.5, max_rhs=16)
    ctx.set_field(x)                                  # x: cuda float64 [T, N]
    ctx.fermion_matvec(HOL_OP_MTM, v, out)           # v, out: [n_rhs, T, N]
    iters, resid = ctx.cg_solve(b, v, tol=1e-8, prec=HOL_F32)
    ctx.force(v, b, dSdx, with_bosonic=True)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._abi import (HOL_ECUDA, HOL_EINVAL, HOL_ENOMEM, HOL_ENOTCONV, HOL_ENUMERIC, HOL_ETIMEOUT,
                   HOL_F32, HOL_F64, HOL_KINETIC_CHECKERBOARD, HOL_KINETIC_EXACT, HOL_OK,
                   HOL_OP_M, HOL_OP_MT, HOL_OP_MTM, HOL_PINV,
                   HOL_PINV_PINVT, HOL_PINVT, HOL_REFLECT, HOL_SWAP, hol_cg_opts, hol_md_opts,
                   hol_params, load, library_path)

__all__ = ["Context", "HolError", "HOL_OP_M", "HOL_OP_MT", "HOL_OP_MTM", "HOL_F64", "HOL_F32",
           "hol_create", "hol_destroy", "hol_set_field", "fermion_matvec", "cg_solve", "force",
           "precond_apply", "HOL_PINV", "HOL_PINVT", "HOL_PINV_PINVT",
           "pseudofermion_phi", "phi_to_rhs", "hol_launch_count", "hol_timer_enable",
           "hol_timer_read", "fermion_matvec_static", "mass_apply", "md_integrate",
           "fourier_accel_leapfrog", "hol_md_opts", "stochastic_measure", "hol_tune",
           "hmc_batch", "hmc_batch_graph", "cg_solve_graph", "measure_batch",
           "measure_batch_graph", "hol_set_option", "hol_get_option", "hol_fma_peak",
           "global_update", "HOL_REFLECT", "HOL_SWAP", "measure_observables",
           "HOL_KINETIC_CHECKERBOARD", "HOL_KINETIC_EXACT", "hol_arnoldi_bounds",
           "hol_get_bounds",
           "library_path", "load"]


class HolError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _check(rc: int) -> None:
    if rc != HOL_OK:
        raise HolError(rc, load().hol_last_error().decode(errors="replace"))


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: torch.Tensor, dtype: torch.dtype, numel: int | None = None, name: str = "tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- ABI mirrors
def hol_create(params: hol_params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().hol_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def hol_destroy(handle) -> None:
    _check(load().hol_destroy(handle))


def hol_set_field(handle, x: torch.Tensor, n: int) -> None:
    _check(load().hol_set_field(handle, _ptr(x, torch.float64, n, "x"), _stream()))


def fermion_matvec(handle, op: int, prec: int, v: torch.Tensor, out: torch.Tensor, n_rhs: int,
                   n: int) -> None:
    dt = torch.float64 if prec == HOL_F64 else torch.float32
    _check(load().fermion_matvec(handle, op, prec, _ptr(v, dt, n_rhs * n, "v"),
                                 _ptr(out, dt, n_rhs * n, "out"), n_rhs, _stream()))


def cg_solve(handle, b: torch.Tensor, v: torch.Tensor, n_rhs: int, n: int, opts: hol_cg_opts,
             raise_on_nonconv: bool = True):
    it = (ctypes.c_int * n_rhs)()
    rs = (ctypes.c_double * n_rhs)()
    rc = load().cg_solve(handle, _ptr(b, torch.float64, n_rhs * n, "b"),
                         _ptr(v, torch.float64, n_rhs * n, "v"), n_rhs, ctypes.byref(opts), it,
                         rs, _stream())
    if rc != HOL_OK and (rc != HOL_ENOTCONV or raise_on_nonconv):
        _check(rc)
    return np.array(it[:], dtype=np.int64), np.array(rs[:], dtype=np.float64)


def cg_solve_graph(handle, b: torch.Tensor, v: torch.Tensor, n_rhs: int, n: int,
                   opts: hol_cg_opts, raise_on_nonconv: bool = True):
    """cg_solve as one CUDA graph launch (include/holstein.h, cg_solve_graph)."""
    it = (ctypes.c_int * n_rhs)()
    rs = (ctypes.c_double * n_rhs)()
    rc = load().cg_solve_graph(handle, _ptr(b, torch.float64, n_rhs * n, "b"),
                               _ptr(v, torch.float64, n_rhs * n, "v"), n_rhs, ctypes.byref(opts),
                               it, rs, _stream())
    if rc != HOL_OK and (rc != HOL_ENOTCONV or raise_on_nonconv):
        _check(rc)
    return np.array(it[:], dtype=np.int64), np.array(rs[:], dtype=np.float64)


def force(handle, v: torch.Tensor, b: torch.Tensor, n_pf: int, dSdx: torch.Tensor | None,
          with_bosonic: bool, S_F: torch.Tensor | None, n: int) -> None:
    """Phonon force into dSdx and/or the action into S_F (dSdx None: action only)."""
    sf = _ptr(S_F, torch.float64, 1, "S_F") if S_F is not None else None
    f = _ptr(dSdx, torch.float64, n, "dSdx") if dSdx is not None else None
    _check(load().force(handle, _ptr(v, torch.float64, n_pf * n, "v"),
                        _ptr(b, torch.float64, n_pf * n, "b"), n_pf, f,
                        int(bool(with_bosonic)), sf, _stream()))


def precond_apply(handle, which: int, prec: int, v: torch.Tensor, out: torch.Tensor, n_rhs: int,
                  n: int) -> None:
    dt = torch.float64 if prec == HOL_F64 else torch.float32
    _check(load().precond_apply(handle, which, prec, _ptr(v, dt, n_rhs * n, "v"),
                                _ptr(out, dt, n_rhs * n, "out"), n_rhs, _stream()))


def pseudofermion_phi(handle, R: torch.Tensor, Phi: torch.Tensor, n_pf: int, n: int) -> None:
    _check(load().pseudofermion_phi(handle, _ptr(R, torch.float64, n_pf * n, "R"),
                                    _ptr(Phi, torch.float64, n_pf * n, "Phi"), n_pf, _stream()))


def phi_to_rhs(handle, Phi: torch.Tensor, b: torch.Tensor, n_pf: int, n: int) -> None:
    _check(load().phi_to_rhs(handle, _ptr(Phi, torch.float64, n_pf * n, "Phi"),
                             _ptr(b, torch.float64, n_pf * n, "b"), n_pf, _stream()))


def fermion_matvec_static(params: hol_params, x: torch.Tensor, op: int, v: torch.Tensor,
                          out: torch.Tensor, n_rhs: int) -> None:
    """Context-free FP64 operator whose scratch is a fixed device array (no
    allocation); see include/holstein.h."""
    n = params.L * params.L * params.Ltau
    _check(load().fermion_matvec_static(ctypes.byref(params), _ptr(x, torch.float64, n, "x"), op,
                                        _ptr(v, torch.float64, n_rhs * n, "v"),
                                        _ptr(out, torch.float64, n_rhs * n, "out"), n_rhs,
                                        _stream()))


def mass_apply(handle, which: int, m_reg: float, p: torch.Tensor, out: torch.Tensor,
               n: int) -> None:
    _check(load().mass_apply(handle, which, float(m_reg), _ptr(p, torch.float64, n, "p"),
                             _ptr(out, torch.float64, n, "out"), _stream()))


def md_integrate(handle, x: torch.Tensor, p: torch.Tensor, Phi: torch.Tensor, n_pf: int,
                 opts: hol_md_opts, n: int) -> None:
    _check(load().md_integrate(handle, _ptr(x, torch.float64, n, "x"),
                               _ptr(p, torch.float64, n, "p"),
                               _ptr(Phi, torch.float64, n_pf * n, "Phi"), n_pf,
                               ctypes.byref(opts), _stream()))


def fourier_accel_leapfrog(handle, x: torch.Tensor, R_pf: torch.Tensor, R_p: torch.Tensor,
                           n_pf: int, opts: hol_md_opts, u: float, n: int):
    acc = ctypes.c_int()
    dH = ctypes.c_double()
    terms = (ctypes.c_double * 6)()
    _check(load().fourier_accel_leapfrog(handle, _ptr(x, torch.float64, n, "x"),
                                         _ptr(R_pf, torch.float64, n_pf * n, "R_pf"),
                                         _ptr(R_p, torch.float64, n, "R_p"), n_pf,
                                         ctypes.byref(opts), float(u), ctypes.byref(acc),
                                         ctypes.byref(dH), terms, _stream()))
    return bool(acc.value), dH.value, np.array(terms[:])


def md_opts(dt: float, n_steps: int, n_sub: int, m_reg: float, force_tol: float = 1e-5,
            action_tol: float = 1e-10, prec: int = HOL_F32, precond: bool = False,
            reliable_every: int = 50, check_every: int = 10) -> hol_md_opts:
    """hol_md_opts with the paper's solver tolerances (Sec. VI B) as defaults."""
    f = hol_cg_opts(force_tol, 100000, int(precond), prec, reliable_every, check_every)
    a = hol_cg_opts(action_tol, 100000, int(precond), prec, reliable_every, check_every)
    return hol_md_opts(dt, n_steps, n_sub, float(m_reg), f, a)


def stochastic_measure(handle, xi: torch.Tensor, n_rv: int, opts: hol_cg_opts, Gxi: torch.Tensor,
                       G2: torch.Tensor, G4: torch.Tensor | None, four_point: int, n: int):
    it = (ctypes.c_int * n_rv)()
    g4 = _ptr(G4, torch.float64, 6 * n, "G4") if G4 is not None else None
    _check(load().stochastic_measure(handle, _ptr(xi, torch.float64, n_rv * n, "xi"), n_rv,
                                     ctypes.byref(opts), _ptr(Gxi, torch.float64, n_rv * n, "Gxi"),
                                     _ptr(G2, torch.float64, 2 * n, "G2"), g4, int(four_point), it,
                                     _stream()))
    return np.array(it[:], dtype=np.int64)


def global_update(handle, x: torch.Tensor, Phi: torch.Tensor, n_pf: int, kind: int, i: int,
                  j: int, u: float, opts: hol_cg_opts, S_cur: float | None, n: int):
    """Reflection / swap move (include/holstein.h); returns (accepted, dS, S)."""
    S = ctypes.c_double(float("nan") if S_cur is None else float(S_cur))
    acc = ctypes.c_int(0)
    d = ctypes.c_double(0.0)
    _check(load().global_update(handle, _ptr(x, torch.float64, n, "x"),
                                _ptr(Phi, torch.float64, n_pf * n, "Phi"), n_pf, int(kind),
                                int(i), int(j), float(u), ctypes.byref(opts), ctypes.byref(S),
                                ctypes.byref(acc), ctypes.byref(d), _stream()))
    return bool(acc.value), d.value, S.value


def measure_observables(handle, G2: torch.Tensor, G4: torch.Tensor, C: torch.Tensor, L: int,
                        T: int) -> dict:
    """density, S_cdw, P_s (host) and C(r) (device) from a measurement."""
    out = (ctypes.c_double * 3)()
    _check(load().measure_observables(handle, _ptr(G2, torch.float64, 2 * T * L * L, "G2"),
                                      _ptr(G4, torch.float64, 6 * T * L * L, "G4"),
                                      _ptr(C, torch.float64, L * L, "C"), out, _stream()))
    return {"density": out[0], "S_cdw": out[1], "P_s": out[2]}


def hol_tune(handle, n_rhs: int) -> dict:
    k, w, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(load().hol_tune(handle, n_rhs, ctypes.byref(k), ctypes.byref(w), ctypes.byref(v),
                           ctypes.byref(ms), _stream()))
    return {"slices_per_group": k.value, "warps_per_block": w.value, "float4_layout": v.value,
            "ms": ms.value}


def hol_arnoldi_bounds(handle, v0: torch.Tensor, N: int, m: int = 20, margin: float = 0.05,
                       install: bool = False) -> dict:
    lo, hi, st = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().hol_arnoldi_bounds(handle, _ptr(v0, torch.float64, N, "v0"), m, margin,
                                     int(bool(install)), ctypes.byref(lo), ctypes.byref(hi),
                                     ctypes.byref(st), _stream()))
    return {"bmin": lo.value, "bmax": hi.value, "steps": st.value}


def hol_get_bounds(handle) -> tuple:
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(load().hol_get_bounds(handle, ctypes.byref(lo), ctypes.byref(hi), _stream()))
    return lo.value, hi.value


def _ptrs(ts, dtype=torch.float64):
    arr = (ctypes.c_void_p * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = _ptr(t, dtype, None, f"tensor {k}").value
    return arr


def hmc_batch(contexts, xs, R_pfs, R_ps, opts: hol_md_opts, us, n_threads: int = 8):
    """Algorithm 1 once for every chain (own context, own stream), run
    concurrently; returns (accepted[n], dH[n])."""
    n = len(contexts)
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in contexts])
    n_pf = R_pfs[0].numel() // contexts[0].n
    acc = (ctypes.c_int * n)()
    dh = (ctypes.c_double * n)()
    u = (ctypes.c_double * n)(*[float(v) for v in us])
    torch.cuda.current_stream().synchronize()   # inputs were written on torch's stream
    _check(load().hmc_batch(hs, n, _ptrs(xs), _ptrs(R_pfs), _ptrs(R_ps), n_pf,
                            ctypes.byref(opts), u, acc, dh, int(n_threads)))
    return np.array(acc[:], dtype=bool), np.array(dh[:])


def hmc_batch_graph(contexts, xs, R_pfs, R_ps, opts: hol_md_opts, us):
    """Algorithm 1 once for every chain, all chains in one captured CUDA graph
    per leapfrog step (include/holstein.h, hmc_batch_graph); returns
    (accepted[n], dH[n])."""
    n = len(contexts)
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in contexts])
    n_pf = R_pfs[0].numel() // contexts[0].n
    acc = (ctypes.c_int * n)()
    dh = (ctypes.c_double * n)()
    u = (ctypes.c_double * n)(*[float(v) for v in us])
    _check(load().hmc_batch_graph(hs, n, _ptrs(xs), _ptrs(R_pfs), _ptrs(R_ps), n_pf,
                                  ctypes.byref(opts), u, acc, dh, _stream()))
    return np.array(acc[:], dtype=bool), np.array(dh[:])


def measure_batch_graph(contexts, xis, Gxis, G2s, opts: hol_cg_opts, G4s=None,
                        four_point: int = 0, concurrency: int = 0) -> None:
    """stochastic_measure for every chain, all chains in one captured CUDA
    graph, at most `concurrency` chains in flight (0: all; include/holstein.h,
    measure_batch_graph)."""
    n = len(contexts)
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in contexts])
    n_rv = xis[0].numel() // contexts[0].n
    g4 = _ptrs(G4s) if G4s is not None else None
    _check(load().measure_batch_graph(hs, n, _ptrs(xis), n_rv, ctypes.byref(opts), _ptrs(Gxis),
                                      _ptrs(G2s), g4, int(four_point), int(concurrency),
                                      _stream()))


def measure_batch(contexts, xis, Gxis, G2s, opts: hol_cg_opts, G4s=None, four_point: int = 0,
                  n_threads: int = 8) -> None:
    n = len(contexts)
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in contexts])
    n_rv = xis[0].numel() // contexts[0].n
    g4 = _ptrs(G4s) if G4s is not None else None
    torch.cuda.current_stream().synchronize()
    _check(load().measure_batch(hs, n, _ptrs(xis), n_rv, ctypes.byref(opts), _ptrs(Gxis),
                                _ptrs(G2s), g4, int(four_point), int(n_threads)))


def hol_set_option(handle, name: str, value: int) -> None:
    _check(load().hol_set_option(handle, name.encode(), int(value)))


def hol_get_option(handle, name: str) -> int:
    out = ctypes.c_int(0)
    _check(load().hol_get_option(handle, name.encode(), ctypes.byref(out)))
    return int(out.value)


def hol_fma_peak(prec: int) -> float:
    """Measured FMA throughput (GFLOP/s) of the current GPU."""
    g = ctypes.c_double()
    _check(load().hol_fma_peak(int(prec), ctypes.byref(g), _stream()))
    return g.value


def hol_launch_count() -> int:
    return int(load().hol_launch_count())


def hol_timer_enable(handle, stride: int) -> None:
    """stride k >= 1: time one in every k kernel regions per class; 0: off."""
    _check(load().hol_timer_enable(handle, int(stride)))


def hol_timer_read(handle, klass: int):
    """(recorded regions, their summed device ms, their summed work units)"""
    cnt = ctypes.c_int()
    ms = ctypes.c_double()
    un = ctypes.c_double()
    _check(load().hol_timer_read(handle, klass, ctypes.byref(cnt), ctypes.byref(ms),
                                 ctypes.byref(un)))
    return cnt.value, ms.value, un.value


TIMER_OPERATOR, TIMER_UPDATE, TIMER_FORCE, TIMER_PRECOND, TIMER_OTHER = range(5)


# ---------------------------------------------------------------- convenience
class Context:
    """One lattice shape and set of couplings (owns the library context)."""

    def __init__(self, L: int, Ltau: int, dtau: float = 0.1, t: float = 1.0, mu: float = 0.0,
                 alpha: float = 1.0, omega0: float = 1.0, max_rhs: int = 1,
                 kinetic: int = HOL_KINETIC_CHECKERBOARD):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2203_01291_gb300 needs a CUDA GPU; there is no CPU fallback")
        self.L, self.Ltau, self.N = L, Ltau, L * L
        self.n = self.N * Ltau
        self.max_rhs = max_rhs
        self.kinetic = kinetic
        self.params = hol_params(L, Ltau, dtau, t, mu, alpha, omega0, max_rhs, kinetic)
        self._h = hol_create(self.params)

    @classmethod
    def from_workload(cls, w, max_rhs: int | None = None) -> "Context":
        return cls(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha,
                   omega0=w.omega0, max_rhs=max_rhs or max(1, w.n_rhs))

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            hol_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _nrhs(self, v: torch.Tensor) -> int:
        if v.numel() % self.n:
            raise ValueError("vector length is not a multiple of N*Ltau")
        return v.numel() // self.n

    def set_field(self, x: torch.Tensor) -> None:
        hol_set_field(self._h, x, self.n)

    def fermion_matvec(self, op: int, v: torch.Tensor, out: torch.Tensor) -> None:
        prec = HOL_F64 if v.dtype == torch.float64 else HOL_F32
        fermion_matvec(self._h, op, prec, v, out, self._nrhs(v), self.n)

    def cg_solve(self, b: torch.Tensor, v: torch.Tensor, tol: float = 1e-10,
                 max_iter: int = 10000, precond: bool = False, prec: int = HOL_F64,
                 reliable_every: int = 50, check_every: int = 10,
                 raise_on_nonconv: bool = True):
        opts = hol_cg_opts(tol, max_iter, int(bool(precond)), prec, reliable_every, check_every)
        return cg_solve(self._h, b, v, self._nrhs(b), self.n, opts, raise_on_nonconv)

    def cg_solve_graph(self, b: torch.Tensor, v: torch.Tensor, tol: float = 1e-10,
                       max_iter: int = 10000, precond: bool = False, prec: int = HOL_F64,
                       reliable_every: int = 50, check_every: int = 10,
                       raise_on_nonconv: bool = True):
        """The solve of cg_solve as one graph launch (device-side control)."""
        opts = hol_cg_opts(tol, max_iter, int(bool(precond)), prec, reliable_every, check_every)
        return cg_solve_graph(self._h, b, v, self._nrhs(b), self.n, opts, raise_on_nonconv)

    def force(self, v: torch.Tensor, b: torch.Tensor, dSdx: torch.Tensor | None,
              with_bosonic: bool = True, S_F: torch.Tensor | None = None) -> None:
        force(self._h, v, b, self._nrhs(v), dSdx, with_bosonic, S_F, self.n)

    def precond_apply(self, which: int, v: torch.Tensor, out: torch.Tensor) -> None:
        prec = HOL_F64 if v.dtype == torch.float64 else HOL_F32
        precond_apply(self._h, which, prec, v, out, self._nrhs(v), self.n)

    def pseudofermion_phi(self, R: torch.Tensor, Phi: torch.Tensor) -> None:
        pseudofermion_phi(self._h, R, Phi, self._nrhs(R), self.n)

    def phi_to_rhs(self, Phi: torch.Tensor, b: torch.Tensor) -> None:
        phi_to_rhs(self._h, Phi, b, self._nrhs(Phi), self.n)

    def mass_apply(self, which: int, m_reg: float, p: torch.Tensor, out: torch.Tensor) -> None:
        mass_apply(self._h, which, m_reg, p, out, self.n)

    def md_integrate(self, x: torch.Tensor, p: torch.Tensor, Phi: torch.Tensor,
                     opts: hol_md_opts) -> None:
        md_integrate(self._h, x, p, Phi, self._nrhs(Phi), opts, self.n)

    def fourier_accel_leapfrog(self, x: torch.Tensor, R_pf: torch.Tensor, R_p: torch.Tensor,
                               opts: hol_md_opts, u: float):
        """Algorithm 1; returns (accepted, dH, [S_B, S_F, K] at start and end)."""
        return fourier_accel_leapfrog(self._h, x, R_pf, R_p, self._nrhs(R_pf), opts, u, self.n)

    def measure_observables(self, G2: torch.Tensor, G4: torch.Tensor, C: torch.Tensor) -> dict:
        """<n>, S_cdw, P_s of one measurement (stochastic_measure with
        four_point = 7); C(r) is written to C ([L][L], device)."""
        return measure_observables(self._h, G2, G4, C, self.L, self.Ltau)

    def global_update(self, x: torch.Tensor, Phi: torch.Tensor, kind: int, i: int, j: int = -1,
                      u: float = 0.5, tol: float = 1e-10, prec: int = HOL_F64,
                      S_cur: float | None = None, max_iter: int = 100000):
        """Reflection (kind HOL_REFLECT, site i) or swap (HOL_SWAP, sites i, j)
        Metropolis move at fixed Phi; x is updated in place. Returns
        (accepted, dS, S of the kept field)."""
        opts = hol_cg_opts(tol, max_iter, 0, prec, 50, 10)
        return global_update(self._h, x, Phi, self._nrhs(Phi), kind, i, j, u, opts, S_cur,
                             self.n)

    def stochastic_measure(self, xi: torch.Tensor, Gxi: torch.Tensor, G2: torch.Tensor,
                           G4: torch.Tensor | None = None, four_point: int = 0,
                           tol: float = 1e-10, prec: int = HOL_F64, precond: bool = False,
                           max_iter: int = 100000):
        opts = hol_cg_opts(tol, max_iter, int(bool(precond)), prec, 50, 10)
        return stochastic_measure(self._h, xi, self._nrhs(xi), opts, Gxi, G2, G4, four_point,
                                  self.n)

    def set_option(self, name: str, value: int) -> None:
        """Launch option (see include/holstein.h, hol_set_option)."""
        hol_set_option(self._h, name, value)

    def get_option(self, name: str) -> int:
        """Current value of a launch option (hol_get_option)."""
        return hol_get_option(self._h, name)

    def arnoldi_bounds(self, v0: torch.Tensor, m: int = 20, margin: float = 0.05,
                       install: bool = False) -> dict:
        """Spectral bounds of Bbar by m Arnoldi steps from v0 (hol_arnoldi_bounds);
        install=True makes the preconditioner use them until the next set_field."""
        return hol_arnoldi_bounds(self._h, v0, self.N, m, margin, install)

    def bounds(self) -> tuple:
        """(bmin, bmax) the preconditioner currently uses (hol_get_bounds)."""
        return hol_get_bounds(self._h)

    def tune(self, n_rhs: int) -> dict:
        """Pick the fastest launch shape of the fused M^T M for n_rhs (needs a field)."""
        return hol_tune(self._h, n_rhs)

    def timer_enable(self, stride: int = 1) -> None:
        hol_timer_enable(self._h, int(stride))

    def timer_read(self, klass: int):
        return hol_timer_read(self._h, klass)
