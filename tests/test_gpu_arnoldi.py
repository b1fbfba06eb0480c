"""GPU parity of the Arnoldi spectral-bound estimate of Bbar (App. C D)
against the oracle's Arnoldi (oracle/dense.py, numpy eigenvalues of the
Hessenberg matrix), and of the preconditioner once those bounds are
installed. Marked gpu.

Tolerances: the two sides run the same FP64 recurrences with reductions in
different orders, so the Hessenberg entries agree to ~1e-14; the extreme
Ritz moduli are well separated at these sizes and agree to 1e-9 relative.
"""
import numpy as np
import pytest
import torch

import holstein_inputs as hi
from oracle import dense as D

pytestmark = pytest.mark.gpu

hg = pytest.importorskip("paper_2203_01291_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hg.build.build()
    torch.cuda.set_device(0)


DEV = "cuda"


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def _setup(L, T, kinetic="checkerboard", seed=3, nr=2):
    w = hi.Workload("a", L=L, Ltau=T, alpha=1.2, mu=0.1, omega0=1.0, x_std=1.0, seed=seed)
    x = hi.phonon_field(w)
    kin = hg.HOL_KINETIC_EXACT if kinetic == "exact" else hg.HOL_KINETIC_CHECKERBOARD
    ctx = hg.Context(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha,
                     omega0=w.omega0, max_rhs=nr, kinetic=kin)
    ctx.set_field(torch.tensor(x, device=DEV))
    return w, x, ctx, D.model_of(w, kinetic=kinetic)


@pytest.mark.parametrize("L,T,kinetic,steps", [(8, 12, "checkerboard", 20), (16, 8, "checkerboard", 20),
                                               (32, 6, "checkerboard", 24), (8, 12, "exact", 20),
                                               (6, 10, "checkerboard", 7)])
def test_arnoldi_bounds_vs_oracle(L, T, kinetic, steps):
    w, x, ctx, m = _setup(L, T, kinetic)
    v0 = hi.site_vector(w, seed=9)
    lo, hi_, runs = D.arnoldi_bounds(m, x, v0, steps=steps, margin=0.05)
    with ctx:
        got = ctx.arnoldi_bounds(torch.tensor(v0, device=DEV), steps, 0.05)
        assert got["steps"] == min(runs["B"][2], runs["Binv"][2])
        assert abs(got["bmin"] - lo) < 1e-9 * lo
        assert abs(got["bmax"] - hi_) < 1e-9 * hi_
        # not installed: the deterministic norm bounds stay in use
        dlo, dhi = D.spectral_bounds(m, x)
        glo, ghi = ctx.bounds()
        assert abs(glo - dlo) < 1e-12 * dlo and abs(ghi - dhi) < 1e-12 * dhi


def test_arnoldi_full_dimension_is_the_spectrum():
    """m = N steps span the space: the bounds are the extreme eigenvalue
    moduli of the dense Bbar (margin 0; the small end through Bbar^{-1})."""
    w, x, ctx, m = _setup(4, 10)
    ev = np.abs(np.linalg.eigvals(D.Bbar(m, x)))
    with ctx:
        got = ctx.arnoldi_bounds(torch.tensor(hi.site_vector(w, seed=2), device=DEV), m.N, 0.0)
    assert got["steps"] == m.N
    assert abs(got["bmin"] - ev.min()) < 1e-9 * ev.max()
    assert abs(got["bmax"] - ev.max()) < 1e-9 * ev.max()


@pytest.mark.parametrize("L,T", [(8, 12), (16, 20)])
def test_installed_bounds_drive_the_preconditioner(L, T):
    """After install, P^{-1} and P^{-T} are the oracle's KPM with the Arnoldi
    bounds; the next set_field restores the deterministic ones."""
    w, x, ctx, m = _setup(L, T, seed=5)
    v0 = hi.site_vector(w, seed=4)
    lo, hi_, _ = D.arnoldi_bounds(m, x, v0, steps=20, margin=0.05)
    v = hi.gaussian_vectors(w, 2, seed=6)
    with ctx:
        got = ctx.arnoldi_bounds(torch.tensor(v0, device=DEV), 20, 0.05, install=True)
        glo, ghi = ctx.bounds()
        assert glo == got["bmin"] and ghi == got["bmax"]
        for which, trans in ((hg.HOL_PINV, False), (hg.HOL_PINVT, True)):
            ref = np.stack([D.precond_inverse_apply(m, x, a, trans=trans, bounds=(lo, hi_))
                            for a in v])
            vt = torch.tensor(v, device=DEV)
            out = torch.empty_like(vt)
            ctx.precond_apply(which, vt, out)
            assert _rel(out.cpu().numpy(), ref) < 1e-10, which
        # a preconditioned solve with the installed bounds is certified
        b = torch.tensor(np.stack([D.MT_apply(m, x, r) for r in v]), device=DEV)
        sol = torch.empty_like(b)
        its, res = ctx.cg_solve(b, sol, tol=1e-10, prec=hg.HOL_F32, precond=True)
        assert max(res) < 1e-10
        ctx.set_field(torch.tensor(x, device=DEV))
        dlo, dhi = D.spectral_bounds(m, x)
        glo, ghi = ctx.bounds()
        assert abs(glo - dlo) < 1e-12 * dlo and abs(ghi - dhi) < 1e-12 * dhi


def test_arnoldi_argument_errors():
    w, x, ctx, m = _setup(8, 8)
    v0 = torch.tensor(hi.site_vector(w, seed=1), device=DEV)
    with ctx:
        for steps, margin in ((0, 0.05), (33, 0.05), (20, 1.0), (20, -0.1)):
            with pytest.raises(hg.HolError):
                ctx.arnoldi_bounds(v0, steps, margin)
