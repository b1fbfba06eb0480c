"""GPU parity of the Fourier-accelerated split leapfrog (Sec. III B,
Algorithm 1) against the dense oracle, plus reversibility and the dt^2
energy error at the hmc16 workload (L=16, Ltau=160). Marked gpu.

Tolerances: the mass operator (FFT along tau, FP64) to 1e-12 of max|ref|;
trajectories with FP64 solves at tol 1e-13 to 1e-8 relative (a few dozen
force evaluations, each carrying the solve error kappa * tol ~ 1e-10).
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


@pytest.mark.parametrize("L,T", [(4, 40), (6, 12), (8, 30), (4, 14)])
@pytest.mark.parametrize("m_reg", [1.0, 0.3, float("inf")])
def test_mass_operators_vs_dense(L, T, m_reg):
    w = hi.Workload("m", L=L, Ltau=T, omega0=0.7)
    m = D.model_of(w)
    p = hi.gaussian_vectors(w, 1, seed=3)[0]
    with hg.Context.from_workload(w) as ctx:
        pt = torch.tensor(p, device=DEV)
        out = torch.empty_like(pt)
        for which, power in ((0, -1.0), (1, 0.5), (2, 1.0)):
            ctx.mass_apply(which, m_reg, pt, out)
            ref = D.mass_apply(m, p, m_reg, power)
            assert _rel(out.cpu().numpy(), ref) < 1e-12, (which, m_reg)


def _tight(prec=hg.HOL_F64, precond=False, tol=1e-13):
    return hg.md_opts(0.0, 0, 1, 1.0, force_tol=tol, action_tol=tol, prec=prec,
                      precond=precond, check_every=1)


@pytest.mark.parametrize("precond", [False, True])
def test_md_integrate_vs_oracle_tiny(precond):
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x0 = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=2)
    Phi = D.phi_from_R(m, x0, R)
    p0 = D.mass_apply(m, hi.gaussian_vectors(w, 1, seed=5)[0], 1.0, 0.5)
    dt, Nt, nt, mreg = 0.05, 3, 2, 1.0
    xr, pr = D.leapfrog_split(m, x0, p0, Phi, dt, Nt, nt, mreg)
    o = _tight(precond=precond)
    o.dt, o.n_steps, o.n_sub, o.m_reg = dt, Nt, nt, mreg
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        x = torch.tensor(x0, device=DEV)
        p = torch.tensor(p0, device=DEV)
        ctx.md_integrate(x, p, torch.tensor(Phi, device=DEV), o)
        assert _rel(x.cpu().numpy(), xr) < 1e-8
        assert _rel(p.cpu().numpy(), pr) < 1e-8


def test_hmc_update_vs_oracle_tiny():
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x0 = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=7)
    Rp = hi.gaussian_vectors(w, 1, seed=8)[0]
    dt, Nt, nt, mreg = 0.04, 4, 3, 1.0
    xf, pf, Hi, Hf = D.hmc_update(m, x0, R, Rp, dt, Nt, nt, mreg)
    o = _tight()
    o.dt, o.n_steps, o.n_sub, o.m_reg = dt, Nt, nt, mreg
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        x = torch.tensor(x0, device=DEV)
        acc, dH, terms = ctx.fourier_accel_leapfrog(x, torch.tensor(R, device=DEV),
                                                    torch.tensor(Rp, device=DEV), o, u=0.0)
        assert acc
        assert abs(terms[:3].sum() - Hi) < 1e-9 * abs(Hi)
        assert abs(terms[3:].sum() - Hf) < 1e-9 * abs(Hf)
        assert abs(dH - (Hf - Hi)) < 1e-7
        assert _rel(x.cpu().numpy(), xf) < 1e-8
        assert abs(terms[1] - 0.5 * np.sum(R * R)) < 1e-10 * terms[1]
        # rejection restores the initial field
        x2 = torch.tensor(x0, device=DEV)
        acc2, dH2, _ = ctx.fourier_accel_leapfrog(x2, torch.tensor(R, device=DEV),
                                                  torch.tensor(Rp, device=DEV), o, u=1.0)
        if not (1.0 < np.exp(-dH2)):
            assert not acc2
            assert float((x2.cpu() - torch.tensor(x0)).abs().max()) == 0.0


def test_reversibility_hmc16():
    """Forward N_t steps, negate p, N_t steps back: x returns (FP64 solves
    from v = 0 make the force a deterministic function of x)."""
    w = hi.WORKLOADS["hmc16"]
    m = D.model_of(w)
    x0 = hi.phonon_field(w)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        x = torch.tensor(x0, device=DEV)
        Rt = torch.tensor(hi.gaussian_vectors(w, 2, seed=4), device=DEV)
        Phi = torch.empty_like(Rt)
        ctx.set_field(x)
        ctx.pseudofermion_phi(Rt, Phi)
        p = torch.empty_like(x)
        ctx.mass_apply(1, w.omega0, torch.tensor(hi.gaussian_vectors(w, 1, seed=6)[0],
                                                 device=DEV), p)
        p0 = p.clone()
        o = hg.md_opts(0.01, 4, 4, w.omega0, force_tol=1e-12, prec=hg.HOL_F64)
        ctx.md_integrate(x, p, Phi, o)
        moved = float((x - torch.tensor(x0, device=DEV)).abs().max())
        assert moved > 1e-3
        p.neg_()
        ctx.md_integrate(x, p, Phi, o)
        assert float((x.cpu() - torch.tensor(x0)).abs().max()) < 1e-9
        assert float((p + p0).abs().max()) < 1e-8 * float(p0.abs().max())


def test_hmc16_trajectory_energy_error_scales_as_dt2():
    """The hmc16 workload's trajectory (N_t=20, n_t=4, dt=0.01, m_reg=omega0,
    adiabatic preconditioner, mixed precision): |dH| small, and halving dt
    (twice the steps) divides it by about 4."""
    w = hi.WORKLOADS["hmc16"]
    x0 = hi.phonon_field(w)
    R = torch.tensor(hi.gaussian_vectors(w, 2, seed=9), device=DEV)
    Rp = torch.tensor(hi.gaussian_vectors(w, 1, seed=10)[0], device=DEV)
    out = []
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        for dt, nsteps in ((0.02, 10), (0.01, 20)):
            o = hg.md_opts(dt, nsteps, 4, w.omega0, force_tol=1e-10, action_tol=1e-10,
                           prec=hg.HOL_F32, precond=True)
            x = torch.tensor(x0, device=DEV)
            acc, dH, terms = ctx.fourier_accel_leapfrog(x, R, Rp, o, u=0.0)
            out.append(dH)
    assert abs(out[1]) < 1.0
    assert 2.5 < abs(out[0]) / abs(out[1]) < 6.0


@pytest.mark.parametrize("m_reg", [1.0, float("inf")])
def test_mass_operators_vs_dense_hmc16_shape(m_reg):
    """The Fourier-acceleration mass at the trajectory workload's own shape
    (L=16, Ltau=160: the tau transform specialised for 160) against the
    dense-DFT oracle."""
    w = hi.WORKLOADS["hmc16"]
    m = D.model_of(w)
    p = hi.gaussian_vectors(w, 1, seed=31)[0]
    with hg.Context.from_workload(w) as ctx:
        pt = torch.tensor(p, device=DEV)
        out = torch.empty_like(pt)
        for which, power in ((0, -1.0), (1, 0.5), (2, 1.0)):
            ctx.mass_apply(which, m_reg, pt, out)
            ref = D.mass_apply(m, p, m_reg, power)
            assert _rel(out.cpu().numpy(), ref) < 1e-12, (which, m_reg)
