"""GPU parity of the exact kinetic propagator exp(-dtau K) (the second
discretisation of B_tau, Sec. II D) against the oracle with kinetic="exact"
(scipy's matrix exponential of the dense hopping matrix), through the C ABI.
Marked gpu.

Tolerances follow tests/test_gpu_core.py (FP64 operators 1e-13, FP32 3e-6
of max|ref|); the exact propagator adds one rounding per kept tap, which
stays inside those bounds for the couplings used here.
"""
import ctypes

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
EXACT = "exact"


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def _w(L, T, seed=3, std=1.0, alpha=1.2, mu=0.1, t=1.0, dtau=0.1):
    return hi.Workload("e", L=L, Ltau=T, alpha=alpha, mu=mu, omega0=0.8, x_std=std, seed=seed,
                       t=t, dtau=dtau)


def _ctx(w, max_rhs, kinetic=None):
    return hg.Context(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha,
                      omega0=w.omega0, max_rhs=max_rhs,
                      kinetic=hg.HOL_KINETIC_EXACT if kinetic is None else kinetic)


def _ops(ctx, v, dt):
    out = {}
    for op in (hg.HOL_OP_M, hg.HOL_OP_MT, hg.HOL_OP_MTM):
        vt = torch.tensor(v, device=DEV, dtype=dt)
        o = torch.empty_like(vt)
        ctx.fermion_matvec(op, vt, o)
        out[op] = o.cpu().double().numpy()
    return out


@pytest.mark.parametrize("L,T,t,dtau", [(4, 8, 1.0, 0.1), (6, 10, 1.0, 0.1), (8, 12, 1.3, 0.1),
                                        (10, 6, 1.0, 0.25), (16, 4, 1.0, 0.1), (6, 4, 0.5, 1.2)])
def test_exact_operators_vs_dense(L, T, t, dtau):
    w = _w(L, T, t=t, dtau=dtau)
    x = hi.phonon_field(w)
    m = D.model_of(w, kinetic=EXACT)
    v = hi.gaussian_vectors(w, 3, seed=7)
    Mx = D.fermion_matrix(m, x)
    ref = {hg.HOL_OP_M: np.stack([(Mx @ a.reshape(-1)).reshape(T, -1) for a in v]),
           hg.HOL_OP_MT: np.stack([(Mx.T @ a.reshape(-1)).reshape(T, -1) for a in v])}
    ref[hg.HOL_OP_MTM] = np.stack([(Mx.T @ (Mx @ a.reshape(-1))).reshape(T, -1) for a in v])
    with _ctx(w, 3) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
            got = _ops(ctx, v, dt)
            for op, r in ref.items():
                assert _rel(got[op], r) < tol, (op, dt)


def test_exact_differs_from_checkerboard():
    """At L = 8 the two discretisations differ at O(dtau^2); at L = 4 they
    coincide (the colours commute there)."""
    for L, same in ((8, False), (4, True)):
        w = _w(L, 6)
        x = hi.phonon_field(w)
        v = hi.gaussian_vectors(w, 1, seed=4)
        res = []
        for kin in (hg.HOL_KINETIC_EXACT, hg.HOL_KINETIC_CHECKERBOARD):
            with _ctx(w, 1, kin) as ctx:
                ctx.set_field(torch.tensor(x, device=DEV))
                res.append(_ops(ctx, v, torch.float64)[hg.HOL_OP_M])
        d = _rel(res[0], res[1])
        assert (d < 1e-13) if same else (d > 1e-4), (L, d)


def test_exact_plane_wave_L32_closed_form():
    """x = 0: B_tau = e^{dtau mu} exp(-dtau K), and a plane wave cos(k.r) on one
    slice tau0 is an eigenvector of exp(-dtau K) with eigenvalue
    lam = exp(2 dtau t (cos kx + cos ky)). So M maps it to itself on tau0 and to
    -e^{dtau mu} lam times itself on tau0 + 1; M^T to itself on tau0 and to
    -e^{dtau mu} lam times itself on tau0 - 1 (closed form, no oracle)."""
    L, T, tau0 = 32, 6, 2
    w = hi.Workload("pw", L=L, Ltau=T, alpha=1.0, mu=0.3, omega0=1.0, x_std=1.0, seed=1)
    ix, iy = np.meshgrid(np.arange(L), np.arange(L), indexing="xy")
    waves, lams = [], []
    for nx, ny in [(0, 0), (1, 0), (3, 7), (16, 16), (5, 29)]:
        kx, ky = 2 * np.pi * nx / L, 2 * np.pi * ny / L
        waves.append(np.cos(kx * ix + ky * iy).reshape(-1))
        lams.append(np.exp(2 * w.dtau * w.t * (np.cos(kx) + np.cos(ky))))
    v = np.zeros((len(waves), T, L * L))
    for k, wave in enumerate(waves):
        v[k, tau0] = wave
    g = np.exp(w.dtau * w.mu)
    with _ctx(w, len(waves)) as ctx:
        ctx.set_field(torch.zeros(T, L * L, dtype=torch.float64, device=DEV))
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
            got = _ops(ctx, v, dt)
            for k, (wave, lam) in enumerate(zip(waves, lams)):
                refM = np.zeros((T, L * L))
                refM[tau0] = wave
                refM[tau0 + 1] = -g * lam * wave
                assert _rel(got[hg.HOL_OP_M][k], refM) < tol, (k, dt)
                refT = np.zeros((T, L * L))
                refT[tau0] = wave
                refT[tau0 - 1] = -g * lam * wave
                assert _rel(got[hg.HOL_OP_MT][k], refT) < tol, (k, dt)


def test_exact_L32_operators_vs_blockwise_oracle():
    w = _w(32, 4, seed=11, std=1.5)
    x = hi.phonon_field(w)
    m = D.model_of(w, kinetic=EXACT)
    C = D.kinetic_propagator(m)
    v = hi.gaussian_vectors(w, 2, seed=12)
    refM = np.stack([D.M_apply_blocks(m, x, a, C) for a in v])
    refT = np.stack([D.MT_apply_blocks(m, x, a, C) for a in v])
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
            got = _ops(ctx, v, dt)
            assert _rel(got[hg.HOL_OP_M], refM) < tol, dt
            assert _rel(got[hg.HOL_OP_MT], refT) < tol, dt


@pytest.mark.parametrize("prec,precond", [(hg.HOL_F64, False), (hg.HOL_F64, True),
                                          (hg.HOL_F32, False), (hg.HOL_F32, True)])
def test_exact_cg_vs_dense_solve(prec, precond):
    w = _w(8, 12, seed=5)
    x = hi.phonon_field(w)
    m = D.model_of(w, kinetic=EXACT)
    R = hi.gaussian_vectors(w, 2, seed=6)
    b = np.stack([D.MT_apply(m, x, r) for r in R])
    Mx = D.fermion_matrix(m, x)
    kappa = np.linalg.cond(Mx.T @ Mx)
    vref = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    tol = 1e-12 if prec == hg.HOL_F64 else 1e-9
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        bt = torch.tensor(b, device=DEV)
        v = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, v, tol=tol, prec=prec, precond=precond)
        vg = v.cpu().numpy()
    for k in range(2):
        assert res[k] < tol
        assert D.rel_residual(m, x, b[k], vg[k]) < 2 * tol
        assert np.linalg.norm(vg[k] - vref[k]) / np.linalg.norm(vref[k]) < 2 * kappa * tol


def test_exact_force_and_action_vs_dense():
    w = _w(6, 10, seed=8)
    x = hi.phonon_field(w)
    m = D.model_of(w, kinetic=EXACT)
    Phi = hi.gaussian_vectors(w, 3, seed=9)
    b = D.b_from_phi(m, x, Phi)
    v = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    with _ctx(w, 3) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        F = torch.empty(w.Ltau, w.N, device=DEV, dtype=torch.float64)
        SF = torch.empty(1, device=DEV, dtype=torch.float64)
        ctx.force(torch.tensor(v, device=DEV), torch.tensor(b, device=DEV), F, True, SF)
        assert _rel(F.cpu().numpy(), D.dS_dx(m, x, Phi)) < 1e-12
        assert abs(float(SF) - D.S_F(m, x, Phi)) < 1e-11 * abs(D.S_F(m, x, Phi))


@pytest.mark.parametrize("L,T", [(8, 12), (16, 6), (6, 20)])
def test_exact_precond_vs_oracle(L, T):
    w = _w(L, T, seed=2, mu=0.0, alpha=1.0)
    x = hi.phonon_field(w)
    m = D.model_of(w, kinetic=EXACT)
    v = hi.gaussian_vectors(w, 2, seed=9)
    refs = {
        hg.HOL_PINV: np.stack([D.precond_inverse_apply(m, x, a) for a in v]),
        hg.HOL_PINVT: np.stack([D.precond_inverse_apply(m, x, a, trans=True) for a in v]),
    }
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for which, ref in refs.items():
            for dt, tol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.precond_apply(which, vt, out)
                assert _rel(out.cpu().double().numpy(), ref) < tol, (which, dt)


def test_exact_measurement_vs_direct_sums():
    w = _w(6, 8, seed=4, mu=0.0)
    x = hi.phonon_field(w)
    m = D.model_of(w, kinetic=EXACT)
    xi = hi.z2_vectors(w, 3, seed=3)
    with _ctx(w, 4) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        xt = torch.tensor(xi, device=DEV)
        Gxi = torch.empty_like(xt)
        G2 = torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
        G4 = torch.empty(3, 2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
        ctx.stochastic_measure(xt, Gxi, G2, G4, 7, tol=1e-13)
        g2, g4 = G2.cpu().numpy(), G4.cpu().numpy()
    assert _rel(g2, D.green_average(m, x, xi)) < 1e-10
    ref4 = D.four_point_pairs(m, x, xi)
    for k in range(3):
        assert _rel(g4[k], ref4[k]) < 1e-10, k


def test_exact_hmc_update_vs_oracle():
    w = _w(6, 8, seed=6)
    m = D.model_of(w, kinetic=EXACT)
    x0 = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=7)
    Rp = hi.gaussian_vectors(w, 1, seed=8)[0]
    dt, Nt, nt, mreg = 0.04, 3, 2, 1.0
    xf, pf, Hi, Hf = D.hmc_update(m, x0, R, Rp, dt, Nt, nt, mreg)
    o = hg.md_opts(dt, Nt, nt, mreg, force_tol=1e-13, action_tol=1e-13, prec=hg.HOL_F64,
                   precond=False, check_every=1)
    with _ctx(w, 2) as ctx:
        x = torch.tensor(x0, device=DEV)
        acc, dH, terms = ctx.fourier_accel_leapfrog(x, torch.tensor(R, device=DEV),
                                                    torch.tensor(Rp, device=DEV), o, u=0.0)
        assert acc
        assert abs(terms[:3].sum() - Hi) < 1e-9 * abs(Hi)
        assert abs(terms[3:].sum() - Hf) < 1e-9 * abs(Hf)
        assert _rel(x.cpu().numpy(), xf) < 1e-8


def test_exact_refuses_other_layouts_and_static_path():
    w = _w(8, 8)
    with _ctx(w, 2) as ctx:
        assert ctx.get_option("layout") == 0
        assert ctx.get_option("kpm_registers") == 0
        for name in ("layout", "fused_cg", "merged_cg", "persistent_cg", "kpm_registers"):
            with pytest.raises(hg.HolError):
                ctx.set_option(name, 2 if name == "layout" else 1)
        ctx.set_field(torch.tensor(hi.phonon_field(w), device=DEV))
        best = ctx.tune(2)
        assert ctx.get_option("layout") == 0, best
    lib = hg._abi.load()
    params = hg.hol_params(w.L, w.Ltau, w.dtau, w.t, w.mu, w.alpha, w.omega0, 1,
                           hg.HOL_KINETIC_EXACT)
    x = torch.zeros(w.Ltau, w.N, dtype=torch.float64, device=DEV)
    v = torch.zeros(1, w.Ltau, w.N, dtype=torch.float64, device=DEV)
    out = torch.empty_like(v)
    p = ctypes.c_void_p
    rc = lib.fermion_matvec_static(ctypes.byref(params), p(x.data_ptr()), hg.HOL_OP_M,
                                   p(v.data_ptr()), p(out.data_ptr()), 1,
                                   p(torch.cuda.current_stream().cuda_stream))
    assert rc == hg.HOL_EINVAL
    bad = hg.hol_params(w.L, w.Ltau, w.dtau, w.t, w.mu, w.alpha, w.omega0, 1, 2)
    with pytest.raises(hg.HolError):
        hg.hol_create(bad)
