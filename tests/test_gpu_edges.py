"""Edge cases of the GPU path against the oracle: the smallest lattice, the
longest imaginary-time axis the preconditioner's single-tile transform
takes, many right-hand sides, degenerate couplings, and shapes the
preconditioner refuses. Marked gpu."""
import numpy as np
import pytest
import torch

import holstein_inputs as hi
from oracle import dense as D
from oracle import matfree as MF

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


def _ctx(w, nr):
    return hg.Context(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha,
                      omega0=w.omega0, max_rhs=nr)


@pytest.mark.parametrize("L,T,alpha,mu", [(4, 2, 1.0, 0.0), (4, 4, 0.0, 0.0), (6, 2, 1.5, 2.0),
                                          (8, 6, 0.0, -1.0)])
def test_smallest_shapes_and_degenerate_couplings(L, T, alpha, mu):
    """Ltau = 2 (the corner block and the tau neighbour are the same slice),
    alpha = 0 (M independent of x) and large |mu|: operators, a mixed and an
    FP64 solve, the preconditioner and the force all match the oracle."""
    w = hi.Workload("e", L=L, Ltau=T, alpha=alpha, mu=mu, omega0=1.0, x_std=1.0, seed=2)
    x = hi.phonon_field(w)
    m = D.model_of(w)
    Mx = D.fermion_matrix(m, x)
    v = hi.gaussian_vectors(w, 2, seed=3)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for op, A in ((hg.HOL_OP_M, Mx), (hg.HOL_OP_MT, Mx.T), (hg.HOL_OP_MTM, Mx.T @ Mx)):
            ref = np.stack([(A @ a.reshape(-1)).reshape(T, -1) for a in v])
            for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.fermion_matvec(op, vt, out)
                assert _rel(out.cpu().double().numpy(), ref) < tol, (op, dt)
        b = np.stack([D.MT_apply(m, x, a) for a in v])
        for prec, pc in ((hg.HOL_F64, False), (hg.HOL_F32, False), (hg.HOL_F32, True)):
            bt = torch.tensor(b, device=DEV)
            sol = torch.empty_like(bt)
            its, res = ctx.cg_solve(bt, sol, tol=1e-10, prec=prec, precond=pc)
            s = sol.cpu().numpy()
            assert max(D.rel_residual(m, x, b[k], s[k]) for k in range(2)) < 2e-10
        ref = np.stack([D.precond_inverse_apply(m, x, a) for a in v])
        vt = torch.tensor(v, device=DEV)
        out = torch.empty_like(vt)
        ctx.precond_apply(hg.HOL_PINV, vt, out)
        assert _rel(out.cpu().numpy(), ref) < 1e-11
        vs = np.stack([D.solve_MTM(m, x, bb) for bb in b])
        F = torch.empty(T, w.N, device=DEV, dtype=torch.float64)
        ctx.force(torch.tensor(vs, device=DEV), torch.tensor(b, device=DEV), F, True)
        Phi = np.stack([(D.Lambda(m, x).T @ bb.reshape(-1)).reshape(T, -1) for bb in b])
        assert _rel(F.cpu().numpy(), D.dS_dx(m, x, Phi)) < 1e-11


def test_preconditioner_refuses_ltau_with_a_large_prime_factor():
    """Ltau = 22 = 2 x 11: the tau transform has radices up to 7 only, so the
    preconditioner (and a preconditioned solve) is refused with HOL_EINVAL;
    the plain solve still runs."""
    w = hi.Workload("e", L=8, Ltau=22, seed=4)
    x = hi.phonon_field(w)
    m = D.model_of(w)
    b = hi.gaussian_vectors(w, 1, seed=5)
    with _ctx(w, 1) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        bt = torch.tensor(b, device=DEV)
        out = torch.empty_like(bt)
        with pytest.raises(hg.HolError) as e:
            ctx.precond_apply(hg.HOL_PINV, bt, out)
        assert e.value.code == hg._abi.HOL_EINVAL
        with pytest.raises(hg.HolError):
            ctx.cg_solve(bt, out, tol=1e-10, precond=True)
        its, res = ctx.cg_solve(bt, out, tol=1e-10)
        assert D.rel_residual(m, x, b[0], out.cpu().numpy()[0]) < 2e-10


def test_longest_ltau_of_the_single_tile_transform():
    """L = 32, Ltau = 400 (the FP64 tau transform's tile then fills 200 KB of
    shared memory): P^{-1} and P^{-T} are exact transposes of each other,
    P^{-1} P^{-T} is positive, and the FP32 path agrees with FP64."""
    w = hi.Workload("e", L=32, Ltau=400, alpha=1.0, omega0=1.0, x_std=1.0, seed=6)
    x = hi.phonon_field(w)
    v = hi.gaussian_vectors(w, 2, seed=7)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        vt = torch.tensor(v, device=DEV)
        a = torch.empty_like(vt)
        bq = torch.empty_like(vt)
        ctx.precond_apply(hg.HOL_PINV, vt[:1].contiguous(), a[:1])
        ctx.precond_apply(hg.HOL_PINVT, vt[1:].contiguous(), bq[:1])
        lhs = float((vt[1] * a[0]).sum())
        rhs = float((bq[0] * vt[0]).sum())
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
        z64 = torch.empty_like(vt)
        ctx.precond_apply(hg.HOL_PINV_PINVT, vt, z64)
        assert float((vt * z64).sum(dim=(1, 2)).min()) > 0
        v32 = vt.float()
        z32 = torch.empty_like(v32)
        ctx.precond_apply(hg.HOL_PINV_PINVT, v32, z32)
        assert _rel(z32.double().cpu().numpy(), z64.cpu().numpy()) < 2e-5


def test_many_right_hand_sides():
    """64 right-hand sides at once: the fused M^T M and a masked mixed solve
    (scales spread over 12 decades) stay certified by the matrix-free oracle."""
    w = hi.Workload("e", L=8, Ltau=12, alpha=1.2, seed=8)
    x = hi.phonon_field(w)
    nr = 64
    scale = 10.0 ** np.linspace(-6, 6, nr)
    v = hi.gaussian_vectors(w, nr, seed=9) * scale[:, None, None]
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        out = torch.empty_like(vt)
        ctx.fermion_matvec(hg.HOL_OP_MTM, vt, out)
        got = out.cpu().double().numpy()
        for k in range(0, nr, 7):
            assert _rel(got[k], MF.MTM_apply(w, x, v[k])) < 3e-6
        bt = torch.tensor(v, device=DEV)
        sol = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, sol, tol=1e-8, prec=hg.HOL_F32)
        s = sol.cpu().numpy()
    assert np.all(res < 1e-8)
    assert max(MF.rel_residual(w, x, v[k], s[k]) for k in range(nr)) < 1.01e-8


@pytest.mark.parametrize("T", [2, 4])
def test_trajectory_measurement_and_moves_on_the_shortest_tau_axis(T):
    """Ltau = 2 and 4 (tau transforms of length 2 and 4, doubled domain of
    length 4 and 8): an HMC trajectory, the stochastic Green's function with
    its Wick products, and a reflection and a swap move match the oracle."""
    w = hi.Workload("e", L=4, Ltau=T, alpha=1.1, mu=0.0, omega0=1.0, x_std=1.0, seed=10)
    m = D.model_of(w)
    x0 = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=11)
    Rp = hi.gaussian_vectors(w, 1, seed=12)[0]
    dt, Nt, nt, mreg = 0.05, 3, 2, 1.0
    xf, pf, Hi, Hf = D.hmc_update(m, x0, R, Rp, dt, Nt, nt, mreg)
    o = hg.md_opts(dt, Nt, nt, mreg, force_tol=1e-13, action_tol=1e-13, prec=hg.HOL_F64,
                   precond=False, check_every=1)
    xi = hi.z2_vectors(w, 3, seed=13)
    Phi = D.phi_from_R(m, x0, R)
    with _ctx(w, 4) as ctx:
        x = torch.tensor(x0, device=DEV)
        acc, dH, terms = ctx.fourier_accel_leapfrog(x, torch.tensor(R, device=DEV),
                                                    torch.tensor(Rp, device=DEV), o, u=0.0)
        assert acc
        assert abs(terms[:3].sum() - Hi) < 1e-9 * abs(Hi)
        assert abs(terms[3:].sum() - Hf) < 1e-9 * abs(Hf)
        assert _rel(x.cpu().numpy(), xf) < 1e-8
        ctx.set_field(torch.tensor(x0, device=DEV))
        xt = torch.tensor(xi, device=DEV)
        Gxi = torch.empty_like(xt)
        G2 = torch.empty(2 * T, w.L, w.L, dtype=torch.float64, device=DEV)
        G4 = torch.empty(3, 2 * T, w.L, w.L, dtype=torch.float64, device=DEV)
        ctx.stochastic_measure(xt, Gxi, G2, G4, 7, tol=1e-13)
        assert _rel(G2.cpu().numpy(), D.green_average(m, x0, xi)) < 1e-10
        ref4 = D.four_point_pairs(m, x0, xi)
        for k in range(3):
            assert _rel(G4.cpu().numpy()[k], ref4[k]) < 1e-10
        for kind, i, j in ((hg.HOL_REFLECT, 5, -1), (hg.HOL_SWAP, 1, 2)):
            xg = torch.tensor(x0, device=DEV)
            a_, dS, S = ctx.global_update(xg, torch.tensor(Phi, device=DEV), kind, i, j, u=0.5,
                                          tol=1e-13)
            a_o, dS_o, x_o = D.global_update(m, x0, Phi, kind, i, j, 0.5)
            assert abs(dS - dS_o) < 1e-8 * D.action(m, x0, Phi)
            if abs(np.log(0.5) + dS_o) > 1e-6:
                assert a_ == a_o


def test_misaligned_device_vectors_are_refused_on_the_host():
    """A device vector that is not 16-byte aligned (a view one element into an
    allocation) is refused with HOL_EINVAL before anything is launched."""
    w = hi.Workload("e", L=8, Ltau=8, seed=14)
    x = hi.phonon_field(w)
    n = w.n
    with _ctx(w, 1) as ctx:
        raw = torch.zeros(n + 1, dtype=torch.float64, device=DEV)
        bad = raw[1:].view(1, w.Ltau, w.N)                 # 8 bytes past a 256-byte boundary
        good = torch.zeros(1, w.Ltau, w.N, dtype=torch.float64, device=DEV)
        with pytest.raises(hg.HolError) as e:
            ctx.set_field(raw[1:].view(w.Ltau, w.N))
        assert e.value.code == hg._abi.HOL_EINVAL
        ctx.set_field(torch.tensor(x, device=DEV))
        calls = [lambda: ctx.fermion_matvec(hg.HOL_OP_M, bad, good),
                 lambda: ctx.fermion_matvec(hg.HOL_OP_M, good, bad),
                 lambda: ctx.precond_apply(hg.HOL_PINV, bad, good),
                 lambda: ctx.cg_solve(bad, good, tol=1e-8),
                 lambda: ctx.force(good, bad, torch.empty(w.Ltau, w.N, dtype=torch.float64,
                                                          device=DEV))]
        for call in calls:
            with pytest.raises(hg.HolError) as e:
                call()
            assert e.value.code == hg._abi.HOL_EINVAL
        raw32 = torch.zeros(n + 2, dtype=torch.float32, device=DEV)
        bad32 = raw32[2:].view(1, w.Ltau, w.N)             # 8 bytes off: float4 loads would fault
        good32 = torch.zeros(1, w.Ltau, w.N, dtype=torch.float32, device=DEV)
        with pytest.raises(hg.HolError):
            ctx.fermion_matvec(hg.HOL_OP_MTM, bad32, good32)
        # the context is still usable
        out = torch.empty_like(good)
        ctx.fermion_matvec(hg.HOL_OP_M, good, out)
        torch.cuda.synchronize()
