"""GPU parity of the adiabatic preconditioner (Sec. VI, App. C) and of
preconditioned CG against the oracle (step-by-step KPM of oracle/dense.py).

Tolerances: FP64 P^{-1} v to 1e-11 of max|ref| (the KPM sums up to ~60 terms
of a recurrence whose vectors stay O(|u|), so roundoff grows like the order
times epsilon; the twisted FFTs add O(log T) epsilon); FP32 to 2e-5 of max|ref|.
"""
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


def _setup(L, T, seed=3, std=1.0, alpha=1.0, nr=2):
    w = hi.Workload("p", L=L, Ltau=T, alpha=alpha, mu=0.0, omega0=1.0, x_std=std, seed=seed)
    x = hi.phonon_field(w)
    ctx = hg.Context(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha,
                     omega0=w.omega0, max_rhs=nr)
    ctx.set_field(torch.tensor(x, device=DEV))
    return w, x, ctx


@pytest.mark.parametrize("L,T", [(4, 40), (6, 12), (8, 24), (12, 10), (4, 14), (8, 30),
                                 (16, 20), (32, 12), (16, 6)])
def test_precond_apply_vs_oracle(L, T):
    w, x, ctx = _setup(L, T)
    m = D.model_of(w)
    v = hi.gaussian_vectors(w, 2, seed=9)
    refs = {
        hg.HOL_PINV: np.stack([D.precond_inverse_apply(m, x, a) for a in v]),
        hg.HOL_PINVT: np.stack([D.precond_inverse_apply(m, x, a, trans=True) for a in v]),
    }
    refs[hg.HOL_PINV_PINVT] = np.stack(
        [D.precond_inverse_apply(m, x, D.precond_inverse_apply(m, x, a, trans=True)) for a in v])
    with ctx:
        for which, ref in refs.items():
            for dt, tol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.precond_apply(which, vt, out)
                assert _rel(out.cpu().double().numpy(), ref) < tol, (which, dt)


@pytest.mark.parametrize("kpm,queue", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1), (2, 3)])
@pytest.mark.parametrize("L,T", [(16, 20), (32, 12), (16, 40), (32, 200)])
def test_precond_fp32_kpm_variants(kpm, queue, L, T):
    """The FP32 KPM kernels (shared-memory, registers with four or two
    columns per lane, one block per problem or a persistent grid taking
    problems from a queue) all match the oracle's step-by-step KPM, also
    twice in a row (the queue resets itself)."""
    w, x, ctx = _setup(L, T, seed=4)
    m = D.model_of(w)
    v = hi.gaussian_vectors(w, 2, seed=10)
    ref = np.stack(
        [D.precond_inverse_apply(m, x, D.precond_inverse_apply(m, x, a, trans=True)) for a in v])
    with ctx:
        ctx.set_option("kpm_registers", kpm)
        ctx.set_option("kpm_queue", queue)
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        for _ in range(2):
            out = torch.full_like(vt, float("nan"))
            ctx.precond_apply(hg.HOL_PINV_PINVT, vt, out)
            assert _rel(out.cpu().double().numpy(), ref) < 2e-5


@pytest.mark.parametrize("L,T,nr", [(4, 12, 3), (6, 10, 3), (8, 12, 3), (10, 8, 2), (12, 12, 3),
                                    (14, 6, 1), (16, 8, 3), (18, 6, 2), (20, 8, 1), (22, 4, 1),
                                    (24, 6, 2), (26, 4, 3), (28, 6, 3), (30, 4, 1), (32, 6, 2)])
def test_precond_fp32_lane_layout_vs_oracle(L, T, nr):
    """The lane-layout FP32 KPM (kpm_registers 3: lane = column, rows in
    registers, real and imaginary parts in two lane groups whose recurrences
    meet only in the coefficient sums) for every lattice shape it has to
    cover: several problems per warp (L <= 16, with an idle lane group when
    32 / L is odd), two warps per problem (L > 16), right-hand side counts
    that leave a block's last slot empty. P^{-1}, P^{-T} and P^{-1} P^{-T}
    against the oracle's step-by-step KPM (FP32; the FP64 path, which keeps
    the shared-memory kernel, is checked alongside)."""
    w, x, ctx = _setup(L, T, seed=5, nr=nr)
    m = D.model_of(w)
    v = hi.gaussian_vectors(w, nr, seed=11)
    refs = {
        hg.HOL_PINV: np.stack([D.precond_inverse_apply(m, x, a) for a in v]),
        hg.HOL_PINVT: np.stack([D.precond_inverse_apply(m, x, a, trans=True) for a in v]),
    }
    refs[hg.HOL_PINV_PINVT] = np.stack(
        [D.precond_inverse_apply(m, x, D.precond_inverse_apply(m, x, a, trans=True)) for a in v])
    with ctx:
        ctx.set_option("kpm_registers", 3)
        for dt, tol in ((torch.float32, 2e-5), (torch.float64, 1e-11)):   # FP64: shared memory
            vt = torch.tensor(v, device=DEV, dtype=dt)
            for which, ref in refs.items():
                out = torch.full_like(vt, float("nan"))
                ctx.precond_apply(which, vt, out)
                assert _rel(out.cpu().double().numpy(), ref) < tol, (L, which, dt)


def test_precond_transpose_identity_and_spd():
    """<w, P^{-1} v> = <P^{-T} w, v> and <v, P^{-1} P^{-T} v> > 0 on the GPU."""
    w_, x, ctx = _setup(8, 40, std=1.5)
    v = torch.tensor(hi.gaussian_vectors(w_, 2, seed=1), device=DEV)
    with ctx:
        a = torch.empty_like(v)
        b = torch.empty_like(v)
        ctx.precond_apply(hg.HOL_PINV, v[:1].contiguous(), a[:1])
        ctx.precond_apply(hg.HOL_PINVT, v[1:].contiguous(), b[:1])
        lhs = float((v[1] * a[0]).sum())
        rhs = float((b[0] * v[0]).sum())
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
        ctx.precond_apply(hg.HOL_PINV_PINVT, v, a)
        assert float((v * a).sum(dim=(1, 2)).min()) > 0


def test_precond_exact_when_x_constant_in_tau():
    """x constant in tau: P = M (Sec. VI B), so P^{-1} is (up to the KPM
    truncation) M^{-1}, and PCG needs far fewer iterations than CG."""
    L, T = 8, 40
    w = hi.Workload("c", L=L, Ltau=T, alpha=1.0, omega0=1.0)
    xc = np.tile(hi.phonon_field(w)[0], (T, 1))
    m = D.model_of(w)
    ctx = hg.Context(L=L, Ltau=T, alpha=1.0, omega0=1.0, max_rhs=1)
    b = hi.gaussian_vectors(w, 1, seed=4)
    with ctx:
        ctx.set_field(torch.tensor(xc, device=DEV))
        bt = torch.tensor(b, device=DEV)
        v = torch.empty_like(bt)
        it_p, res_p = ctx.cg_solve(bt, v, tol=1e-10, precond=True, check_every=1)
        it_0, res_0 = ctx.cg_solve(bt, v, tol=1e-10, precond=False, check_every=1)
        assert res_p[0] < 1e-10 and res_0[0] < 1e-10
        assert it_p[0] * 4 < it_0[0]
        assert D.rel_residual(m, xc, b[0], v.cpu().numpy()[0]) < 1e-10


@pytest.mark.parametrize("prec", [hg.HOL_F32, hg.HOL_F64])
@pytest.mark.parametrize("L,T", [(12, 40), (16, 160), (28, 24)])
def test_pcg_fused_update_matches_unfused(prec, L, T):
    """PCG with the vector update fused into the preconditioner's forward
    transform (fused_pc_update) runs the same iteration as the separate
    update kernel: the same iteration counts (up to the regrouped r.r
    partials of the convergence estimate, which can move a chunk decision by
    one chunk), certified residuals, and solutions within the residual's
    bound of each other and of the oracle's residual check."""
    w = hi.Workload("f", L=L, Ltau=T, alpha=1.0, omega0=1.0, x_std=1.0, seed=40 + L)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 3, seed=41)
    tol = 1e-8 if prec == hg.HOL_F32 else 1e-10
    out = {}
    with hg.Context.from_workload(w, max_rhs=3) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        Rt = torch.tensor(R, device=DEV)
        bt = torch.empty_like(Rt)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rt, bt)
        for fused in (0, 1):
            ctx.set_option("fused_pc_update", fused)
            v = torch.empty_like(bt)
            its, res = ctx.cg_solve(bt, v, tol=tol, prec=prec, precond=True, check_every=2,
                                    reliable_every=20)
            out[fused] = (its, res, v.cpu().numpy())
        b = bt.cpu().numpy()
    for fused in (0, 1):
        assert np.all(out[fused][1] < tol)
    assert np.all(np.abs(out[0][0] - out[1][0]) <= 2)
    d = np.abs(out[0][2] - out[1][2]).max() / np.abs(out[0][2]).max()
    assert d < 1e-4 if prec == hg.HOL_F32 else d < 1e-6
    for k in range(3):
        assert MF.rel_residual(w, x, b[k], out[1][2][k]) < 1.01 * tol


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("prec,tol", [(hg.HOL_F64, 1e-12), (hg.HOL_F32, 1e-8)])
def test_pcg_tiny_vs_lu(prec, tol, fused):
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=2)
    b = np.stack([D.MT_apply(m, x, r) for r in R])
    vref = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    Mx = D.fermion_matrix(m, x)
    kappa = np.linalg.cond(Mx.T @ Mx)
    _, it_ref = D.pcg(m, x, b[0], tol=tol, precond=True)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("fused_pc_update", fused)   # the update inside the forward transform
        bt = torch.tensor(b, device=DEV)
        v = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, v, tol=tol, precond=True, prec=prec, check_every=1,
                                reliable_every=25)
        vg = v.cpu().numpy()
    for k in range(2):
        assert res[k] < tol
        assert D.rel_residual(m, x, b[k], vg[k]) < 1.01 * tol
        assert np.linalg.norm(vg[k] - vref[k]) / np.linalg.norm(vref[k]) < 2 * kappa * tol
    if prec == hg.HOL_F64:
        # same algorithm as the oracle's textbook PCG: same iteration count
        assert abs(int(its[0]) - it_ref) <= 1


def test_pcg_hmc16_certified_by_oracle():
    """The preconditioned solve of the L=16, Ltau=160 HMC workload, mixed
    precision, residual recomputed by the matrix-free oracle."""
    w = hi.WORKLOADS["hmc16"]
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=3)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        Rt = torch.tensor(R, device=DEV)
        bt = torch.empty_like(Rt)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rt, bt)
        v = torch.empty_like(bt)
        its_p, res_p = ctx.cg_solve(bt, v, tol=1e-8, precond=True, prec=hg.HOL_F32)
        vp = v.cpu().numpy()
        its_0, _ = ctx.cg_solve(bt, v, tol=1e-8, precond=False, prec=hg.HOL_F32)
        b = bt.cpu().numpy()
    for k in range(2):
        assert res_p[k] < 1e-8
        assert MF.rel_residual(w, x, b[k], vp[k]) < 1.01e-8
    assert np.mean(its_p) < np.mean(its_0)


FULL_SIZE = {
    # the fields the benchmark rows precondition: the L=32 CG workload, the
    # hmc16 trajectory workload, and the L=28 chain of the batching workload;
    # Ltau = 200, 160 and 120 run the tau transforms specialised for them
    "big32": hi.WORKLOADS["big32"],
    "hmc16": hi.WORKLOADS["hmc16"],
    "chain28": hi.chain_workloads(8, 120)[-1],
}


@pytest.mark.parametrize("name", sorted(FULL_SIZE))
def test_precond_full_size_vs_oracle(name):
    """P^{-1}, P^{-T} and P^{-1} P^{-T} at the workloads' own shapes, with the
    launch dispatch the benchmark takes (default options, tuned operator
    shapes), element by element against the oracle's step-by-step KPM in
    FP64 (1e-11) and FP32 (2e-5), 2 right-hand sides. A wrong twiddle in a
    length-specialised transform would give a preconditioner that is still
    SPD (so PCG still converges) but not this one."""
    w = FULL_SIZE[name]
    assert w.Ltau in (120, 160, 200)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    v = hi.gaussian_vectors(w, 2, seed=19)
    refs = {
        hg.HOL_PINV: np.stack([D.precond_inverse_apply(m, x, a) for a in v]),
        hg.HOL_PINVT: np.stack([D.precond_inverse_apply(m, x, a, trans=True) for a in v]),
    }
    refs[hg.HOL_PINV_PINVT] = np.stack(
        [D.precond_inverse_apply(m, x, D.precond_inverse_apply(m, x, a, trans=True)) for a in v])
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.tune(2)
        for which, ref in refs.items():
            for dt, tol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.precond_apply(which, vt, out)
                err = _rel(out.cpu().double().numpy(), ref)
                assert err < tol, (name, which, dt, err)


@pytest.mark.parametrize("a1,a2", [(50, 100), (150, 50), (25, 200)])
def test_precond_order_constants_vs_oracle(a1, a2):
    """The Chebyshev orders N_P(omega) = max(1, floor(db (a1/phi + a2))) of
    Eq. (NP_heuristic) with other constants than the paper's a1 = a2 = 1
    (launch options, in percent): P^{-1} P^{-T} against the oracle's KPM with
    the same constants, FP64 and FP32."""
    w, x, ctx = _setup(16, 40, seed=8, std=1.2)
    m = D.model_of(w)
    v = hi.gaussian_vectors(w, 2, seed=11)
    ref = np.stack([D.precond_inverse_apply(
        m, x, D.precond_inverse_apply(m, x, a, trans=True, a1=a1 / 100, a2=a2 / 100),
        a1=a1 / 100, a2=a2 / 100) for a in v])
    with ctx:
        ctx.set_option("kpm_a1_percent", a1)
        ctx.set_option("kpm_a2_percent", a2)
        assert ctx.get_option("kpm_a1_percent") == a1
        ctx.set_field(torch.tensor(x, device=DEV))       # the plan is formed here
        for dt, tol in ((torch.float64, 1e-11), (torch.float32, 2e-5)):
            vt = torch.tensor(v, device=DEV, dtype=dt)
            out = torch.empty_like(vt)
            ctx.precond_apply(hg.HOL_PINV_PINVT, vt, out)
            assert _rel(out.cpu().double().numpy(), ref) < tol, dt
