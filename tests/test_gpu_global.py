"""GPU parity of the reflection and swap updates (Sec. IV) against the dense
oracle, through the C ABI. Marked gpu.

Tolerance: the actions are evaluated with FP64 solves to 1e-13; dS agrees
with the dense definition to 1e-8 of |S| (S ~ 1e3 here; the solve error
enters S_F through b . v, bounded by kappa(M^T M) * tol * |b|^2)."""
import numpy as np
import pytest
import torch

import holstein_inputs as hi
from oracle import dense as D

pytestmark = pytest.mark.gpu

hg = pytest.importorskip("paper_2203_01291_gb300")
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hg.build.build()
    torch.cuda.set_device(0)


def _setup(L, T, alpha=1.2, t=1.0, seed=51, n_pf=2):
    w = hi.Workload("g", L=L, Ltau=T, t=t, alpha=alpha, mu=0.0, omega0=1.0, x_std=1.0, seed=seed)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, n_pf, seed=seed + 1)
    Phi = D.phi_from_R(m, x, R)
    ctx = hg.Context(L=L, Ltau=T, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha, omega0=w.omega0,
                     max_rhs=n_pf)
    return w, m, x, Phi, ctx


@pytest.mark.parametrize("L,T", [(4, 40), (8, 24)])
@pytest.mark.parametrize("kind,i,j", [(0, 3, -1), (1, 2, 3), (1, 0, 9)])
def test_global_update_matches_oracle(L, T, kind, i, j):
    w, m, x, Phi, ctx = _setup(L, T)
    with ctx:
        xt = torch.tensor(x, device=DEV)
        Pt = torch.tensor(Phi, device=DEV)
        for u in (1e-6, 0.999999):   # accept (unless dS is huge) / reject (unless dS < 0)
            xg = xt.clone()
            acc, dS, S = ctx.global_update(xg, Pt, kind, i, j, u=u, tol=1e-13)
            acc_o, dS_o, x_o = D.global_update(m, x, Phi, kind, i, j, u)
            S0 = D.action(m, x, Phi)
            assert abs(dS - dS_o) < 1e-8 * S0
            if abs(np.log(u) + dS_o) > 1e-6:
                assert acc == acc_o
            assert np.array_equal(xg.cpu().numpy(), x_o if acc else x)
            S_kept = D.action(m, xg.cpu().numpy(), Phi)
            assert abs(S - S_kept) < 1e-8 * S_kept
            # the context now describes the kept field
            v = torch.tensor(hi.gaussian_vectors(w, 1, seed=9), device=DEV)
            out = torch.empty_like(v)
            ctx.fermion_matvec(hg.HOL_OP_M, v, out)
            ref = D.M_apply(m, xg.cpu().numpy(), v.cpu().numpy()[0])
            assert np.abs(out.cpu().numpy()[0] - ref).max() < 1e-12 * np.abs(ref).max()


def test_global_update_chain_reuses_the_action():
    """A sequence of moves passing S along needs one solve per move and gives
    the same actions as fresh evaluations."""
    w, m, x, Phi, ctx = _setup(4, 40, seed=61)
    rng = np.random.default_rng(62)
    with ctx:
        xt = torch.tensor(x, device=DEV)
        Pt = torch.tensor(Phi, device=DEV)
        S = None
        for k in range(6):
            kind = k % 2
            i = int(rng.integers(0, w.N))
            j = (i + 1) % w.N
            acc, dS, S = ctx.global_update(xt, Pt, kind, i, j, u=float(rng.random()), tol=1e-13,
                                           S_cur=S)
            assert abs(S - D.action(m, xt.cpu().numpy(), Phi)) < 1e-8 * S


def test_global_update_free_without_coupling_and_errors():
    w, m, x, Phi, ctx = _setup(4, 40, alpha=0.0, seed=71)
    with ctx:
        xt = torch.tensor(x, device=DEV)
        Pt = torch.tensor(Phi, device=DEV)
        for kind, i, j in ((0, 5, -1), (1, 5, 6)):
            acc, dS, S = ctx.global_update(xt, Pt, kind, i, j, u=0.999, tol=1e-13)
            assert acc and abs(dS) < 1e-8 * S
        for bad in ((2, 0, 1), (0, -1, 0), (0, 16, 0), (1, 3, 3), (1, 3, 16)):
            with pytest.raises(hg.HolError):
                ctx.global_update(xt, Pt, *bad, u=0.5)


def test_global_update_mixed_precision_solve():
    """The tight action solve in mixed precision (FP32 iterations, FP64
    certified residual 1e-10) gives the same dS to the accuracy the
    certification implies."""
    w, m, x, Phi, ctx = _setup(8, 24, seed=81)
    with ctx:
        xt = torch.tensor(x, device=DEV)
        Pt = torch.tensor(Phi, device=DEV)
        acc, dS, S = ctx.global_update(xt.clone(), Pt, 0, 10, -1, u=0.5, tol=1e-10,
                                       prec=hg.HOL_F32)
        _, dS_o, _ = D.global_update(m, x, Phi, 0, 10, -1, 0.5)
        assert abs(dS - dS_o) < 1e-6 * D.action(m, x, Phi)
