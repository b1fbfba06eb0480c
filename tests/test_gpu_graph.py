"""Device-driven solves and batched trajectories as CUDA graphs
(cg_solve_graph, hmc_batch_graph) give bitwise the results of the
host-driven cg_solve and fourier_accel_leapfrog: the same kernels run with
the same decisions, only taken on the device. Marked gpu."""
import numpy as np
import pytest
import torch

import holstein_inputs as hi

pytestmark = pytest.mark.gpu

hg = pytest.importorskip("paper_2203_01291_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hg.build.build()
    torch.cuda.set_device(0)


DEV = "cuda"


def _both(w, nr, options=None, **kw):
    x = torch.tensor(hi.phonon_field(w), device=DEV)
    R = torch.tensor(hi.gaussian_vectors(w, nr, seed=w.seed + 1), device=DEV)
    with hg.Context.from_workload(w, max_rhs=nr) as ctx:
        ctx.set_field(x)
        for name, value in (options or {}).items():
            ctx.set_option(name, value)
        b = torch.empty_like(R)
        ctx.fermion_matvec(hg.HOL_OP_MT, R, b)
        v0 = torch.empty_like(b)
        v1 = torch.full_like(b, float("nan"))
        it0, r0 = ctx.cg_solve(b, v0, **kw)
        it1, r1 = ctx.cg_solve_graph(b, v1, **kw)
        torch.cuda.synchronize()
        return it0, r0, v0.cpu().numpy(), it1, r1, v1.cpu().numpy()


@pytest.mark.parametrize("prec", [hg.HOL_F64, hg.HOL_F32])
@pytest.mark.parametrize("precond,fused", [(False, 0), (True, 0), (True, 1)])
def test_graph_solve_equals_host_solve(prec, precond, fused):
    w = hi.Workload("g", L=8, Ltau=24, alpha=1.2, omega0=1.0, x_std=1.0, seed=71)
    it0, r0, v0, it1, r1, v1 = _both(w, 3, tol=1e-10, prec=prec, precond=precond,
                                     reliable_every=20, check_every=4,
                                     options={"fused_pc_update": fused})
    assert np.array_equal(it0, it1) and np.array_equal(r0, r1)
    assert np.array_equal(v0, v1)
    assert np.all(r1 < 1e-10)


def test_graph_solve_equals_host_solve_big32_mixed():
    """The benchmark's solve: L=32, Ltau=200, 16 rhs, mixed, reliable update
    every 50 iterations, certified 1e-8."""
    w = hi.WORKLOADS["big32"]
    it0, r0, v0, it1, r1, v1 = _both(w, 16, tol=1e-8, prec=hg.HOL_F32, reliable_every=50,
                                     check_every=10, max_iter=50000)
    assert np.array_equal(it0, it1) and np.array_equal(r0, r1)
    assert np.array_equal(v0, v1)


def test_graph_solve_stops_at_the_iteration_cap():
    """The device-side loop is bounded: an unreachable tolerance ends at
    max_iter (within one chunk) with HOL_ENOTCONV, like cg_solve."""
    w = hi.Workload("g", L=8, Ltau=24, alpha=1.2, seed=72)
    x = torch.tensor(hi.phonon_field(w), device=DEV)
    b = torch.tensor(hi.gaussian_vectors(w, 2, seed=3), device=DEV)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        ctx.set_field(x)
        v = torch.empty_like(b)
        with pytest.raises(hg.HolError) as e:
            ctx.cg_solve_graph(b, v, tol=1e-30, max_iter=12, check_every=4)
        assert e.value.code == hg._abi.HOL_ENOTCONV
        its, res = ctx.cg_solve_graph(b, v, tol=1e-30, max_iter=12, check_every=4,
                                      raise_on_nonconv=False)
        assert np.all(its >= 12) and np.all(its < 12 + 4) and np.all(res > 0)
        with pytest.raises(hg.HolError) as e:
            ctx.cg_solve_graph(b, v, tol=1e-8, check_every=5)
        assert e.value.code == hg._abi.HOL_EINVAL


SIZES = (8, 12, 16, 10, 8, 20)


def _chains(Ltau=20):
    return [hi.Workload(f"c{k}", L=L, Ltau=Ltau, omega0=1.0, alpha=1.0, seed=500 + k)
            for k, L in enumerate(SIZES)]


@pytest.mark.parametrize("prec,precond,n_steps", [(hg.HOL_F32, False, 3), (hg.HOL_F32, True, 4),
                                                  (hg.HOL_F64, True, 1)])
def test_hmc_batch_graph_equals_sequential(prec, precond, n_steps):
    ws = _chains()
    o = hg.md_opts(0.02, n_steps, 2, 1.0, force_tol=1e-8, action_tol=1e-10, prec=prec,
                   precond=precond)
    u = hi.uniforms(len(ws), seed=9)
    ctxs = [hg.Context.from_workload(w, max_rhs=2) for w in ws]
    try:
        ref_x, ref_dh, ref_acc = [], [], []
        for w, c, uk in zip(ws, ctxs, u):
            x = torch.tensor(hi.phonon_field(w), device=DEV)
            R = torch.tensor(hi.gaussian_vectors(w, 2, seed=w.seed + 1), device=DEV)
            Rp = torch.tensor(hi.gaussian_vectors(w, 1, seed=w.seed + 2)[0], device=DEV)
            acc, dh, _ = c.fourier_accel_leapfrog(x, R, Rp, o, uk)
            ref_x.append(x.cpu().numpy())
            ref_dh.append(dh)
            ref_acc.append(acc)
        xs = [torch.tensor(hi.phonon_field(w), device=DEV) for w in ws]
        Rs = [torch.tensor(hi.gaussian_vectors(w, 2, seed=w.seed + 1), device=DEV) for w in ws]
        Rps = [torch.tensor(hi.gaussian_vectors(w, 1, seed=w.seed + 2)[0], device=DEV)
               for w in ws]
        acc, dh = hg.hmc_batch_graph(ctxs, xs, Rs, Rps, o, u)
        torch.cuda.synchronize()
        for k in range(len(ws)):
            assert dh[k] == ref_dh[k], (k, dh[k], ref_dh[k])
            assert bool(acc[k]) == bool(ref_acc[k])
            assert np.array_equal(xs[k].cpu().numpy(), ref_x[k])
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("concurrency", [0, 3])
def test_measure_batch_graph_equals_stochastic_measure(concurrency):
    """Every chain's 2-point function, Wick products and probe solutions from
    the one-graph batched measurement are bitwise those of stochastic_measure
    run chain by chain (mixed precision, probes in blocks of max_rhs), with
    all chains in flight or at most three."""
    ws = _chains()[:4]
    opts = hg.hol_cg_opts(1e-10, 100000, 0, hg.HOL_F32, 50, 10)
    ctxs = [hg.Context.from_workload(w, max_rhs=4) for w in ws]
    try:
        xis, G2s, G4s, Gxis, refs = [], [], [], [], []
        for w, c in zip(ws, ctxs):
            c.set_field(torch.tensor(hi.phonon_field(w), device=DEV))
            xi = torch.tensor(hi.z2_vectors(w, 6, seed=w.seed + 3), device=DEV)
            Gxi = torch.empty_like(xi)
            G2 = torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
            G4 = torch.empty(3, 2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
            c.stochastic_measure(xi, Gxi, G2, G4, 7, tol=1e-10, prec=hg.HOL_F32)
            refs.append((Gxi.cpu().numpy(), G2.cpu().numpy(), G4.cpu().numpy()))
            xis.append(xi)
            Gxis.append(torch.full_like(xi, float("nan")))
            G2s.append(torch.full_like(G2, float("nan")))
            G4s.append(torch.full_like(G4, float("nan")))
        hg.measure_batch_graph(ctxs, xis, Gxis, G2s, opts, G4s=G4s, four_point=7,
                               concurrency=concurrency)
        torch.cuda.synchronize()
        for k in range(len(ws)):
            assert np.array_equal(Gxis[k].cpu().numpy(), refs[k][0])
            assert np.array_equal(G2s[k].cpu().numpy(), refs[k][1])
            assert np.array_equal(G4s[k].cpu().numpy(), refs[k][2])
    finally:
        for c in ctxs:
            c.close()
