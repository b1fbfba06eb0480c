"""GPU parity of the core path (set-up, M / M^T / M^T M, CG, force, Phi and b)
against the oracle, through the C ABI. Marked gpu.

Tolerances
----------
* FP64 operators: 1e-13 of max|ref| (a handful of roundings per entry).
* FP32 operators: 3e-6 of max|ref| (FP32 epsilon 6e-8 times the ~20
  roundings of a checkerboard sweep, two sweeps for M^T M, some headroom).
* FP64 CG: the certified true residual is below tol; the solution error is
  bounded by kappa(M^T M) * tol with kappa computed from the dense matrix.
* Forces from the same (v, b): 1e-12 of max|ref| in FP64.
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
SHAPES = [(4, 40), (6, 12), (8, 24), (12, 10), (16, 8)]
MF_SHAPES = [(20, 6), (24, 8), (28, 4), (32, 6), (10, 14), (30, 4)]


def _field(L, T, seed=3, std=1.0):
    w = hi.Workload("t", L=L, Ltau=T, alpha=1.2, mu=0.1, omega0=0.8, x_std=std, seed=seed)
    return w, hi.phonon_field(w)


def _ctx(w, max_rhs):
    return hg.Context(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu, alpha=w.alpha,
                      omega0=w.omega0, max_rhs=max_rhs)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("L,T", SHAPES)
def test_operators_vs_dense(L, T):
    w, x = _field(L, T)
    m = D.model_of(w)
    nr = 3
    v = hi.gaussian_vectors(w, nr, seed=7)
    Mx = D.fermion_matrix(m, x)
    ref = {hg.HOL_OP_M: np.stack([(Mx @ a.reshape(-1)).reshape(T, -1) for a in v]),
           hg.HOL_OP_MT: np.stack([(Mx.T @ a.reshape(-1)).reshape(T, -1) for a in v])}
    ref[hg.HOL_OP_MTM] = np.stack([(Mx.T @ (Mx @ a.reshape(-1))).reshape(T, -1) for a in v])
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for op, r in ref.items():
            for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.fermion_matvec(op, vt, out)
                assert _rel(out.cpu().double().numpy(), r) < tol, (op, dt)


@pytest.mark.parametrize("L,T", MF_SHAPES)
def test_operators_vs_matrix_free(L, T):
    w, x = _field(L, T, seed=11)
    v = hi.gaussian_vectors(w, 2, seed=8)
    ref_M = np.stack([MF.M_apply(w, x, a) for a in v])
    ref_MT = np.stack([MF.MT_apply(w, x, a) for a in v])
    ref_MTM = np.stack([MF.MTM_apply(w, x, a) for a in v])
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for op, r in ((hg.HOL_OP_M, ref_M), (hg.HOL_OP_MT, ref_MT), (hg.HOL_OP_MTM, ref_MTM)):
            for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.fermion_matvec(op, vt, out)
                assert _rel(out.cpu().double().numpy(), r) < tol, (op, dt)


def test_operators_full_size_big32():
    """L=32, Ltau=200, 16 right-hand sides (the benchmark workload): every
    output element against the matrix-free oracle."""
    w = hi.WORKLOADS["big32"]
    x = hi.phonon_field(w)
    v = hi.gaussian_vectors(w, w.n_rhs, seed=21)
    with _ctx(w, w.n_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for op, f in ((hg.HOL_OP_M, MF.M_apply), (hg.HOL_OP_MT, MF.MT_apply),
                      (hg.HOL_OP_MTM, MF.MTM_apply)):
            ref = np.stack([f(w, x, a) for a in v])
            for dt, tol in ((torch.float64, 1e-13), (torch.float32, 3e-6)):
                vt = torch.tensor(v, device=DEV, dtype=dt)
                out = torch.empty_like(vt)
                ctx.fermion_matvec(op, vt, out)
                assert _rel(out.cpu().double().numpy(), ref) < tol, (op, dt)


def test_cg_fp64_tiny_vs_lu():
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=2)
    b = np.stack([D.MT_apply(m, x, r) for r in R])        # b = M^T R (Phi = A^T R)
    Mx = D.fermion_matrix(m, x)
    kappa = np.linalg.cond(Mx.T @ Mx)
    vref = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    tol = 1e-13
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        bt = torch.tensor(b, device=DEV)
        v = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, v, tol=tol, prec=hg.HOL_F64)
        vg = v.cpu().numpy()
    for k in range(2):
        assert res[k] < tol
        assert D.rel_residual(m, x, b[k], vg[k]) < 2 * tol
        assert np.linalg.norm(vg[k] - vref[k]) / np.linalg.norm(vref[k]) < 2 * kappa * tol
        # v = M^{-1} R (Sec. II D)
        assert _rel(D.M_apply(m, x, vg[k]), R[k]) < 1e-9


@pytest.mark.parametrize("check_every", [1, 7, 25])
def test_cg_mixed_tiny(check_every):
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=2)
    b = np.stack([D.MT_apply(m, x, r) for r in R])
    vref = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    Mx = D.fermion_matrix(m, x)
    kappa = np.linalg.cond(Mx.T @ Mx)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        bt = torch.tensor(b, device=DEV)
        v = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, v, tol=1e-8, prec=hg.HOL_F32, reliable_every=20,
                                check_every=check_every)
        vg = v.cpu().numpy()
    for k in range(2):
        assert res[k] < 1e-8
        assert D.rel_residual(m, x, b[k], vg[k]) < 1e-8
        assert np.linalg.norm(vg[k] - vref[k]) / np.linalg.norm(vref[k]) < kappa * 1e-8


def test_cg_big32_mixed_and_fp64_certified_by_oracle():
    """The benchmark solve: 16 right-hand sides b = M^T R at L=32, Ltau=200,
    mixed precision to 1e-8 and FP64 to 1e-8; residuals recomputed by the
    matrix-free oracle; the two solutions agree to the conditioning bound."""
    w = hi.WORKLOADS["big32"]
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, w.n_rhs, seed=2)
    with _ctx(w, w.n_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        Rt = torch.tensor(R, device=DEV)
        bt = torch.empty_like(Rt)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rt, bt)          # b = M^T R on the GPU
        b = bt.cpu().numpy()
        assert _rel(b[0], MF.MT_apply(w, x, R[0])) < 1e-13
        vm = torch.empty_like(bt)
        its_m, res_m = ctx.cg_solve(bt, vm, tol=1e-8, prec=hg.HOL_F32, reliable_every=50)
        v64 = torch.empty_like(bt)
        its_d, res_d = ctx.cg_solve(bt, v64, tol=1e-8, prec=hg.HOL_F64)
        vm, v64 = vm.cpu().numpy(), v64.cpu().numpy()
    for k in range(w.n_rhs):
        assert res_m[k] < 1e-8 and res_d[k] < 1e-8
        assert MF.rel_residual(w, x, b[k], vm[k]) < 1.01e-8
        assert MF.rel_residual(w, x, b[k], v64[k]) < 1.01e-8
        # v = M^{-1} R: |M v - R| / |R| <= |M^{-T}| |b - M^T M v| / |R| is small
        assert np.linalg.norm(MF.M_apply(w, x, vm[k]) - R[k]) / np.linalg.norm(R[k]) < 1e-4


def test_cg_zero_rhs_and_errors():
    w = hi.WORKLOADS["tiny"]
    x = hi.phonon_field(w)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        b = torch.zeros(2, w.Ltau, w.N, device=DEV, dtype=torch.float64)
        b[1] = 1.0
        v = torch.empty_like(b)
        its, res = ctx.cg_solve(b, v, tol=1e-10)
        assert res[0] == 0.0 and float(v[0].abs().max()) == 0.0 and res[1] < 1e-10
        with pytest.raises(hg.HolError) as e:
            ctx.cg_solve(b, v, tol=1e-12, max_iter=1)
        assert e.value.code == hg._abi.HOL_ENOTCONV
        with pytest.raises(hg.HolError):
            ctx.cg_solve(b, b, tol=1e-10)              # aliasing refused
        bad = torch.zeros(3, w.Ltau, w.N, device=DEV, dtype=torch.float64)
        with pytest.raises(hg.HolError):
            ctx.cg_solve(bad, torch.empty_like(bad))  # n_rhs > max_rhs


@pytest.mark.parametrize("L,T", [(32, 40), (12, 20)])
def test_autotuner_choice_keeps_results(L, T):
    """hol_tune picks a launch shape; the fused M^T M and a mixed solve stay
    correct with it."""
    w, x = _field(L, T, seed=17)
    v = hi.gaussian_vectors(w, 3, seed=18)
    ref = np.stack([MF.MTM_apply(w, x, a) for a in v])
    with _ctx(w, 3) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        choice = ctx.tune(3)
        assert T % choice["slices_per_group"] == 0 and choice["ms"] > 0
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        out = torch.empty_like(vt)
        ctx.fermion_matvec(hg.HOL_OP_MTM, vt, out)
        assert _rel(out.cpu().double().numpy(), ref) < 3e-6
        bt = torch.tensor(v, device=DEV)
        sol = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, sol, tol=1e-8, prec=hg.HOL_F32)
        assert np.all(res < 1e-8)
        assert max(MF.rel_residual(w, x, v[k], sol.cpu().numpy()[k]) for k in range(3)) < 1.01e-8


LAYOUT_CASES = [(32, 40, 2), (32, 30, 5), (16, 30, 3), (8, 24, 1), (24, 12, 4)]


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("L,T,K", LAYOUT_CASES)
def test_fused_mtm_every_layout(layout, L, T, K):
    """Each register layout of the fused FP32 M^T M (scalar, float4, float4
    with a two- or three-slice prefetch ring, streaming float4, split float4
    over 2 or 4 warps, one slice per warp with the halos in shared memory)
    and each slice grouping gives the oracle's M^T M, and a masked mixed
    solve (right-hand sides of different scale converge at different
    iterations) stays certified."""
    if layout in (4, 5, 7) and L != 32:
        pytest.skip("split and one-slice-per-warp layouts are for L = 32")
    w, x = _field(L, T, seed=21)
    nr = 5
    v = hi.gaussian_vectors(w, nr, seed=22) * np.array([1.0, 1e-3, 1e3, 1.0, 1e-6])[:, None, None]
    ref = np.stack([MF.MTM_apply(w, x, a) for a in v])
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("slices_per_group", K)
        ctx.set_option("layout", layout)
        if L % 8 == 0:
            ctx.set_option("fused_cg", 0)              # the solve below runs this layout's kernel
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        out = torch.empty_like(vt)
        ctx.fermion_matvec(hg.HOL_OP_MTM, vt, out)
        got = out.cpu().double().numpy()
        for k in range(nr):
            assert _rel(got[k], ref[k]) < 3e-6
        bt = torch.tensor(v, device=DEV)
        sol = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, sol, tol=1e-8, prec=hg.HOL_F32, reliable_every=30)
        s = sol.cpu().numpy()
    assert np.all(res < 1e-8)
    assert max(MF.rel_residual(w, x, v[k], s[k]) for k in range(nr)) < 1.01e-8


@pytest.mark.parametrize("L,T", [(16, 40), (32, 20)])
def test_fp64_operators_do_not_depend_on_the_slice_grouping(L, T):
    """The FP64 M and M^T launches without partial sums pick their own slice
    grouping (as many warps as fit one resident wave); every element is the
    same arithmetic whatever the grouping, so the results are bitwise those
    of every slices_per_group and of the context-free static operator, and
    within 1e-13 of the oracle."""
    w, x = _field(L, T, seed=28)
    nr = 3
    v = hi.gaussian_vectors(w, nr, seed=29)
    vt = torch.tensor(v, device=DEV)
    got = {}
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        for k in (1, 2, 4, 5):
            ctx.set_option("slices_per_group", k)
            for op in (hg.HOL_OP_M, hg.HOL_OP_MT):
                out = torch.full_like(vt, float("nan"))
                ctx.fermion_matvec(op, vt, out)
                got[(k, op)] = out.cpu().numpy()
    for op in (hg.HOL_OP_M, hg.HOL_OP_MT):
        for k in (2, 4, 5):
            assert np.array_equal(got[(k, op)], got[(1, op)])
        st = torch.full_like(vt, float("nan"))
        hg.fermion_matvec_static(hg.hol_params(L=L, Ltau=T, dtau=w.dtau, t=w.t, mu=w.mu,
                                               alpha=w.alpha, omega0=w.omega0, max_rhs=nr),
                                 torch.tensor(x, device=DEV), op, vt, st, nr)
        assert np.array_equal(st.cpu().numpy(), got[(1, op)])
    ref_m = np.stack([MF.M_apply(w, x, a) for a in v])
    ref_mt = np.stack([MF.MT_apply(w, x, a) for a in v])
    assert _rel(got[(1, hg.HOL_OP_M)], ref_m) < 1e-13
    assert _rel(got[(1, hg.HOL_OP_MT)], ref_mt) < 1e-13


UNEVEN_CASES = [(12, 20, 2), (12, 8, 8), (20, 10, 5), (28, 24, 4), (28, 30, 3)]


@pytest.mark.parametrize("layout", [2, 6])
@pytest.mark.parametrize("L,T,K", UNEVEN_CASES)
def test_fused_mtm_uneven_row_chunks(layout, L, T, K):
    """L % 8 == 4: the float4 ring kernels hold row chunks of L/4 + 1 and
    L/4 - 1 rows (the y-bond at each chunk edge crosses lanes, the two unused
    registers of a short chunk are never loaded, stored or summed). The fused
    M^T M matches the oracle on right-hand sides of very different scale, and
    the masked mixed solve through the same kernel is certified."""
    w, x = _field(L, T, seed=24)
    nr = 5
    v = hi.gaussian_vectors(w, nr, seed=25) * np.array([1.0, 1e-3, 1e3, 1.0, 1e-6])[:, None, None]
    ref = np.stack([MF.MTM_apply(w, x, a) for a in v])
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("slices_per_group", K)
        ctx.set_option("layout", layout)
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        out = torch.full_like(vt, float("nan"))
        ctx.fermion_matvec(hg.HOL_OP_MTM, vt, out)
        got = out.cpu().double().numpy()
        for k in range(nr):
            assert _rel(got[k], ref[k]) < 3e-6
        bt = torch.tensor(v, device=DEV)
        sol = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, sol, tol=1e-8, prec=hg.HOL_F32, reliable_every=30)
        s = sol.cpu().numpy()
    assert np.all(res < 1e-8)
    assert max(MF.rel_residual(w, x, v[k], s[k]) for k in range(nr)) < 1.01e-8


def test_uneven_row_chunks_full_size_and_layout_limits():
    """The measurement lattice (L = 28, Ltau = 120) with 64 right-hand sides in
    the three-slice ring layout: every right-hand side matches the oracle.
    Layouts 1 and 3 (equal chunks only) are refused for L % 8 == 4; the ring
    layouts are refused where L % 4 != 0."""
    w = hi.Workload("chain28", L=28, Ltau=120, omega0=1.0, alpha=1.0, seed=1047)
    x = hi.phonon_field(w)
    nr = 64
    v = hi.gaussian_vectors(w, nr, seed=26)
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("layout", 6)
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        out = torch.full_like(vt, float("nan"))
        ctx.fermion_matvec(hg.HOL_OP_MTM, vt, out)
        got = out.cpu().double().numpy()
        for lay in (1, 3):
            with pytest.raises(hg.HolError):
                ctx.set_option("layout", lay)
        assert ctx.get_option("layout") == 6
    for k in (0, 1, 31, 62, 63):
        assert _rel(got[k], MF.MTM_apply(w, x, v[k])) < 3e-6
    w6 = hi.Workload("l6", L=6, Ltau=8, seed=27)
    with _ctx(w6, 1) as ctx:
        for lay in (2, 6):
            with pytest.raises(hg.HolError):
                ctx.set_option("layout", lay)


@pytest.mark.parametrize("layout,K", [(3, 1), (3, 2), (4, 2), (5, 4), (6, 4), (2, 8), (7, 1),
                                      (7, 4), (7, 5), (7, 8)])
def test_vector_layouts_full_size(layout, K):
    """The streaming layout (resident warps walk several of the 3200 or 1600
    units each) and the split layouts at L=32, Ltau=200 with 16 right-hand
    sides: the fused M^T M matches the oracle on every right-hand side."""
    w = hi.WORKLOADS["big32"]
    x = hi.phonon_field(w)
    v = hi.gaussian_vectors(w, w.n_rhs, seed=23)
    with _ctx(w, w.n_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("slices_per_group", K)
        ctx.set_option("layout", layout)
        vt = torch.tensor(v, device=DEV, dtype=torch.float32)
        out = torch.empty_like(vt)
        ctx.fermion_matvec(hg.HOL_OP_MTM, vt, out)
        got = out.cpu().double().numpy()
    for k in range(w.n_rhs):
        assert _rel(got[k], MF.MTM_apply(w, x, v[k])) < 3e-6


MERGED_CASES = [(8, 24, 1, 7, 20), (16, 30, 3, 10, 50), (24, 12, 4, 3, 9), (32, 40, 2, 10, 50),
                (32, 30, 5, 1, 5), (16, 8, 2, 4, 1000)]


@pytest.mark.parametrize("solver", ["merged_cg", "fused_cg"])
@pytest.mark.parametrize("L,T,K,check_every,reliable_every", MERGED_CASES)
def test_merged_cg_certified(L, T, K, check_every, reliable_every, solver):
    """The one-kernel-per-iteration mixed CG loops (merged: Chronopoulos-Gear
    recurrences with deferred x updates; fused: the vector update folded into
    the next operator pass, beta from the expansion of |r - alpha q|^2), with
    restarts after reliable updates, reach the certified residual on
    right-hand sides of very different scale (they leave the active set at
    different chunks), in about as many iterations as the two-kernel
    solver."""
    w, x = _field(L, T, seed=31)
    nr = 5
    v = hi.gaussian_vectors(w, nr, seed=32) * np.array([1.0, 1e-3, 1e3, 1.0, 1e-6])[:, None, None]
    with _ctx(w, nr) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("slices_per_group", K)
        ctx.set_option("fused_cg", 0)                  # reference: the two-kernel iteration
        bt = torch.tensor(v, device=DEV)
        ref = torch.empty_like(bt)
        its0, res0 = ctx.cg_solve(bt, ref, tol=1e-8, prec=hg.HOL_F32,
                                  reliable_every=reliable_every, check_every=check_every)
        ctx.set_option(solver, 1)
        sol = torch.empty_like(bt)
        its1, res1 = ctx.cg_solve(bt, sol, tol=1e-8, prec=hg.HOL_F32,
                                  reliable_every=reliable_every, check_every=check_every)
        s = sol.cpu().numpy()
    assert np.all(res1 < 1e-8)
    for k in range(nr):
        assert MF.rel_residual(w, x, v[k], s[k]) < 1.01e-8
    assert np.all(np.asarray(its1) <= 1.5 * np.asarray(its0) + 2 * check_every + 10), (its0, its1)


@pytest.mark.parametrize("solver", ["merged_cg", "fused_cg"])
def test_merged_cg_big32_certified_by_oracle(solver):
    """The benchmark solve with the merged or fused kernel: 16 right-hand
    sides b = M^T R at L=32, Ltau=200 to 1e-8, residuals recomputed by the
    oracle."""
    w = hi.WORKLOADS["big32"]
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, w.n_rhs, seed=2)
    with _ctx(w, w.n_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.set_option("fused_cg", 0)
        ctx.set_option(solver, 1)
        ctx.tune(w.n_rhs)
        Rt = torch.tensor(R, device=DEV)
        bt = torch.empty_like(Rt)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rt, bt)
        b = bt.cpu().numpy()
        vm = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, vm, tol=1e-8, prec=hg.HOL_F32, reliable_every=50,
                                check_every=10)
        vm = vm.cpu().numpy()
    for k in range(w.n_rhs):
        assert res[k] < 1e-8
        assert MF.rel_residual(w, x, b[k], vm[k]) < 1.01e-8


@pytest.mark.parametrize("solver", ["merged_cg", "fused_cg"])
def test_merged_cg_option_rules(solver):
    w, x = _field(12, 10)
    with _ctx(w, 2) as ctx:
        with pytest.raises(hg.HolError):
            ctx.set_option(solver, 1)                  # needs L % 8 == 0
    w, x = _field(8, 10)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        assert ctx.get_option("fused_cg") == 0         # the two-kernel iteration by default
        ctx.set_option("fused_cg", 0)
        ctx.set_option(solver, 1)
        assert ctx.get_option(solver) == 1
        # FP64 and preconditioned solves keep the two-kernel loop
        bt = torch.tensor(hi.gaussian_vectors(w, 2, seed=3), device=DEV)
        sol = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, sol, tol=1e-10, prec=hg.HOL_F64)
        assert np.all(res < 1e-10)
        # the autotuner times the iteration kernel; the tuned solve stays certified
        choice = ctx.tune(2)
        assert w.Ltau % choice["slices_per_group"] == 0
        assert ctx.get_option("slices_per_group") == choice["slices_per_group"]
        its, res = ctx.cg_solve(bt, sol, tol=1e-8, prec=hg.HOL_F32)
        assert np.all(res < 1e-8)
        v = bt.cpu().numpy()
        assert max(MF.rel_residual(w, x, v[k], sol.cpu().numpy()[k]) for k in range(2)) < 1.01e-8


def test_invalid_shapes_rejected():
    for L, T in ((3, 8), (34, 8), (8, 7), (2, 8)):
        with pytest.raises(hg.HolError):
            hg.Context(L=L, Ltau=T)


def test_phi_and_rhs_vs_dense():
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=5)
    Phi_ref = D.phi_from_R(m, x, R)
    x2 = x + 0.3
    b_ref = D.b_from_phi(m, x2, Phi_ref)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        Phi = torch.empty(2, w.Ltau, w.N, device=DEV, dtype=torch.float64)
        ctx.pseudofermion_phi(torch.tensor(R, device=DEV), Phi)
        assert _rel(Phi.cpu().numpy(), Phi_ref) < 1e-13
        ctx.set_field(torch.tensor(x2, device=DEV))
        b = torch.empty_like(Phi)
        ctx.phi_to_rhs(Phi, b)
        assert _rel(b.cpu().numpy(), b_ref) < 1e-13


@pytest.mark.parametrize("L,T", [(4, 40), (6, 10), (8, 12)])
def test_force_vs_dense_definition(L, T):
    w, x = _field(L, T, seed=13)
    m = D.model_of(w)
    Phi = hi.gaussian_vectors(w, 2, seed=14)
    b = D.b_from_phi(m, x, Phi)
    v = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    F_ref = D.dS_dx(m, x, Phi)
    SF_ref = D.S_F(m, x, Phi)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        F = torch.empty(w.Ltau, w.N, device=DEV, dtype=torch.float64)
        SF = torch.empty(1, device=DEV, dtype=torch.float64)
        ctx.force(torch.tensor(v, device=DEV), torch.tensor(b, device=DEV), F, True, SF)
        assert _rel(F.cpu().numpy(), F_ref) < 1e-12
        assert abs(float(SF) - SF_ref) < 1e-11 * abs(SF_ref)
        Fb = torch.empty_like(F)
        ctx.force(torch.tensor(v, device=DEV), torch.tensor(b, device=DEV), Fb, False)
        assert _rel(Fb.cpu().numpy(), D.dSF_dx(m, x, Phi)) < 1e-12


@pytest.mark.parametrize("L,T,n_pf", [(8, 12, 0), (8, 12, 1), (8, 12, 2), (6, 10, 3),
                                      (8, 12, 7), (10, 6, 9), (8, 12, 16)])
def test_force_many_pseudofermions(L, T, n_pf):
    """The pseudofermions are split into groups of blocks whose partial
    forces are summed in a fixed order: same force and S_F as the dense
    definition for one to sixteen of them, including lattice sides that
    leave idle lanes in a warp (n_pf = 0 leaves the bosonic force alone)."""
    w, x = _field(L, T, seed=15)
    m = D.model_of(w)
    Phi = hi.gaussian_vectors(w, max(n_pf, 1), seed=16)[:n_pf]
    with _ctx(w, 16) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        F = torch.empty(w.Ltau, w.N, device=DEV, dtype=torch.float64)
        SF = torch.empty(1, device=DEV, dtype=torch.float64)
        if n_pf == 0:
            import ctypes
            z = torch.zeros(1, w.Ltau, w.N, device=DEV, dtype=torch.float64)
            p = ctypes.c_void_p
            rc = hg._abi.load().force(ctx._h, p(z.data_ptr()), p(z.data_ptr()), 0,
                                      p(F.data_ptr()), 1, p(SF.data_ptr()),
                                      p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0
            torch.cuda.synchronize()
            assert _rel(F.cpu().numpy(), D.dSB_dx(m, x)) < 1e-13
            assert float(SF) == 0.0
            return
        b = D.b_from_phi(m, x, Phi)
        v = np.stack([D.solve_MTM(m, x, bb) for bb in b])
        ctx.force(torch.tensor(v, device=DEV), torch.tensor(b, device=DEV), F, True, SF)
        assert _rel(F.cpu().numpy(), D.dS_dx(m, x, Phi)) < 1e-12
        assert abs(float(SF) - D.S_F(m, x, Phi)) < 1e-11 * abs(D.S_F(m, x, Phi))


def test_force_full_size_grad24_vs_matrix_free():
    w = hi.WORKLOADS["grad24"]
    x = hi.phonon_field(w)
    v = hi.gaussian_vectors(w, 2, seed=30)
    b = hi.gaussian_vectors(w, 2, seed=31)
    ref = MF.force_fermion(w, x, v[0], b[0]) + MF.force_fermion(w, x, v[1], b[1]) \
        + MF.force_boson(w, x)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        F = torch.empty(w.Ltau, w.N, device=DEV, dtype=torch.float64)
        SF = torch.empty(1, device=DEV, dtype=torch.float64)
        ctx.force(torch.tensor(v, device=DEV), torch.tensor(b, device=DEV), F, True, SF)
        assert _rel(F.cpu().numpy(), ref) < 1e-12
        assert abs(float(SF) - 0.5 * np.sum(b * v)) < 1e-10 * np.abs(b * v).sum()


def test_end_to_end_force_matches_oracle_tiny():
    """x -> Phi (GPU) -> b -> CG (GPU, FP64) -> force (GPU) against the dense
    oracle's Eq. (dSF_dx) at the same Phi."""
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x0 = hi.phonon_field(w)
    x = x0 + 0.05 * hi.gaussian_vectors(w, 1, seed=40)[0]
    R = hi.gaussian_vectors(w, 2, seed=41)
    Phi_ref = D.phi_from_R(m, x0, R)
    F_ref = D.dS_dx(m, x, Phi_ref)
    with _ctx(w, 2) as ctx:
        ctx.set_field(torch.tensor(x0, device=DEV))
        Phi = torch.empty(2, w.Ltau, w.N, device=DEV, dtype=torch.float64)
        ctx.pseudofermion_phi(torch.tensor(R, device=DEV), Phi)
        ctx.set_field(torch.tensor(x, device=DEV))
        b = torch.empty_like(Phi)
        ctx.phi_to_rhs(Phi, b)
        v = torch.empty_like(b)
        ctx.cg_solve(b, v, tol=1e-13)
        F = torch.empty(w.Ltau, w.N, device=DEV, dtype=torch.float64)
        ctx.force(v, b, F, True)
        assert _rel(F.cpu().numpy(), F_ref) < 1e-9


@pytest.mark.parametrize("shape", ["tuned", (2, 4, 1), (2, 4, 2), (6, 4, 1), (0, 4, 1),
                                   (7, 4, 1), (7, 8, 1)])
def test_big32_step_in_the_benchmark_launch_configuration(shape):
    """The timed step of bench.py at full size (L=32, Ltau=200, 16 rhs), in
    the launch shapes it runs (the autotuner's pick, and the shapes the
    profiles were taken with): b = M^T R, mixed CG to 1e-8 with reliable
    updates every 50 and polls every 10, then the force of the 16 solutions.
    Every residual is recomputed by the matrix-free oracle, and the force is
    compared with the oracle's on the same (v, b)."""
    w = hi.WORKLOADS["big32"]
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, w.n_rhs, seed=2)
    with _ctx(w, w.n_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        if shape == "tuned":
            ctx.tune(w.n_rhs)
        else:
            layout, k, wpb = shape
            ctx.set_option("layout", layout)
            ctx.set_option("slices_per_group", k)
            ctx.set_option("warps_per_block", wpb)
        Rt = torch.tensor(R, device=DEV)
        bt = torch.empty_like(Rt)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rt, bt)
        vt = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, vt, tol=1e-8, prec=hg.HOL_F32, reliable_every=50,
                                check_every=10, max_iter=50000)
        F = torch.empty(w.Ltau, w.N, device=DEV, dtype=torch.float64)
        SF = torch.empty(1, device=DEV, dtype=torch.float64)
        ctx.force(vt, bt, F, True, SF)
        b, v, Fg = bt.cpu().numpy(), vt.cpu().numpy(), F.cpu().numpy()
    Fref = MF.force_boson(w, x)
    for k in range(w.n_rhs):
        assert res[k] < 1e-8
        assert MF.rel_residual(w, x, b[k], v[k]) < 1.01e-8
        Fref = Fref + MF.force_fermion(w, x, v[k], b[k])
    assert _rel(Fg, Fref) < 1e-12
    sf = 0.5 * sum(float(np.dot(b[k].ravel(), v[k].ravel())) for k in range(w.n_rhs))
    assert abs(float(SF) - sf) < 1e-11 * abs(sf)


def test_big32_preconditioned_solve_certified():
    """The preconditioned solve of the benchmark's comparison line at full
    size (register KPM, default shapes): certified by the matrix-free oracle."""
    w = hi.WORKLOADS["big32"]
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 4, seed=3)
    with _ctx(w, 4) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        Rt = torch.tensor(R, device=DEV)
        bt = torch.empty_like(Rt)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rt, bt)
        vt = torch.empty_like(bt)
        its, res = ctx.cg_solve(bt, vt, tol=1e-8, prec=hg.HOL_F32, precond=True,
                                max_iter=50000)
        b, v = bt.cpu().numpy(), vt.cpu().numpy()
    for k in range(4):
        assert res[k] < 1e-8
        assert MF.rel_residual(w, x, b[k], v[k]) < 1.01e-8


def test_force_action_only_mode():
    """force with a null dSdx computes the action alone: the same S_F as the
    full call, and HOL_EINVAL when both outputs are null."""
    import ctypes
    w, x = _field(8, 12, seed=17)
    m = D.model_of(w)
    Phi = hi.gaussian_vectors(w, 3, seed=18)
    b = D.b_from_phi(m, x, Phi)
    v = np.stack([D.solve_MTM(m, x, bb) for bb in b])
    with _ctx(w, 3) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        vt, bt = torch.tensor(v, device=DEV), torch.tensor(b, device=DEV)
        SF = torch.empty(1, device=DEV, dtype=torch.float64)
        ctx.force(vt, bt, None, False, SF)
        assert abs(float(SF) - D.S_F(m, x, Phi)) < 1e-11 * abs(D.S_F(m, x, Phi))
        p = ctypes.c_void_p
        rc = hg._abi.load().force(ctx._h, p(vt.data_ptr()), p(bt.data_ptr()), 3, None, 0, None,
                                  p(torch.cuda.current_stream().cuda_stream))
        assert rc == hg._abi.HOL_EINVAL
