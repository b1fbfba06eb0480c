"""GPU parity of the FFT-accelerated stochastic measurements (Sec. V) against
the oracle's direct O(N^2) sums. Marked gpu.

Tolerance 1e-10 of max|ref|: the probes are solved with FP64 CG to 1e-13
(error ~ kappa * 1e-13 ~ 1e-10 relative at these sizes) and the FFT adds
O(log n) epsilon.
"""
import numpy as np
import pytest
import scipy.linalg
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


def _run(w, x, xi, four_point=0, max_rhs=4):
    with hg.Context.from_workload(w, max_rhs=max_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        xt = torch.tensor(xi, device=DEV)
        Gxi = torch.empty_like(xt)
        G2 = torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
        G4 = torch.empty(3, 2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV) \
            if four_point else None
        its = ctx.stochastic_measure(xt, Gxi, G2, G4, four_point, tol=1e-13)
        torch.cuda.synchronize()
        return (Gxi.cpu().numpy(), G2.cpu().numpy(),
                None if G4 is None else G4.cpu().numpy(), its)


@pytest.mark.parametrize("L,T,nrv", [(4, 8, 3), (6, 12, 5), (4, 10, 2)])
def test_two_and_four_point_vs_direct_sums(L, T, nrv):
    w = hi.Workload("g", L=L, Ltau=T, alpha=1.1, mu=0.0)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    xi = hi.z2_vectors(w, nrv, seed=3)
    Gxi, G2, G4, its = _run(w, x, xi, four_point=7)
    G = D.green_matrix(m, x)
    Gref = np.array([(G @ v.reshape(-1)).reshape(T, -1) for v in xi])
    assert _rel(Gxi, Gref) < 1e-10
    ref2 = D.green_average(m, x, xi)
    assert _rel(G2, ref2) < 1e-10
    ref4 = D.four_point_pairs(m, x, xi)
    for k in range(3):
        assert _rel(G4[k], ref4[k]) < 1e-10, k


def test_complete_hadamard_probes_give_exact_average():
    """The rows of a Hadamard matrix are +-1 vectors with sum_k h_k h_k^T = n I,
    so the probe average equals the exact space-time average of G^ext."""
    w = hi.Workload("h", L=4, Ltau=4, alpha=1.0)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    H = scipy.linalg.hadamard(w.n).astype(float).reshape(w.n, w.Ltau, w.N)
    _, G2, _, _ = _run(w, x, H, max_rhs=16)
    assert _rel(G2, D.green_average_exact(m, x)) < 1e-10


def test_chain_size_two_point_and_type2():
    """An L=8, Ltau=20 chain-sized case with 12 probes (two solve batches),
    the 2-point function and the type-2 Wick product."""
    w = hi.Workload("c", L=8, Ltau=20, alpha=1.0)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    xi = hi.z2_vectors(w, 12, seed=5)
    Gxi, G2, G4, _ = _run(w, x, xi, four_point=2, max_rhs=8)
    G = D.green_matrix(m, x)
    Gref = np.array([(G @ v.reshape(-1)).reshape(w.Ltau, -1) for v in xi])
    assert _rel(G2, D.green_average(m, x, xi, Gref)) < 1e-10
    assert _rel(G4[1], D.four_point_pairs(m, x, xi, Gref)[1]) < 1e-10
    assert float(np.abs(G4[0]).max()) == 0.0 and float(np.abs(G4[2]).max()) == 0.0


@pytest.mark.parametrize("L,T,nrv", [(4, 10, 6), (6, 12, 4)])
def test_observables_vs_oracle(L, T, nrv):
    """<n>, C(r), S_cdw and P_s contracted on the GPU from its own 2-point
    function and Wick products equal the oracle's contraction of the same
    arrays, and of the oracle's direct-sum estimates with the same probes."""
    w = hi.Workload("o", L=L, Ltau=T, alpha=1.1, mu=0.05)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    xi = hi.z2_vectors(w, nrv, seed=5)
    with hg.Context.from_workload(w, max_rhs=4) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        xt = torch.tensor(xi, device=DEV)
        Gxi = torch.empty_like(xt)
        G2 = torch.empty(2 * T, L, L, dtype=torch.float64, device=DEV)
        G4 = torch.empty(3, 2 * T, L, L, dtype=torch.float64, device=DEV)
        ctx.stochastic_measure(xt, Gxi, G2, G4, 7, tol=1e-13)
        C = torch.empty(L, L, dtype=torch.float64, device=DEV)
        obs = ctx.measure_observables(G2, G4, C)
        Cg = C.cpu().numpy()
        g2, g4 = G2.cpu().numpy(), G4.cpu().numpy()
    same = D.observables_from_estimates(m, g2, g4)
    for k in ("density", "S_cdw", "P_s"):
        assert abs(obs[k] - same[k]) < 1e-12 * max(1.0, abs(same[k]))
    assert np.abs(Cg - same["C"]).max() < 1e-12 * np.abs(same["C"]).max()
    ref = D.observables_from_estimates(m, D.green_average(m, x, xi), D.four_point_pairs(m, x, xi))
    for k in ("density", "S_cdw", "P_s"):
        assert abs(obs[k] - ref[k]) < 1e-9 * max(1.0, abs(ref[k]))
    assert np.abs(Cg - ref["C"]).max() < 1e-9 * np.abs(ref["C"]).max()


# ---------------------------------------------------------------------------
# The batching workload's chain shapes (L = 20, 24, 28; Ltau = 120)
# ---------------------------------------------------------------------------
def _deltas(L, T):
    """About 70 offsets (dl, dy, dx): zero, the axes, the diagonal, the
    half-lattice points and a generic one, at tau offsets 0, 1, 2, 5, T/2,
    the antiperiodic mirror T - 1, T, T + 1 and 2T - 1."""
    dls = [0, 1, 2, 5, T // 2, T - 1, T, T + 1, 2 * T - 1]
    sp = [(0, 0), (0, 1), (1, 0), (1, 1), (0, L // 2), (L // 2, L // 2), (L - 1, 0), (3, L - 2)]
    return [(dl, dy, dx) for dl in dls for dy, dx in sp]


def _oracle_solutions(w, x, xi, tol=1e-12):
    """G xi = (M^T M)^{-1} M^T xi by the matrix-free oracle's textbook CG."""
    out = []
    for v in xi:
        g, _, res = MF.cg(w, x, MF.MT_apply(w, x, v), tol=tol, max_iter=100000)
        assert res < tol
        out.append(g)
    return np.array(out)


def _check_at(w, xi, Gg, Go, G2, G4, deltas, types=(0, 1, 2)):
    """GPU arrays against the oracle's direct sums (with the oracle's own
    solutions) at the offsets. The two sides' G xi differ by the two solves'
    tolerances; with delta = max|dGxi| / max|Gxi| and |xi| = 1 the 2-point
    average moves by at most delta max|Gxi| (each term is xi . Gxi, summed
    over 2 N T sites and divided by 2 N T), and each 4-point product (two
    G xi factors) by at most (2 delta + delta^2) max|Gxi|^2; 1e-12 covers the
    transforms' rounding."""
    m = D.model_of(w)
    gmax = float(np.abs(Go).max())
    delta = float(np.abs(Gg - Go).max()) / gmax
    assert delta < 1e-6, delta
    ref2 = D.green_average_at(m, xi, Go, deltas)
    got2 = np.array([G2[d] for d in deltas])
    assert np.abs(got2 - ref2).max() <= delta * gmax + 1e-12, (np.abs(got2 - ref2).max(), delta)
    if G4 is None:
        return
    ref4 = D.four_point_pairs_at(m, xi, Go, deltas)
    bound4 = (2 * delta + delta * delta) * gmax * gmax + 1e-12
    for k in types:
        got = np.array([G4[k][d] for d in deltas])
        assert np.abs(got - ref4[k]).max() <= bound4, (k, np.abs(got - ref4[k]).max(), bound4)


def _measure(w, x, xi, max_rhs, four_point, prec, tol):
    with hg.Context.from_workload(w, max_rhs=max_rhs) as ctx:
        ctx.set_field(torch.tensor(x, device=DEV))
        ctx.tune(max_rhs)                     # the launch shapes the benchmark legs pick
        xt = torch.tensor(xi, device=DEV)
        Gxi = torch.empty_like(xt)
        G2 = torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
        G4 = torch.empty(3, 2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV) \
            if four_point else None
        ctx.stochastic_measure(xt, Gxi, G2, G4, four_point, tol=tol, prec=prec)
        torch.cuda.synchronize()
        return (Gxi.cpu().numpy(), G2.cpu().numpy(),
                None if G4 is None else G4.cpu().numpy())


def test_chain28_block_of_64_probes_and_wick_products():
    """The L=28, Ltau=120 chain of the batching workload (radix-7 spatial
    transform, Ltau = 120 tau transform): 64 Z2 probes solved as one
    64-right-hand-side block in mixed precision (the benchmark's path), the
    2-point function at ~70 offsets against the oracle's direct sums with
    the oracle's own solutions; then the first 8 probes with all three Wick
    products (FP64 solves). Every GPU solution is also certified by the
    oracle's residual."""
    w = hi.chain_workloads(8, 120)[-1]
    assert w.L == 28
    x = hi.phonon_field(w)
    xi = hi.z2_vectors(w, 64, seed=w.seed + 3)
    Go = _oracle_solutions(w, x, xi)
    deltas = _deltas(w.L, w.Ltau)
    Gg, G2, _ = _measure(w, x, xi, 64, 0, hg.HOL_F32, 1e-11)
    for k in (0, 31, 63):
        b = MF.MT_apply(w, x, xi[k])
        assert MF.rel_residual(w, x, b, Gg[k]) < 1.01e-11
    _check_at(w, xi, Gg, Go, G2, None, deltas)
    Gg8, G2_8, G4_8 = _measure(w, x, xi[:8], 8, 7, hg.HOL_F64, 1e-12)
    _check_at(w, xi[:8], Gg8, Go[:8], G2_8, G4_8, deltas)


@pytest.mark.parametrize("idx,prec", [(24, hg.HOL_F64), (32, hg.HOL_F32)])
def test_chain20_24_wick_products(idx, prec):
    """L=20 and L=24 chains of the batching workload (Ltau=120), 8 probes,
    the 2-point function and all three Wick products at ~70 offsets."""
    w = hi.chain_workloads(8, 120)[idx]
    assert w.L in (20, 24)
    x = hi.phonon_field(w)
    xi = hi.z2_vectors(w, 8, seed=w.seed + 3)
    Go = _oracle_solutions(w, x, xi)
    tol = 1e-12 if prec == hg.HOL_F64 else 1e-11
    Gg, G2, G4 = _measure(w, x, xi, 8, 7, prec, tol)
    _check_at(w, xi, Gg, Go, G2, G4, _deltas(w.L, w.Ltau))
