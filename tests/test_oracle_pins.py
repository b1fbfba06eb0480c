"""Pins of the oracle against what the paper and mathematics fix (no GPU).

Each test checks oracle/dense.py or oracle/matfree.c against an independent
fact: a closed form, an exact identity, brute force on a tiny case, a library
routine reached by a different route, or a number the paper prints
(tests/golden/paper_numbers.json).
"""
import json
import os

import numpy as np
import pytest

import holstein_inputs as hi
from oracle import dense as D
from oracle import matfree as MF

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- free fermions
@pytest.mark.parametrize("L", [4, 6])
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_free_fermion_logdet_exact_kinetic(L, mu):
    """x = 0, exact kinetic: det M = prod_k (1 + e^{-beta (eps_k - mu)}) with
    eps_k = -2t(cos kx + cos ky) (Eq. (detM_alt) for free fermions)."""
    m = D.Model(L=L, Ltau=10, mu=mu, kinetic="exact")
    x = np.zeros((m.Ltau, m.N))
    ks = 2 * np.pi * np.arange(L) / L
    eps = np.array([-2 * m.t * (np.cos(kx) + np.cos(ky)) for kx in ks for ky in ks])
    ref = np.sum(np.log1p(np.exp(-m.beta * (eps - m.mu))))
    assert abs(D.logdet_M(m, x) - ref) < 1e-11


def test_checkerboard_exact_at_L4_and_second_order():
    """At L = 4 the two x-colours (and the two y-colours) commute, so the
    checkerboard product equals exp(-dtau K) exactly; at L = 8 the error is
    O(dtau^2) (halving dtau quarters it) (Sec. II D)."""
    m4 = D.Model(L=4, Ltau=4)
    ex = D.kinetic_propagator(D.Model(L=4, Ltau=4, kinetic="exact"))
    assert np.abs(D.kinetic_propagator(m4) - ex).max() < 1e-14
    errs = []
    for dt in (0.1, 0.05):
        a = D.kinetic_propagator(D.Model(L=8, Ltau=4, dtau=dt))
        b = D.kinetic_propagator(D.Model(L=8, Ltau=4, dtau=dt, kinetic="exact"))
        errs.append(np.abs(a - b).max())
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_checkerboard_factors_spectrum_and_transpose():
    """Each colour is symmetric with eigenvalues exp(+-dtau t) (N/2 each), and
    C^T = C1 C2 C3 C4."""
    m = D.Model(L=6, Ltau=4, t=1.3)
    Cs = D.checkerboard_factors(m)
    for C in Cs:
        assert np.allclose(C, C.T)
        ev = np.sort(np.linalg.eigvalsh(C))
        ref = np.sort([np.exp(-m.dtau * m.t)] * (m.N // 2) + [np.exp(m.dtau * m.t)] * (m.N // 2))
        assert np.abs(ev - ref).max() < 1e-13
    C1, C2, C3, C4 = Cs
    assert np.abs(D.kinetic_propagator(m).T - C1 @ C2 @ C3 @ C4).max() < 1e-14


def test_exact_propagator_plane_waves():
    """exp(-dtau K) acts on the plane wave e^{i k.r} as multiplication by
    exp(2 dtau t (cos kx + cos ky)) (K = -t sum over nearest-neighbour bonds)."""
    m = D.Model(L=6, Ltau=4, t=0.9, dtau=0.15, kinetic="exact")
    C = D.kinetic_propagator(m)
    L = m.L
    ix, iy = np.meshgrid(np.arange(L), np.arange(L), indexing="xy")
    for nx, ny in [(0, 0), (1, 0), (2, 3), (5, 1), (3, 3)]:
        kx, ky = 2 * np.pi * nx / L, 2 * np.pi * ny / L
        wave = np.exp(1j * (kx * ix + ky * iy)).reshape(-1)   # index ix + L*iy
        lam = np.exp(2 * m.dtau * m.t * (np.cos(kx) + np.cos(ky)))
        assert np.abs(C @ wave - lam * wave).max() < 1e-13


@pytest.mark.parametrize("kinetic", ["checkerboard", "exact"])
def test_blockwise_M_equals_dense_definition(kinetic):
    """The block-by-block M and M^T used at large lattices are the dense
    Eq. (M_def) matrix and its transpose (brute force on a small lattice)."""
    m = D.Model(L=6, Ltau=5, alpha=1.1, mu=0.2, kinetic=kinetic)
    x = rng(7).standard_normal((m.Ltau, m.N))
    v = rng(8).standard_normal((m.Ltau, m.N))
    Mx = D.fermion_matrix(m, x)
    assert np.abs(D.M_apply_blocks(m, x, v).reshape(-1) - Mx @ v.reshape(-1)).max() < 1e-13
    assert np.abs(D.MT_apply_blocks(m, x, v).reshape(-1) - Mx.T @ v.reshape(-1)).max() < 1e-13


def test_free_fermion_checkerboard_close_to_exact():
    m = D.Model(L=8, Ltau=10)
    x = np.zeros((m.Ltau, m.N))
    me = D.Model(L=8, Ltau=10, kinetic="exact")
    assert abs(D.logdet_M(m, x) - D.logdet_M(me, x)) < 0.05


# ---------------------------------------------------------------- particle-hole
@pytest.mark.parametrize("kinetic", ["exact", "checkerboard"])
def test_particle_hole_logdet(kinetic):
    """mu = 0, bipartite lattice: log det M(-x) - log det M(x) = dtau alpha sum x,
    so |det A(-x)| = |det A(x)| with det Lambda^2 = e^{dtau alpha sum x}
    (Eqs. (Z_path_orig), (Lambda_constraint))."""
    m = D.Model(L=4, Ltau=8, alpha=1.3, kinetic=kinetic)
    x = rng(1).standard_normal((m.Ltau, m.N))
    lhs = D.logdet_M(m, -x) - D.logdet_M(m, x)
    assert abs(lhs - m.dtau * m.alpha * x.sum()) < 1e-11
    s, la = np.linalg.slogdet(D.A_matrix(m, x))
    s2, la2 = np.linalg.slogdet(D.A_matrix(m, -x))
    assert abs(la - la2) < 1e-11


def test_lambda_determinant_and_inverse():
    """det Lambda^2 = exp(dtau alpha sum x) (Eq. (Lambda_constraint)) and
    Eq. (Lambda_inv) is the inverse of Eq. (Lambda_def)."""
    m = D.Model(L=4, Ltau=6, alpha=0.7)
    x = rng(2).standard_normal((m.Ltau, m.N))
    Lm, Li = D.Lambda(m, x), D.Lambda_inv(m, x)
    assert np.abs(Lm @ Li - np.eye(m.n)).max() < 1e-13
    s, ld = np.linalg.slogdet(Lm)
    assert abs(2 * ld - m.dtau * m.alpha * x.sum()) < 1e-11


# ---------------------------------------------------------------- t = 0
def test_atomic_limit_logdet():
    """t = 0: det M = prod_i (1 + exp(-dtau sum_tau (alpha x_{i,tau} - mu)))
    (single-site form of Sec. IV, Eq. (detM_alt))."""
    m = D.Model(L=4, Ltau=8, t=0.0, mu=0.2, alpha=1.1)
    x = rng(3).standard_normal((m.Ltau, m.N))
    ref = np.sum(np.log1p(np.exp(-m.dtau * np.sum(m.alpha * x - m.mu, axis=0))))
    assert abs(D.logdet_M(m, x) - ref) < 1e-12


def test_single_site_adiabatic_reflection_symmetry():
    """t = 0, mu = 0, x constant in tau: D_x = D_{-x} (App. B, Eq. (A_x)), so
    S_F(xbar, Phi) = S_F(-xbar, Phi) for any Phi."""
    m = D.Model(L=4, Ltau=6, t=0.0, alpha=1.4)
    xbar = rng(4).standard_normal(m.N)
    x = np.tile(xbar, (m.Ltau, 1))
    Phi = rng(5).standard_normal((2, m.Ltau, m.N))
    assert abs(D.S_F(m, x, Phi) - D.S_F(m, -x, Phi)) < 1e-11 * abs(D.S_F(m, x, Phi))


# ---------------------------------------------------------------- S_F at x0
def test_SF_at_sampling_point_and_solution():
    """Phi = A(x0)^T R gives S_F(x0, Phi) = |R|^2 / 2 (Sec. II D) and
    v = (M^T M)^{-1} Lambda^{-T} Phi = M^{-1} R."""
    m = D.Model(L=4, Ltau=8, alpha=1.2)
    x = rng(6).standard_normal((m.Ltau, m.N))
    R = rng(7).standard_normal((2, m.Ltau, m.N))
    Phi = D.phi_from_R(m, x, R)
    assert abs(D.S_F(m, x, Phi) - 0.5 * np.sum(R * R)) < 1e-10
    b = D.b_from_phi(m, x, Phi[0])
    assert np.abs(b - D.MT_apply(m, x, R[0])).max() < 1e-12
    v = D.solve_MTM(m, x, b)
    assert np.abs(D.M_apply(m, x, v) - R[0]).max() < 1e-12


# ---------------------------------------------------------------- forces
def test_force_matches_finite_differences():
    """dS_F/dx (Eq. (dSF_dx)) against central differences of S_F at fixed Phi."""
    m = D.Model(L=4, Ltau=8, alpha=1.2)
    g = rng(8)
    x = g.standard_normal((m.Ltau, m.N))
    Phi = D.phi_from_R(m, x + 0.3 * g.standard_normal(x.shape), g.standard_normal((2, m.Ltau, m.N)))
    F = D.dSF_dx(m, x, Phi)
    h = 1e-5
    for _ in range(12):
        tau, i = g.integers(m.Ltau), g.integers(m.N)
        xp, xm = x.copy(), x.copy()
        xp[tau, i] += h
        xm[tau, i] -= h
        fd = (D.S_F(m, xp, Phi) - D.S_F(m, xm, Phi)) / (2 * h)
        assert abs(fd - F[tau, i]) < 1e-7 * max(1.0, abs(F[tau, i]))


def test_force_structured_equals_fully_dense():
    m = D.Model(L=4, Ltau=5, alpha=0.9)
    g = rng(9)
    x = g.standard_normal((m.Ltau, m.N))
    Phi = g.standard_normal((2, m.Ltau, m.N))
    F = D.dSF_dx(m, x, Phi)
    comps = [(0, 0), (0, 7), (1, 3), (4, 15), (2, 9)]
    ref = D.dSF_dx_fully_dense(m, x, Phi, comps)
    assert np.abs(ref - np.array([F[c] for c in comps])).max() < 1e-12


@pytest.mark.parametrize("L,kinetic", [(4, "checkerboard"), (6, "exact")])
def test_force_phi_average_is_logdet_derivative(L, kinetic):
    """Phi ~ N(0, A^T A): E[dS_F,sigma/dx] = -d ln|det M|/dx - dtau alpha / 2.
    Exact (no sampling): sum over Phi_k = A^T e_k for all unit vectors e_k,
    since sum_k e_k e_k^T = I; right side by central differences of slogdet."""
    m = D.Model(L=L, Ltau=4, alpha=1.1, kinetic=kinetic)
    g = rng(10)
    x = g.standard_normal((m.Ltau, m.N))
    A = D.A_matrix(m, x)
    Phis = A.T @ np.eye(m.n)          # column k = A^T e_k
    Phis = Phis.T.reshape(m.n, m.Ltau, m.N)
    F = D.dSF_dx(m, x, Phis)          # sums over the "pseudofermions"
    h = 1e-5
    for (tau, i) in [(0, 0), (1, 5), (3, 15), (2, 8)]:
        xp, xm = x.copy(), x.copy()
        xp[tau, i] += h
        xm[tau, i] -= h
        dld = (D.logdet_M(m, xp) - D.logdet_M(m, xm)) / (2 * h)
        assert abs(F[tau, i] - (-dld - 0.5 * m.dtau * m.alpha)) < 1e-7, (tau, i)


def test_bosonic_force_finite_differences():
    m = D.Model(L=4, Ltau=12, omega0=0.7)
    x = rng(11).standard_normal((m.Ltau, m.N))
    F = D.dSB_dx(m, x)
    h = 1e-5
    for (tau, i) in [(0, 0), (11, 3), (5, 9)]:
        xp, xm = x.copy(), x.copy()
        xp[tau, i] += h
        xm[tau, i] -= h
        assert abs((D.S_B(m, xp) - D.S_B(m, xm)) / (2 * h) - F[tau, i]) < 1e-6


# ---------------------------------------------------------------- Fourier
def test_Q_fourier_equals_stencil():
    """Qx = F^{-1} Qtilde F x equals the stencil of Eq. (dSB_dx)."""
    m = D.Model(L=4, Ltau=20, omega0=0.8)
    x = rng(12).standard_normal((m.Ltau, m.N))
    assert np.abs(D.Q_apply(m, x) - D.dSB_dx(m, x)).max() < 1e-12


def test_Q_extremes_and_ratio():
    """Qtilde/dtau = omega0^2 at omega = 0 and omega0^2 + 4/dtau^2 at
    omega = Ltau/2 (Sec. III B)."""
    m = D.Model(L=4, Ltau=40, omega0=0.5)
    q = D.Q_tilde(m) / m.dtau
    assert abs(q[0] - m.omega0 ** 2) < 1e-12
    assert abs(q[m.Ltau // 2] - (m.omega0 ** 2 + 4 / m.dtau ** 2)) < 1e-9
    assert abs(q.max() / q.min() - (1 + 4 / (m.omega0 ** 2 * m.dtau ** 2))) < 1e-9


def test_fourier_acceleration_dt_ratio():
    """Paper: dt = 1e-2 with m_reg = omega0 and dt = 7.05e-4 with m_reg = inf
    give the top mode omega = Ltau/2 the same time scale."""
    gd = GOLD["dt_equal_top_mode"]
    m = D.Model(L=4, Ltau=40, omega0=gd["omega0"], dtau=gd["dtau"])
    w = m.Ltau // 2
    Om1 = np.sqrt(D.Q_tilde(m)[w] / D.mass_tilde(m, m.omega0)[w])
    Oinf = np.sqrt(D.Q_tilde(m)[w] / D.mass_tilde(m, np.inf)[w])
    dt_inf = gd["dt_mreg_omega0"] * Om1 / Oinf
    assert abs(dt_inf - gd["dt_mreg_inf"]) < 0.005e-4


def test_mass_operator_powers():
    """Mass^{1/2} Mass^{1/2} = Mass and Mass Mass^{-1} = I along tau; the mass
    is constant dtau when m_reg = inf (Sec. III B 1)."""
    m = D.Model(L=4, Ltau=16)
    p = rng(13).standard_normal((m.Ltau, m.N))
    h = D.mass_apply(m, D.mass_apply(m, p, 1.0, 0.5), 1.0, 0.5)
    assert np.abs(h - D.mass_apply(m, p, 1.0, 1.0)).max() < 1e-12
    assert np.abs(D.mass_apply(m, D.mass_apply(m, p, 1.0, -1.0), 1.0, 1.0) - p).max() < 1e-12
    assert np.abs(D.mass_apply(m, p, np.inf, 1.0) - m.dtau * p).max() < 1e-14


# ---------------------------------------------------------------- leapfrog
def test_leapfrog_reversible():
    m = D.Model(L=4, Ltau=8, alpha=1.0)
    g = rng(14)
    x = g.standard_normal((m.Ltau, m.N))
    Phi = D.phi_from_R(m, x, g.standard_normal((2, m.Ltau, m.N)))
    p = D.mass_apply(m, g.standard_normal((m.Ltau, m.N)), 1.0, 0.5)
    x1, p1 = D.leapfrog_split(m, x, p, Phi, 0.02, 4, 3, 1.0)
    x2, p2 = D.leapfrog_split(m, x1, -p1, Phi, 0.02, 4, 3, 1.0)
    assert np.abs(x2 - x).max() < 1e-11
    assert np.abs(p2 + p).max() < 1e-10


def test_leapfrog_energy_error_second_order():
    """|dH| scales as dt^2 at fixed trajectory length."""
    m = D.Model(L=4, Ltau=8, alpha=1.0)
    g = rng(15)
    x = g.standard_normal((m.Ltau, m.N))
    R = g.standard_normal((2, m.Ltau, m.N))
    Rp = g.standard_normal((m.Ltau, m.N))
    dH = []
    for dt, Nt in ((0.04, 5), (0.02, 10)):
        _, _, Hi, Hf = D.hmc_update(m, x, R, Rp, dt, Nt, 2, 1.0)
        dH.append(abs(Hf - Hi))
    assert 3.0 < dH[0] / dH[1] < 5.0


def test_harmonic_modes_without_fermions():
    """alpha = 0: S = S_B and every Fourier mode of x is a harmonic oscillator
    of frequency sqrt(Qtilde/Mass~); leapfrog follows it to O(dt^2)."""
    m = D.Model(L=4, Ltau=16, alpha=0.0, omega0=1.0)
    g = rng(16)
    x0 = g.standard_normal((m.Ltau, m.N))
    Phi = np.zeros((1, m.Ltau, m.N))
    p0 = np.zeros_like(x0)
    dt, Nt, nt = 0.01, 50, 2
    x1, _ = D.leapfrog_split(m, x0, p0, Phi, dt, Nt, nt, 1.0)
    Om = np.sqrt(D.Q_tilde(m) / D.mass_tilde(m, 1.0))
    F = D.fourier_matrix(m.Ltau)
    ref = (F.conj().T @ (np.cos(Om * dt * Nt)[:, None] * (F @ x0))).real
    assert np.abs(x1 - ref).max() < 5e-3 * np.abs(x0).max()


# ---------------------------------------------------------------- preconditioner
def test_precond_block_diagonal_in_U_basis():
    """U P U^dag is block diagonal with blocks I - e^{-i phi_omega} Bbar
    (Eqs. (Mww), (P_block))."""
    m = D.Model(L=4, Ltau=6)
    x = rng(17).standard_normal((m.Ltau, m.N))
    N, T = m.N, m.Ltau
    UU = np.kron(D.U_matrix(T), np.eye(N))
    Pt = UU @ D.precond_matrix(m, x) @ UU.conj().T
    Bb = D.Bbar(m, x)
    for w in range(T):
        for w2 in range(T):
            blk = Pt[w * N:(w + 1) * N, w2 * N:(w2 + 1) * N]
            ref = np.eye(N) - np.exp(-1j * D.phi_omega(T, w)) * Bb if w == w2 else 0.0
            assert np.abs(blk - ref).max() < 1e-13


def test_precond_exact_in_adiabatic_limit():
    """x constant in tau: P = M (Sec. VI B), so PCG with the exact-enough KPM
    inverse converges in very few iterations."""
    m = D.Model(L=4, Ltau=8)
    xc = np.tile(rng(18).standard_normal(m.N), (m.Ltau, 1))
    assert np.abs(D.precond_matrix(m, xc) - D.fermion_matrix(m, xc)).max() < 1e-15
    b = rng(19).standard_normal((m.Ltau, m.N))
    _, it_exact = D.pcg(m, xc, b, tol=1e-10, precond=True, a1=16, a2=16)
    assert it_exact <= 2
    _, it1 = D.pcg(m, xc, b, tol=1e-10, precond=True)
    _, it0 = D.pcg(m, xc, b, tol=1e-10, precond=False)
    assert it0 > 2 * it1


def test_kpm_converges_to_lu_inverse():
    """With growing order (a1 = a2 -> large) the KPM P^{-1} v approaches the LU
    solve of Eq. (P_def)."""
    m = D.Model(L=4, Ltau=8)
    x = rng(20).standard_normal((m.Ltau, m.N))
    v = rng(21).standard_normal((m.Ltau, m.N))
    ref = np.linalg.solve(D.precond_matrix(m, x), v.reshape(-1)).reshape(m.Ltau, m.N)
    errs = [np.abs(D.precond_inverse_apply(m, x, v, a1=a, a2=a) - ref).max() for a in (1, 4, 16)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-12


def test_kpm_transpose_is_exact_transpose():
    m = D.Model(L=4, Ltau=8)
    g = rng(22)
    x = g.standard_normal((m.Ltau, m.N))
    v, w = g.standard_normal((2, m.Ltau, m.N))
    lhs = np.sum(w * D.precond_inverse_apply(m, x, v))
    rhs = np.sum(v * D.precond_inverse_apply(m, x, w, trans=True))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_kpm_mirror_half_is_conjugate():
    """f_{T-1-omega} = conj(f_omega) on real b (App. C B): coefficients
    computed directly at phi_{T-1-omega} are the conjugates."""
    T = 40
    for w in (0, 3, 11):
        c = D.chebyshev_coeffs(D.phi_omega(T, w), 0.7, 1.6, 12)
        c2 = D.chebyshev_coeffs(D.phi_omega(T, T - 1 - w), 0.7, 1.6, 12)
        assert np.abs(c2 - np.conj(c)).max() < 1e-13


def test_spectral_bounds_contain_Bbar_spectrum():
    """The deterministic bounds contain the spectrum of Bbar, and for x = 0
    they match the paper's estimates 0.7 and 1.6 (App. C)."""
    for seed in range(3):
        m = D.Model(L=6, Ltau=8, alpha=1.0)
        x = rng(30 + seed).standard_normal((m.Ltau, m.N)) * 2
        ev = np.linalg.eigvals(D.Bbar(m, x))
        bmin, bmax = D.spectral_bounds(m, x)
        # the norm bound holds for every eigenvalue modulus; with the
        # checkerboard C the spectrum may leave the real axis slightly for
        # strongly fluctuating fields
        assert bmin <= np.abs(ev).min() and np.abs(ev).max() <= bmax
        assert np.abs(ev.imag).max() < 0.05 * np.abs(ev).max()
        assert bmin <= ev.real.min() and ev.real.max() <= bmax
    gb = GOLD["bbar_bounds_free"]
    m = D.Model(L=6, Ltau=8)
    bmin, bmax = D.spectral_bounds(m, np.zeros((m.Ltau, m.N)))
    assert abs(bmin - gb["bmin"]) < 0.05 and abs(bmax - gb["bmax"]) < 0.15


def test_chebyshev_coefficients_closed_form():
    """For f(y) = 1/(a - c y) the Chebyshev series is geometric:
    c_0 = 2r/(c(1-r^2)), c_m = 4 r^{m+1}/(c(1-r^2)) with r + 1/r = 2a/c, |r| < 1;
    the quadrature of Eq. (Cheby-Gauss) reproduces it."""
    for phi in (0.05, 0.3, 2.0):
        bmin, bmax = 0.7, 1.6
        db = bmax - bmin
        a = 1 - np.exp(-1j * phi) * (bmin + db / 2)
        c = np.exp(-1j * phi) * db / 2
        z = a / c
        r = z - np.sqrt(z * z - 1)
        if abs(r) > 1:
            r = z + np.sqrt(z * z - 1)
        K = 24
        ref = np.array([2 * r / (c * (1 - r * r))] + [4 * r ** (k + 1) / (c * (1 - r * r)) for k in range(1, K)])
        got = D.chebyshev_coeffs(phi, bmin, bmax, K, NQ=max(2 * K, 4000))
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_matvec_count_worked_example():
    g1, g2 = GOLD["n_matvec_per_Ltau"], GOLD["n_matvec_bound_per_Ltau"]
    T = g1["Ltau"]
    assert abs(D.n_matvec_count(T, g1["delta_b"]) / T - g1["value"]) < 1e-9
    assert abs(D.n_matvec_bound(T, g2["delta_b"]) / T - g2["value"]) < 0.01


# ---------------------------------------------------------------- measurements
def test_cross_correlation_direct_equals_fft():
    g = rng(40)
    a, b = g.standard_normal((2, 8, 16))
    out = D.cross_corr_direct(a, b, 4)
    fa, fb = np.fft.fftn(a.reshape(8, 4, 4)), np.fft.fftn(b.reshape(8, 4, 4))
    ref = np.fft.ifftn(np.conj(fa) * fb).real
    assert np.abs(out - ref).max() < 1e-12


def test_cross_correlation_at_offsets_equals_fft_and_full_estimators():
    """The selected-offset sums equal the FFT cross-correlation (numpy's
    fftn, a different route) at those offsets, and the selected-offset 2-
    and 4-point estimators equal the full-array ones there (probes and
    stand-in solutions random; the estimators are bilinear in them)."""
    g = rng(43)
    L, T2 = 6, 10
    a, b = g.standard_normal((2, T2, L * L))
    deltas = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 2, 5), (9, 5, 1), (5, 3, 3),
              (7, 0, 4)]
    fa, fb = np.fft.fftn(a.reshape(T2, L, L)), np.fft.fftn(b.reshape(T2, L, L))
    full = np.fft.ifftn(np.conj(fa) * fb).real
    out = D.cross_corr_at(a, b, L, deltas)
    assert np.abs(out - np.array([full[d] for d in deltas])).max() < 1e-12
    m = D.Model(L=L, Ltau=T2 // 2)
    xi = np.sign(g.standard_normal((4, m.Ltau, m.N)))
    gx = g.standard_normal((4, m.Ltau, m.N))
    G2 = D.green_average(m, None, xi, gx)
    G4 = D.four_point_pairs(m, None, xi, gx)
    assert np.abs(D.green_average_at(m, xi, gx, deltas) - np.array([G2[d] for d in deltas])).max() \
        < 1e-13
    at4 = D.four_point_pairs_at(m, xi, gx, deltas)
    for k in range(3):
        assert np.abs(at4[k] - np.array([G4[k][d] for d in deltas])).max() < 1e-13


def test_green_average_complete_probe_sets_are_exact():
    """sum_k (G xi_k) xi_k^T = G for the unit vectors and (times n) for the
    rows of a Hadamard matrix, so the stochastic average (Eq. (G_approx_better))
    over a complete +-1 set equals the exact average of Eq. (G_avg-1)."""
    import scipy.linalg
    m = D.Model(L=4, Ltau=4, alpha=1.0)
    x = rng(41).standard_normal((m.Ltau, m.N))
    exact = D.green_average_exact(m, x)
    H = scipy.linalg.hadamard(m.n).astype(float).reshape(m.n, m.Ltau, m.N)
    est = D.green_average(m, x, H)
    assert np.abs(est - exact).max() < 1e-12
    # antiperiodicity of the doubled domain
    assert np.abs(exact[m.Ltau:] + exact[:m.Ltau]).max() < 1e-13


def test_four_point_pair_sum_identity():
    """Type-2 products: sum_{n<m} (c_n star c_m) at +Delta and -Delta adds up to
    (sum c) star (sum c) - sum_n c_n star c_n (computed here with FFTs)."""
    m = D.Model(L=4, Ltau=4, alpha=1.0)
    g = rng(42)
    x = g.standard_normal((m.Ltau, m.N))
    xi = np.sign(g.standard_normal((4, m.Ltau, m.N)))
    G = D.green_matrix(m, x)
    Gxi = np.array([(G @ v.reshape(-1)).reshape(m.Ltau, m.N) for v in xi])
    out = D.four_point_pairs(m, x, xi, Gxi)
    npairs = 6
    c = [(D.extend(a) * D.extend(b)).reshape(2 * m.Ltau, m.L, m.L) for a, b in zip(xi, Gxi)]
    F = [np.fft.fftn(ci) for ci in c]
    S = sum(F)
    tot = np.fft.ifftn(np.conj(S) * S - sum(np.conj(f) * f for f in F)).real
    neg = np.roll(np.flip(out[1], axis=(0, 1, 2)), 1, axis=(0, 1, 2))  # value at -Delta
    assert np.abs((out[1] + neg) * (2.0 * m.n * npairs) - tot).max() < 1e-10


# ---------------------------------------------------------------- matrix-free C oracle
def test_matfree_operators_equal_dense():
    m = D.Model(L=4, Ltau=10, alpha=1.2, mu=0.1)
    g = rng(50)
    x = g.standard_normal((m.Ltau, m.N))
    v = g.standard_normal((m.Ltau, m.N))
    assert np.abs(MF.M_apply(m, x, v) - D.M_apply(m, x, v)).max() < 1e-13
    assert np.abs(MF.MT_apply(m, x, v) - D.MT_apply(m, x, v)).max() < 1e-13


@pytest.mark.parametrize("L,T", [(6, 4), (8, 6), (4, 10)])
def test_matfree_exact_propagator_equals_dense(L, T):
    """The C oracle's exact exp(-dtau K) (ring Fourier modes) against the
    dense oracle's (scipy's matrix exponential of the hopping matrix):
    M, M^T and the fermion force."""
    m = D.Model(L=L, Ltau=T, alpha=1.1, mu=0.2, kinetic="exact")
    g = rng(52)
    x = g.standard_normal((m.Ltau, m.N))
    v = g.standard_normal((m.Ltau, m.N))
    assert np.abs(MF.M_apply(m, x, v) - D.M_apply(m, x, v)).max() < 1e-13
    assert np.abs(MF.MT_apply(m, x, v) - D.MT_apply(m, x, v)).max() < 1e-13
    R = g.standard_normal((1, m.Ltau, m.N))
    Phi = D.phi_from_R(m, x + 0.1, R)
    b = D.b_from_phi(m, x, Phi[0])
    vd = D.solve_MTM(m, x, b)
    F = MF.force_fermion(m, x, vd, b)
    Fd = D.dSF_dx(m, x, Phi)
    assert np.abs(F - Fd).max() < 1e-11 * np.abs(Fd).max()


def test_matfree_cg_and_force_equal_dense():
    m = D.Model(L=4, Ltau=10, alpha=1.2)
    g = rng(51)
    x = g.standard_normal((m.Ltau, m.N))
    R = g.standard_normal((1, m.Ltau, m.N))
    Phi = D.phi_from_R(m, x + 0.2, R)
    b = D.b_from_phi(m, x, Phi[0])
    v, it, res = MF.cg(m, x, b, tol=1e-13)
    assert it > 0 and res < 1e-13
    vd = D.solve_MTM(m, x, b)
    assert np.abs(v - vd).max() < 1e-9 * np.abs(vd).max()
    F = MF.force_fermion(m, x, vd, b) + MF.force_boson(m, x)
    Fd = D.dSF_dx(m, x, Phi) + D.dSB_dx(m, x)
    assert np.abs(F - Fd).max() < 1e-11 * np.abs(Fd).max()


# ----------------------------------------------------------------------------
# Reflection and swap updates (Sec. IV)
# ----------------------------------------------------------------------------
def test_global_moves_leave_S_B_invariant():
    """S_B is a sum of per-site terms, each even in x: reflecting one site's
    line or exchanging two lines does not change it (any x)."""
    w = hi.WORKLOADS["tiny"]
    m = D.model_of(w)
    x = hi.phonon_field(w, seed=41)
    for kind, i, j in ((D.REFLECT, 3, -1), (D.SWAP, 3, 7), (D.SWAP, 0, 15)):
        y = D.propose_global(x, kind, i, j)
        assert abs(D.S_B(m, y) - D.S_B(m, x)) < 1e-12 * D.S_B(m, x)
    # two swaps of the same pair restore x; a reflection twice too
    y = D.propose_global(D.propose_global(x, D.SWAP, 2, 9), D.SWAP, 2, 9)
    assert np.array_equal(y, x)
    y = D.propose_global(D.propose_global(x, D.REFLECT, 5), D.REFLECT, 5)
    assert np.array_equal(y, x)


def test_global_moves_free_without_coupling():
    """alpha = 0: M and Lambda do not depend on x, so every reflection and
    swap has dS = 0 and is accepted for any u < 1."""
    w = hi.Workload("a0", L=4, Ltau=20, alpha=0.0, mu=0.2, omega0=1.0, x_std=1.0, seed=43)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 2, seed=44)
    Phi = D.phi_from_R(m, x, R)
    for kind, i, j in ((D.REFLECT, 6, -1), (D.SWAP, 1, 2)):
        acc, dS, y = D.global_update(m, x, Phi, kind, i, j, 0.999)
        assert acc and abs(dS) < 1e-10
        assert np.array_equal(y, D.propose_global(x, kind, i, j))


def test_single_site_reflection_is_free_for_constant_lines():
    """Single-site limit (t = 0) at half filling with tau-constant fields
    (App. B; the symmetry behind Eq. (Delta_S_sym)): S_F(-x, Phi) = S_F(x, Phi)
    for any Phi, so reflecting a site costs nothing. With tau fluctuations the
    move is no longer free (the pin is not vacuous)."""
    w = hi.Workload("ss", L=4, Ltau=20, t=0.0, alpha=2.0, mu=0.0, omega0=1.0, x_std=1.0, seed=45)
    m = D.model_of(w)
    rng = np.random.default_rng(46)
    xbar = rng.normal(0.0, 1.0, size=w.N)
    x = np.tile(xbar, (w.Ltau, 1))
    Phi = rng.normal(size=(2, w.Ltau, w.N))
    for i in (0, 5, 11):
        y = D.propose_global(x, D.REFLECT, i)
        assert abs(D.S_F(m, y, Phi) - D.S_F(m, x, Phi)) < 1e-9 * D.S_F(m, x, Phi)
    xf = x + 0.3 * rng.normal(size=x.shape)
    y = D.propose_global(xf, D.REFLECT, 5)
    assert abs(D.S_F(m, y, Phi) - D.S_F(m, xf, Phi)) > 1e-3


# ----------------------------------------------------------------------------
# Observables (Eq. (Scdw), P_s)
# ----------------------------------------------------------------------------
def test_observables_from_products_match_wick_definitions():
    """The contraction of the space-time averaged G and the three Wick
    products (what the stochastic measurement estimates) reproduces the
    observables formed from the dense G by Wick's theorem for every pair of
    sites (independent index sums)."""
    w = hi.Workload("ob", L=4, Ltau=10, alpha=1.0, mu=0.1, omega0=1.0, x_std=0.7, seed=91)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    ex = D.observables_exact(m, x)
    es = D.observables_from_estimates(m, D.green_average_exact(m, x), D.wick_products_exact(m, x))
    for k in ("density", "S_cdw", "P_s"):
        assert abs(ex[k] - es[k]) < 1e-12 * max(1.0, abs(ex[k]))
    assert np.abs(ex["C"] - es["C"]).max() < 1e-12


def test_observables_particle_hole_at_half_filling():
    """mu = 0 on the bipartite lattice: x -> -x maps n -> 2 - n, so
    <n>(x) + <n>(-x) = 2 and C_{-x}(r) = C_x(r) + 4 - 4 <n>(x), for every
    configuration (the same symmetry as the log det pin); free fermions are
    exactly half filled."""
    w = hi.Workload("ph", L=4, Ltau=10, alpha=1.3, mu=0.0, omega0=1.0, x_std=0.7, seed=92)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    a = D.observables_exact(m, x)
    b = D.observables_exact(m, -x)
    assert abs(a["density"] + b["density"] - 2.0) < 1e-12
    assert np.abs(b["C"] - (a["C"] + 4.0 - 4.0 * a["density"])).max() < 1e-12
    assert abs(D.observables_exact(m, np.zeros_like(x))["density"] - 1.0) < 1e-12


@pytest.mark.parametrize("L,T,mu", [(4, 10, 0.3), (6, 8, -0.45)])
def test_observables_free_fermion_closed_form(L, T, mu):
    """Free fermions (x = 0) with the exact propagator: B = exp(-dtau (K - mu))
    is diagonal in momentum with b_k = exp(-dtau (eps_k - mu)), so G = M^{-1}
    splits into one T x T matrix per k, G_k(l, l') = b^(l-l') / (1 + b^T) for
    l >= l' and -b^(T+l-l') / (1 + b^T) for l < l' (the inverse of the
    antiperiodic bidiagonal matrix of Eq. (M_def)). Written from that:
      <n>  = 2 (1 - (1/N) sum_k 1/(1 + b_k^T));
      C(r) = 4 (1 - g(0))^2 + 2 (delta_r0 - g(r)) g(r),
             g(r) = (1/N) sum_k e^{i k.r} / (1 + b_k^T) (equal-time G, even in r);
      P_s  = dtau / (N T) sum_{l, l'} sum_{r, r'} G^2 = dtau / (N T) sum_k
             sum_{l, l'} G_k(l, l')^2 (the Fourier transform keeps the
             Frobenius norm of every N x N block).
    A wrong dtau, 1/N or slice range in P_s, or a wrong sign or index in the
    C(r) contraction, fails it."""
    m = D.Model(L=L, Ltau=T, mu=mu, kinetic="exact")
    x = np.zeros((T, m.N))
    ks = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(ks, ks, indexing="xy")         # [iky][ikx]
    eps = -2 * m.t * (np.cos(kx) + np.cos(ky))
    b = np.exp(-m.dtau * (eps - mu))
    occ = 1.0 / (1.0 + b ** T)                            # G_k(l, l)
    dens = 2.0 * (1.0 - occ.mean())
    g = np.real(np.fft.ifft2(occ))                        # g(r) at [dy][dx]
    delta = np.zeros((L, L))
    delta[0, 0] = 1.0
    C = 4.0 * (1.0 - g[0, 0]) ** 2 + 2.0 * (delta - g) * g
    ps = 0.0
    for bk in b.ravel():
        for d in range(T):                                # l - l' = d >= 0: T - d pairs
            ps += (T - d) * (bk ** d / (1.0 + bk ** T)) ** 2
        for d in range(1, T):                             # l' - l = d > 0: T - d pairs
            ps += (T - d) * (bk ** (T - d) / (1.0 + bk ** T)) ** 2
    ps *= m.dtau / (m.N * T)
    ex = D.observables_exact(m, x)
    assert abs(ex["density"] - dens) < 1e-12
    assert np.abs(ex["C"] - C).max() < 1e-12
    assert abs(ex["P_s"] - ps) < 1e-12 * ps
    S = float(np.sum(np.array([[(-1.0) ** (dx + dy) for dx in range(L)] for dy in range(L)]) * C))
    assert abs(ex["S_cdw"] - S) < 1e-12 * max(1.0, abs(S))
    # the contraction of the estimators' expectations gives the same P_s
    es = D.observables_from_estimates(m, D.green_average_exact(m, x), D.wick_products_exact(m, x))
    assert abs(es["P_s"] - ps) < 1e-12 * ps
    assert np.abs(es["C"] - C).max() < 1e-12


# ---------------------------------------------------------------- Arnoldi bounds (App. C D)
def test_arnoldi_full_dimension_gives_the_spectrum():
    """N steps of Arnoldi span the whole space: the Ritz values are the
    eigenvalues, so with margin 0 bmax is the largest eigenvalue modulus of
    Bbar and bmin (from Bbar^{-1}) the smallest (numpy's eigvals of the dense
    Bbar, a different route)."""
    w = hi.Workload("a", L=4, Ltau=10, alpha=1.3, mu=0.2, x_std=1.0, seed=5)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    lo, hi_, runs = D.arnoldi_bounds(m, x, hi.site_vector(w, seed=6), steps=m.N, margin=0.0)
    ev = np.abs(np.linalg.eigvals(D.Bbar(m, x)))
    assert runs["B"][2] == m.N and runs["Binv"][2] == m.N
    assert abs(lo - ev.min()) < 1e-10 * ev.max()
    assert abs(hi_ - ev.max()) < 1e-10 * ev.max()


@pytest.mark.parametrize("kinetic", ["checkerboard", "exact"])
def test_arnoldi_relation_and_orthonormal_basis(kinetic):
    """A V_k = V_{k+1} H (the Arnoldi relation) with orthonormal V for Bbar
    and Bbar^{-1}, and the 20-step bounds lie inside the deterministic norm
    bounds; Bbar^{-1} is the inverse of Bbar."""
    w = hi.Workload("a", L=8, Ltau=12, alpha=1.1, x_std=1.0, seed=7)
    m = D.model_of(w, kinetic=kinetic)
    x = hi.phonon_field(w)
    lo, hi_, runs = D.arnoldi_bounds(m, x, hi.site_vector(w, seed=8), steps=20, margin=0.0)
    B = D.Bbar(m, x)
    Binv = np.linalg.inv(B)
    for key, A in (("B", B), ("Binv", Binv)):
        H, V, k = runs[key]
        assert k == 20
        assert np.abs(A @ V[:k].T - V.T @ H).max() < 1e-11 * np.abs(A).max()
        assert np.abs(V @ V.T - np.eye(k + 1)).max() < 1e-12
    dlo, dhi = D.spectral_bounds(m, x)
    assert dlo <= lo <= hi_ <= dhi


# ---------------------------------------------------------------- further pins
def test_leapfrog_is_symplectic():
    """Algorithm 1's map (x, p) -> (x', p') at fixed Phi is symplectic: its
    Jacobian J (central differences, h = 1e-6) satisfies J^T Omega J = Omega
    for the canonical form Omega. A force that is not the gradient of the
    action (a dropped or mis-signed term) breaks this."""
    w = hi.Workload("s", L=4, Ltau=2, alpha=1.1, mu=0.2, omega0=1.0, x_std=1.0, seed=5)
    m = D.model_of(w)
    x0 = hi.phonon_field(w)
    R = hi.gaussian_vectors(w, 1, seed=6)
    Phi = D.phi_from_R(m, x0, R)
    p0 = hi.gaussian_vectors(w, 1, seed=7)[0]
    n = m.n
    dt, Nt, nt, mreg = 0.05, 2, 2, 1.0

    def flow(z):
        xf, pf = D.leapfrog_split(m, z[:n].reshape(m.Ltau, m.N), z[n:].reshape(m.Ltau, m.N),
                                  Phi, dt, Nt, nt, mreg)
        return np.concatenate([xf.ravel(), pf.ravel()])

    z0 = np.concatenate([x0.ravel(), p0.ravel()])
    h = 1e-6
    J = np.empty((2 * n, 2 * n))
    for k in range(2 * n):
        e = np.zeros(2 * n)
        e[k] = h
        J[:, k] = (flow(z0 + e) - flow(z0 - e)) / (2 * h)
    Om = np.block([[np.zeros((n, n)), np.eye(n)], [-np.eye(n), np.zeros((n, n))]])
    # the Fourier-accelerated kinetic term p M^{-1} p / 2 is a constant metric,
    # so the flow preserves the canonical form of (x, p) itself
    assert np.abs(J.T @ Om @ J - Om).max() < 1e-6
    assert abs(np.linalg.det(J) - 1.0) < 1e-6


def test_atomic_limit_density():
    """t = 0: every site decouples and its occupation per spin is
    1 / (1 + exp(dtau sum_tau (alpha x_tau - mu))) (det M factorises over sites
    at t = 0, Eq. (M_def)), so <n> is twice its site average."""
    w = hi.Workload("a", L=4, Ltau=6, t=0.0, alpha=0.9, mu=0.3, x_std=1.0, seed=8)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    occ = 1.0 / (1.0 + np.exp(m.dtau * (m.alpha * x - m.mu).sum(axis=0)))
    obs = D.observables_exact(m, x)
    assert abs(obs["density"] - 2.0 * occ.mean()) < 1e-12


def test_stochastic_estimators_are_unbiased_over_z2_probes():
    """Sec. V B-C: with Z2 probes (<xi_i xi_j> = delta_ij) the 2-point average
    and the pair-averaged Wick products are unbiased estimates of the exact
    space-time averages: their mean over many independent probe sets lies
    within a few standard errors of the dense-G values, and the spread of a
    single set shrinks as the probe count grows."""
    w = hi.Workload("u", L=4, Ltau=4, alpha=1.0, mu=0.1, x_std=1.0, seed=21)
    m = D.model_of(w)
    x = hi.phonon_field(w)
    G = D.green_matrix(m, x)
    exact2 = D.green_average_exact(m, x)
    exact4 = D.wick_products_exact(m, x)
    sets, nrv = 200, 4
    e2, e4 = [], []
    for k in range(sets):
        xi = hi.z2_vectors(w, nrv, seed=1000 + k)
        Gxi = np.array([(G @ v.reshape(-1)).reshape(m.Ltau, m.N) for v in xi])
        e2.append(D.green_average(m, x, xi, Gxi))
        e4.append(D.four_point_pairs(m, x, xi, Gxi))
    e2, e4 = np.array(e2), np.array(e4)
    for est, exact in ((e2, exact2), (e4, exact4)):
        mean = est.mean(axis=0)
        se = est.std(axis=0, ddof=1) / np.sqrt(sets) + 1e-12
        z = np.abs(mean - exact) / se
        assert np.median(z) < 1.5 and z.max() < 6.0
    # a set of 16 probes is closer to the exact value than a set of 4, on average
    err4 = np.mean([np.abs(D.green_average(m, x, hi.z2_vectors(w, 4, seed=5000 + k)) - exact2).mean()
                    for k in range(20)])
    err16 = np.mean([np.abs(D.green_average(m, x, hi.z2_vectors(w, 16, seed=6000 + k)) - exact2).mean()
                     for k in range(20)])
    assert err16 < 0.75 * err4
