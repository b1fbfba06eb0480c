"""Dense FP64 oracle for the Holstein HMC hot path -- TEST INFRASTRUCTURE ONLY.

Every matrix of the method is formed densely and every result follows the
paper's definition with a library primitive (dense solve, slogdet, matrix
exponential) as the only building block. Sizes: n = N * Ltau up to a few
thousand.

Conventions
-----------
* site index i = ix + L*iy on the periodic L x L square lattice, N = L*L;
* a space-time vector is laid out [tau][i]; flattened index tau*N + i;
* s_0 = +1 (the antiperiodic corner block), s_tau = -1 for tau >= 1.

Readings of the paper taken here:

* B_tau = exp(-dtau V_tau) exp(-dtau K): the diagonal acts last (Eq. (B_def)).
* The "minimal split checkerboard" exp(-dtau K) (Sec. II D) is the product
  C = C4 C3 C2 C1 of four bond colours: 1 = x-bonds from even ix, 2 = x-bonds
  from odd ix, 3 = y-bonds from even iy, 4 = y-bonds from odd iy; each bond
  contributes the exact two-site factor [[cosh, sinh], [sinh, cosh]](dtau t).
* sin^2 argument in the bosonic spectrum and the Fourier-acceleration mass
  (Eq. (Qww_def) and the mass of Eq. (dynamical_M_def)) is pi*omega/Ltau:
  the printed 2*pi*omega/Ltau contradicts Eq. (dSB_dx) and the stated
  extremes at omega = Ltau/2.
* Chebyshev order N_P = max(1, floor(db (a1/phi + a2))) (Eq. (NP_heuristic)), a1 = a2 = 1.
* Spectral bounds of Bbar (App. C D): the deterministic bound
  bmax = max_i dbar_i exp(4 dtau |t|), bmin = min_i dbar_i exp(-4 dtau |t|),
  which bounds the modulus of every eigenvalue (norm bound on Bbar and on
  Bbar^{-1}); the paper reports the spectrum real for equilibrium fields,
  while strongly fluctuating i.i.d. fields can give it small imaginary parts.
* The transpose of the approximate P^{-1} is U^dag diag(sum conj(c_m)
  T_m(A^T)) U, so that P^{-1} P^{-T} stays symmetric positive definite.
* Space-time averaged Green function (Eq. (G_avg-1)): the average over the
  original N*Ltau sites, i.e. the circular sum over the doubled domain
  divided by 2*N*Ltau.

Each function is pinned against closed forms, invariants or brute force in
tests/test_oracle_pins.py.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg


# ----------------------------------------------------------------------------
# Model (Sec. II A-C)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Model:
    L: int
    Ltau: int
    dtau: float = 0.1
    t: float = 1.0
    mu: float = 0.0
    alpha: float = 1.0
    omega0: float = 1.0
    kinetic: str = "checkerboard"   # or "exact"

    @property
    def N(self) -> int:
        return self.L * self.L

    @property
    def n(self) -> int:
        return self.N * self.Ltau

    @property
    def beta(self) -> float:
        return self.dtau * self.Ltau


def model_of(w, kinetic: str = "checkerboard") -> Model:
    """Model from a holstein_inputs.Workload."""
    return Model(L=w.L, Ltau=w.Ltau, dtau=w.dtau, t=w.t, mu=w.mu,
                 alpha=w.alpha, omega0=w.omega0, kinetic=kinetic)


def site(ix: int, iy: int, L: int) -> int:
    return (ix % L) + L * (iy % L)


def hopping_matrix(m: Model) -> np.ndarray:
    """K_ij = -t_ij, nearest neighbours of the periodic square lattice (Eq. (V_K_def))."""
    N, L = m.N, m.L
    K = np.zeros((N, N))
    for iy in range(L):
        for ix in range(L):
            i = site(ix, iy, L)
            for j in (site(ix + 1, iy, L), site(ix, iy + 1, L)):
                K[i, j] -= m.t
                K[j, i] -= m.t
    return K


def bond_colours(L: int):
    """Four perfect matchings of the bonds (L even): x-even, x-odd, y-even, y-odd."""
    assert L % 2 == 0 and L >= 4
    cols = [[], [], [], []]
    for iy in range(L):
        for ix in range(L):
            i = site(ix, iy, L)
            cols[ix % 2].append((i, site(ix + 1, iy, L)))
            cols[2 + iy % 2].append((i, site(ix, iy + 1, L)))
    return cols


def checkerboard_factors(m: Model):
    """C_c = exp(dtau * t * sum_{bonds in colour c} (|i><j| + |j><i|)), exact
    for each colour because its bonds are disjoint."""
    ch, sh = np.cosh(m.dtau * m.t), np.sinh(m.dtau * m.t)
    out = []
    for pairs in bond_colours(m.L):
        C = np.eye(m.N)
        for i, j in pairs:
            C[i, i] = ch
            C[j, j] = ch
            C[i, j] = sh
            C[j, i] = sh
        out.append(C)
    return out


def kinetic_propagator(m: Model) -> np.ndarray:
    """exp(-dtau K): checkerboard C4 C3 C2 C1, or the exact matrix exponential."""
    if m.kinetic == "exact":
        return scipy.linalg.expm(-m.dtau * hopping_matrix(m))
    C1, C2, C3, C4 = checkerboard_factors(m)
    return C4 @ C3 @ C2 @ C1


def expV(m: Model, x: np.ndarray) -> np.ndarray:
    """Diagonal of exp(-dtau V_tau), (V_tau)_ii = alpha x_{i,tau} - mu (Eq. (V_K_def)). [T][N]"""
    return np.exp(-m.dtau * (m.alpha * np.asarray(x) - m.mu))


def B_blocks(m: Model, x: np.ndarray):
    """B_tau = exp(-dtau V_tau) exp(-dtau K) (Eq. (B_def))."""
    C = kinetic_propagator(m)
    d = expV(m, x)
    return [d[tau][:, None] * C for tau in range(m.Ltau)]


def fermion_matrix(m: Model, x: np.ndarray) -> np.ndarray:
    """M of Eq. (M_def): identity diagonal blocks, -B_tau below the diagonal and
    +B_0 in the top-right corner."""
    N, T = m.N, m.Ltau
    B = B_blocks(m, x)
    M = np.eye(N * T)
    for tau in range(1, T):
        M[tau * N:(tau + 1) * N, (tau - 1) * N:tau * N] = -B[tau]
    M[0:N, (T - 1) * N:T * N] = B[0]
    return M


def Lambda(m: Model, x: np.ndarray) -> np.ndarray:
    """Lambda of Eq. (Lambda_def): entry ((i,tau),(i,tau+1)) = (2 delta_{tau+1,0} - 1)
    exp(+dtau alpha x_{i,tau+1} / 2), tau periodic."""
    N, T = m.N, m.Ltau
    Lm = np.zeros((N * T, N * T))
    for tau in range(T):
        tp = (tau + 1) % T
        sgn = 1.0 if tp == 0 else -1.0
        for i in range(N):
            Lm[tau * N + i, tp * N + i] = sgn * np.exp(0.5 * m.dtau * m.alpha * x[tp, i])
    return Lm


def Lambda_inv(m: Model, x: np.ndarray) -> np.ndarray:
    """Lambda^{-1} of Eq. (Lambda_inv): entry ((i,tau),(i,tau-1)) = (2 delta_{tau,0} - 1)
    exp(-dtau alpha x_{i,tau} / 2)."""
    N, T = m.N, m.Ltau
    Li = np.zeros((N * T, N * T))
    for tau in range(T):
        tm = (tau - 1) % T
        sgn = 1.0 if tau == 0 else -1.0
        for i in range(N):
            Li[tau * N + i, tm * N + i] = sgn * np.exp(-0.5 * m.dtau * m.alpha * x[tau, i])
    return Li


def A_matrix(m: Model, x: np.ndarray) -> np.ndarray:
    """A = M Lambda (Sec. II D)."""
    return fermion_matrix(m, x) @ Lambda(m, x)


def logdet_M(m: Model, x: np.ndarray) -> float:
    sign, ld = np.linalg.slogdet(fermion_matrix(m, x))
    return ld


# ----------------------------------------------------------------------------
# Operators on vectors (matrix-vector products with the dense matrices)
# ----------------------------------------------------------------------------
def M_apply(m: Model, x, v):
    return (fermion_matrix(m, x) @ np.asarray(v).reshape(-1)).reshape(m.Ltau, m.N)


def M_apply_blocks(m: Model, x, v, C=None):
    """M v block by block from Eq. (M_def): (M v)_0 = v_0 + B_0 v_{T-1},
    (M v)_tau = v_tau - B_tau v_{tau-1}, B_tau = diag(expV_tau) C with the
    dense N x N propagator C (passed in to reuse it). For lattices whose
    full M does not fit in memory."""
    C = kinetic_propagator(m) if C is None else C
    d = expV(m, x)
    v = np.asarray(v).reshape(m.Ltau, m.N)
    out = np.empty_like(v)
    for tau in range(m.Ltau):
        s = 1.0 if tau == 0 else -1.0
        out[tau] = v[tau] + s * d[tau] * (C @ v[tau - 1])
    return out


def MT_apply_blocks(m: Model, x, u, C=None):
    """M^T u block by block: (M^T u)_tau = u_tau + s_{tau+1} C^T diag(expV_{tau+1}) u_{tau+1}."""
    C = kinetic_propagator(m) if C is None else C
    d = expV(m, x)
    u = np.asarray(u).reshape(m.Ltau, m.N)
    T = m.Ltau
    out = np.empty_like(u)
    for tau in range(T):
        tp = (tau + 1) % T
        s = 1.0 if tp == 0 else -1.0
        out[tau] = u[tau] + s * (C.T @ (d[tp] * u[tp]))
    return out


def MT_apply(m: Model, x, v):
    return (fermion_matrix(m, x).T @ np.asarray(v).reshape(-1)).reshape(m.Ltau, m.N)


def MTM_apply(m: Model, x, v):
    M = fermion_matrix(m, x)
    return (M.T @ (M @ np.asarray(v).reshape(-1))).reshape(m.Ltau, m.N)


def solve_MTM(m: Model, x, b):
    """v = (M^T M)^{-1} b (Eq. (CG)) by two dense LU solves: M^T w = b, M v = w."""
    M = fermion_matrix(m, x)
    w = scipy.linalg.solve(M.T, np.asarray(b).reshape(-1))
    v = scipy.linalg.solve(M, w)
    return v.reshape(m.Ltau, m.N)


def rel_residual(m: Model, x, b, v) -> float:
    """epsilon = |b - M^T M v| / |b| (Sec. VI B)."""
    r = np.asarray(b).reshape(-1) - MTM_apply(m, x, v).reshape(-1)
    return float(np.linalg.norm(r) / np.linalg.norm(np.asarray(b).reshape(-1)))


# ----------------------------------------------------------------------------
# Actions and pseudofermions (Sec. II D)
# ----------------------------------------------------------------------------
def S_B(m: Model, x) -> float:
    """Bosonic action, Eq. (S_B)."""
    x = np.asarray(x)
    xp = np.roll(x, -1, axis=0)
    return 0.5 * m.dtau * float(np.sum(m.omega0 ** 2 * x * x + ((xp - x) / m.dtau) ** 2))


def dSB_dx(m: Model, x) -> np.ndarray:
    """Bosonic force, Eq. (dSB_dx)."""
    x = np.asarray(x)
    lap = np.roll(x, -1, axis=0) - 2.0 * x + np.roll(x, 1, axis=0)
    return m.dtau * (m.omega0 ** 2 * x - lap / m.dtau ** 2)


def phi_from_R(m: Model, x, R):
    """Phi = A^T(x) R (Eq. (PhiSample-1)). R: [..., T, N]."""
    A = A_matrix(m, x)
    R = np.asarray(R)
    return (R.reshape(-1, m.n) @ A).reshape(R.shape)


def b_from_phi(m: Model, x, Phi):
    """b = Lambda^{-T} Phi (Sec. II D, below Eq. (psi_def))."""
    Li = Lambda_inv(m, x)
    Phi = np.asarray(Phi)
    return (Phi.reshape(-1, m.n) @ Li).reshape(Phi.shape)


def S_F(m: Model, x, Phi) -> float:
    """Fermionic action, Eq. (S_F): (1/2) sum_sigma |A^{-T} Phi_sigma|^2."""
    A = A_matrix(m, x)
    Phi = np.asarray(Phi).reshape(-1, m.n)
    y = scipy.linalg.solve(A.T, Phi.T)
    return 0.5 * float(np.sum(y * y))


def dSF_dx(m: Model, x, Phi) -> np.ndarray:
    """Fermionic force, Eq. (dSF_dx): -sum_sigma Psi^T A^T (dA/dx_{i,tau}) Psi with
    Psi = (A^T A)^{-1} Phi and dA = (dM) Lambda + M (dLambda) (Sec. III A).

    dM/dx_{i,tau} has one nonzero row, (i,tau): the row of s_tau B_tau whose
    diagonal factor is differentiated, d exp(-dtau(alpha x - mu)) / dx =
    -dtau alpha exp(-dtau(alpha x - mu)). dLambda/dx_{i,tau} has one nonzero
    entry, ((i,tau-1),(i,tau)), equal to (dtau alpha / 2) times that entry of
    Lambda. Both products with Psi are taken entry by entry from these rows
    and columns."""
    N, T = m.N, m.Ltau
    x = np.asarray(x)
    M = fermion_matrix(m, x)
    Lm = Lambda(m, x)
    A = M @ Lm
    C = kinetic_propagator(m)
    d = expV(m, x)
    Phi = np.asarray(Phi).reshape(-1, m.n)
    AtA = A.T @ A
    F = np.zeros((T, N))
    for phi in Phi:
        Psi = scipy.linalg.solve(AtA, phi)
        u = A @ Psi                      # A Psi
        LPsi = (Lm @ Psi).reshape(T, N)  # Lambda Psi
        MTu = (M.T @ u).reshape(T, N)
        u = u.reshape(T, N)
        Psi = Psi.reshape(T, N)
        for tau in range(T):
            s = 1.0 if tau == 0 else -1.0
            tm = (tau - 1) % T
            CL = C @ LPsi[tm]            # e^{-dtau K} (Lambda Psi)_{tau-1}
            for i in range(N):
                # row (i,tau) of dM times Lambda Psi
                dM_LPsi = s * (-m.dtau * m.alpha * d[tau, i]) * CL[i]
                term1 = u[tau, i] * dM_LPsi
                # M dLambda Psi = column (i,tau-1) of M times the single entry
                lam = (1.0 if tau == 0 else -1.0) * np.exp(0.5 * m.dtau * m.alpha * x[tau, i])
                dL_Psi = 0.5 * m.dtau * m.alpha * lam * Psi[tau, i]
                term2 = MTu[tm, i] * dL_Psi
                F[tau, i] -= term1 + term2
    return F


def dSF_dx_fully_dense(m: Model, x, Phi, comps):
    """Same as dSF_dx but builds dA/dx_{i,tau} as a full dense matrix for each
    requested component (i, tau): the definition with no structure used.
    Slow; for cross-checking dSF_dx on tiny sizes."""
    N, T = m.N, m.Ltau
    x = np.asarray(x)
    M = fermion_matrix(m, x)
    Lm = Lambda(m, x)
    A = M @ Lm
    C = kinetic_propagator(m)
    d = expV(m, x)
    Phi = np.asarray(Phi).reshape(-1, m.n)
    AtA = A.T @ A
    Psis = [scipy.linalg.solve(AtA, phi) for phi in Phi]
    out = []
    for (tau, i) in comps:
        dM = np.zeros_like(M)
        s = 1.0 if tau == 0 else -1.0
        tm = (tau - 1) % T
        dM[tau * N + i, tm * N:(tm + 1) * N] = s * (-m.dtau * m.alpha * d[tau, i]) * C[i, :]
        dL = np.zeros_like(Lm)
        dL[tm * N + i, tau * N + i] = 0.5 * m.dtau * m.alpha * Lm[tm * N + i, tau * N + i]
        dA = dM @ Lm + M @ dL
        out.append(-sum(float(P @ A.T @ dA @ P) for P in Psis))
    return np.array(out)


def dS_dx(m: Model, x, Phi) -> np.ndarray:
    """Total force dS/dx = dS_B/dx + dS_F/dx (Sec. III A)."""
    return dSB_dx(m, x) + dSF_dx(m, x, Phi)


# ----------------------------------------------------------------------------
# Fourier acceleration (Sec. III B)
# ----------------------------------------------------------------------------
def fourier_matrix(T: int) -> np.ndarray:
    """Unitary DFT along tau, F_{omega,tau} = exp(-2 pi i omega tau / T)/sqrt(T) (Eq. (F_def))."""
    w = np.arange(T)[:, None]
    tau = np.arange(T)[None, :]
    return np.exp(-2j * np.pi * w * tau / T) / np.sqrt(T)


def Q_tilde(m: Model) -> np.ndarray:
    """Bosonic stiffness per Fourier mode, Eq. (Qww_def) with sin^2(pi omega / T)."""
    w = np.arange(m.Ltau)
    return m.dtau * (m.omega0 ** 2 + 4.0 / m.dtau ** 2 * np.sin(np.pi * w / m.Ltau) ** 2)


def mass_tilde(m: Model, m_reg: float) -> np.ndarray:
    """Fourier-acceleration mass per mode, Eq. (dynamical_M_def) with sin^2(pi omega / T).
    m_reg = inf gives the constant mass dtau."""
    w = np.arange(m.Ltau)
    s2 = 4.0 / m.dtau ** 2 * np.sin(np.pi * w / m.Ltau) ** 2
    if np.isinf(m_reg):
        return np.full(m.Ltau, m.dtau)
    mr2 = m_reg ** 2 + m.omega0 ** 2
    return m.dtau * (mr2 + s2) / mr2


def tau_operator(T: int, diag: np.ndarray) -> np.ndarray:
    """Real T x T matrix F^{-1} diag F (Eqs. (bosonic_force), (dynamical_M_def))."""
    F = fourier_matrix(T)
    op = F.conj().T @ np.diag(diag) @ F
    assert np.max(np.abs(op.imag)) < 1e-10
    return op.real


def Q_apply(m: Model, x) -> np.ndarray:
    """Q x = F^{-1} Qtilde F x along tau for each site (Eq. (bosonic_force))."""
    return tau_operator(m.Ltau, Q_tilde(m)) @ np.asarray(x)


def mass_apply(m: Model, p, m_reg, power: float = 1.0) -> np.ndarray:
    """Mass^power p along tau for each site, power in {1, -1, 1/2}."""
    return tau_operator(m.Ltau, mass_tilde(m, m_reg) ** power) @ np.asarray(p)


def kinetic_energy(m: Model, p, m_reg) -> float:
    """p^T Mass^{-1} p / 2 (Sec. III A)."""
    p = np.asarray(p)
    return 0.5 * float(np.sum(p * mass_apply(m, p, m_reg, -1.0)))


def hamiltonian(m: Model, x, p, Phi, m_reg) -> float:
    """H = S_B + S_F + p^T Mass^{-1} p / 2."""
    return S_B(m, x) + S_F(m, x, Phi) + kinetic_energy(m, p, m_reg)


def leapfrog_split(m: Model, x, p, Phi, dt, N_t, n_t, m_reg):
    """The molecular-dynamics part of Algorithm 1: N_t fermionic steps of size
    dt, each containing n_t bosonic sub-steps of size dt/n_t. Returns (x, p)."""
    x = np.array(x, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    dtp = dt / n_t
    for _ in range(N_t):
        p = p - 0.5 * dt * dSF_dx(m, x, Phi)
        for _ in range(n_t):
            p = p - 0.5 * dtp * dSB_dx(m, x)
            x = x + dtp * mass_apply(m, p, m_reg, -1.0)
            p = p - 0.5 * dtp * dSB_dx(m, x)
        p = p - 0.5 * dt * dSF_dx(m, x, Phi)
    return x, p


def hmc_update(m: Model, x, R_pf, R_p, dt, N_t, n_t, m_reg):
    """Algorithm 1 up to the Metropolis test: returns (x_f, p_f, H_i, H_f).
    R_pf: [n_pf][T][N] Gaussian draws for Phi; R_p: [T][N] for the momentum."""
    x = np.asarray(x, dtype=np.float64)
    Phi = phi_from_R(m, x, R_pf)
    p = mass_apply(m, R_p, m_reg, 0.5)
    H_i = hamiltonian(m, x, p, Phi, m_reg)
    xf, pf = leapfrog_split(m, x, p, Phi, dt, N_t, n_t, m_reg)
    H_f = hamiltonian(m, xf, pf, Phi, m_reg)
    return xf, pf, H_i, H_f


# ----------------------------------------------------------------------------
# Reflection and swap updates (Sec. IV)
# ----------------------------------------------------------------------------
REFLECT, SWAP = 0, 1


def propose_global(x, kind: int, i: int, j: int = -1) -> np.ndarray:
    """The proposed field of a global move (Sec. IV): reflection x_{i,tau} ->
    -x_{i,tau} at every tau, or swap of the site lines x_{i,.} and x_{j,.}."""
    y = np.array(x, dtype=np.float64, copy=True)
    if kind == REFLECT:
        y[:, i] = -y[:, i]
    elif kind == SWAP:
        y[:, [i, j]] = y[:, [j, i]]
    else:
        raise ValueError(kind)
    return y


def action(m: Model, x, Phi) -> float:
    """S = S_B + S_F at fixed pseudofermion fields (Eq. (S_decompose))."""
    return S_B(m, x) + S_F(m, x, Phi)


def global_update(m: Model, x, Phi, kind: int, i: int, j: int, u: float):
    """Metropolis test (Eq. (metropolis)) of a reflection or swap move at
    fixed Phi: returns (accepted, dS, x_kept)."""
    y = propose_global(x, kind, i, j)
    dS = action(m, y, Phi) - action(m, x, Phi)
    acc = bool(u < np.exp(-dS))
    return acc, dS, (y if acc else np.array(x, dtype=np.float64, copy=True))


# ----------------------------------------------------------------------------
# Adiabatic preconditioner (Sec. VI A, App. C)
# ----------------------------------------------------------------------------
def dbar(m: Model, x) -> np.ndarray:
    """Diagonal of exp(-dtau Vbar) = mean over tau of exp(-dtau V_tau) (Eq. (expnVbar))."""
    return expV(m, x).mean(axis=0)


def Bbar(m: Model, x) -> np.ndarray:
    """Bbar = exp(-dtau Vbar) exp(-dtau K) (Eq. (Bbar))."""
    return dbar(m, x)[:, None] * kinetic_propagator(m)


def precond_matrix(m: Model, x) -> np.ndarray:
    """P of Eq. (P_def): M with every B_tau replaced by Bbar."""
    N, T = m.N, m.Ltau
    Bb = Bbar(m, x)
    P = np.eye(N * T)
    for tau in range(1, T):
        P[tau * N:(tau + 1) * N, (tau - 1) * N:tau * N] = -Bb
    P[0:N, (T - 1) * N:T * N] = Bb
    return P


def U_matrix(T: int) -> np.ndarray:
    """U_{omega,tau} = exp(-2 pi i tau (omega + 1/2) / T) / sqrt(T) (Eq. (U_omega))."""
    w = np.arange(T)[:, None]
    tau = np.arange(T)[None, :]
    return np.exp(-2j * np.pi * tau * (w + 0.5) / T) / np.sqrt(T)


def phi_omega(T: int, w) -> np.ndarray:
    return 2.0 * np.pi / T * (np.asarray(w) + 0.5)


def spectral_bounds(m: Model, x):
    """Deterministic bounds on the (real, positive) spectrum of Bbar: each
    checkerboard colour has eigenvalues exp(+-dtau t), so
    |Bbar| <= max(dbar) exp(4 dtau |t|) and |Bbar^{-1}| <= exp(4 dtau |t|)/min(dbar)."""
    db = dbar(m, x)
    g = np.exp(4.0 * m.dtau * abs(m.t))
    return float(db.min() / g), float(db.max() * g)


def np_order(db: float, phi: float, a1: float = 1.0, a2: float = 1.0) -> int:
    """Chebyshev order heuristic, Eq. (NP_heuristic), floored at 1."""
    return max(1, int(np.floor(db * (a1 / phi + a2))))


def chebyshev_coeffs(phi: float, bmin: float, bmax: float, NP: int, NQ: int | None = None):
    """c_m, m < NP, of f(y) = (1 - e^{-i phi} b(y))^{-1}, b(y) = bmin + (y+1) db / 2
    (Eqs. (f_y), (y_to_b)), by Chebyshev-Gauss quadrature with NQ = 2 NP points (Eq. (Cheby-Gauss))."""
    if NQ is None:
        NQ = 2 * NP
    db = bmax - bmin
    theta = np.pi * (np.arange(NQ) + 0.5) / NQ
    y = np.cos(theta)
    b = bmin + (y + 1.0) * db / 2.0
    f = 1.0 / (1.0 - np.exp(-1j * phi) * b)
    c = np.empty(NP, dtype=np.complex128)
    for mm in range(NP):
        q = np.pi / 2.0 * (2.0 if mm == 0 else 1.0)
        c[mm] = np.pi / (q * NQ) * np.sum(np.cos(mm * theta) * f)
    return c


def arnoldi(A: np.ndarray, v0, steps: int):
    """`steps` steps of the Arnoldi process on the dense matrix A from v0
    (modified Gram-Schmidt, each new vector orthogonalised twice so the basis
    stays orthonormal); stops early on an invariant subspace (new vector
    below 1e-12 of |A v_j|). Returns (H [k+1][k], V [k+1][N], k)."""
    N = A.shape[0]
    V = np.zeros((steps + 1, N))
    H = np.zeros((steps + 1, steps))
    v0 = np.asarray(v0, dtype=np.float64).reshape(N)
    V[0] = v0 / np.linalg.norm(v0)
    k = steps
    for j in range(steps):
        w = A @ V[j]
        wn0 = np.linalg.norm(w)
        for _ in range(2):
            for i in range(j + 1):
                c = V[i] @ w
                H[i, j] += c
                w = w - c * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if not H[j + 1, j] > 1e-12 * wn0:
            k = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return H[:k + 1, :k], V[:k + 1], k


def arnoldi_bounds(m: Model, x, v0, steps: int = 20, margin: float = 0.05):
    """Spectral bounds of Bbar as App. C D estimates them: bmax from `steps`
    Arnoldi steps on Bbar (largest Ritz modulus, increased by the margin),
    bmin from the same on Bbar^{-1} = exp(dtau K) exp(dtau Vbar) (the inverse
    of its largest Ritz modulus increased by the margin). Ritz values are
    numpy's eigvals of the square Hessenberg matrix.
    Returns (bmin, bmax, runs) with runs = {"B": (H, V, k), "Binv": (H, V, k)}."""
    B = Bbar(m, x)
    Binv = np.linalg.inv(kinetic_propagator(m)) / dbar(m, x)[None, :]
    runs = {"B": arnoldi(B, v0, steps), "Binv": arnoldi(Binv, v0, steps)}
    top = {}
    for key, (H, _, k) in runs.items():
        top[key] = float(np.abs(np.linalg.eigvals(H[:k, :k])).max())
    return 1.0 / ((1.0 + margin) * top["Binv"]), (1.0 + margin) * top["B"], runs


def kpm_plan(m: Model, x, a1=1.0, a2=1.0, bounds=None):
    """Per omega < T/2: (N_P, c_m); the mirrored half uses conj (App. C B).
    bounds: (bmin, bmax) to use instead of the deterministic spectral_bounds."""
    bmin, bmax = spectral_bounds(m, x) if bounds is None else bounds
    T = m.Ltau
    plan = []
    for w in range(T // 2):
        ph = phi_omega(T, w)
        NP = np_order(bmax - bmin, ph, a1, a2)
        plan.append((NP, chebyshev_coeffs(ph, bmin, bmax, NP)))
    return bmin, bmax, plan


def kpm_block_apply(Amat: np.ndarray, coeffs, u: np.ndarray) -> np.ndarray:
    """sum_m c_m T_m(A) u via alpha_0 = u, alpha_1 = A u,
    alpha_{m+1} = 2 A alpha_m - alpha_{m-1} (Eqs. (Minv_KPM), (alpha_recur))."""
    a_prev = u
    acc = coeffs[0] * a_prev
    if len(coeffs) == 1:
        return acc
    a_cur = Amat @ u
    acc = acc + coeffs[1] * a_cur
    for mm in range(2, len(coeffs)):
        a_next = 2.0 * (Amat @ a_cur) - a_prev
        acc = acc + coeffs[mm] * a_next
        a_prev, a_cur = a_cur, a_next
    return acc


def precond_inverse_apply(m: Model, x, v, trans: bool = False, a1=1.0, a2=1.0, bounds=None):
    """KPM approximation of P^{-1} v = U^dag Ptilde^{-1} U v (Eq. (P_change_basis), App. C D);
    with trans=True the exact transpose of that approximation,
    U^dag diag(sum conj(c_m) T_m(A^T)) U v. bounds as in kpm_plan."""
    N, T = m.N, m.Ltau
    bmin, bmax, plan = kpm_plan(m, x, a1, a2, bounds)
    db = bmax - bmin
    Bb = Bbar(m, x)
    if trans:
        Bb = Bb.T
    Amat = 2.0 * (Bb - bmin * np.eye(N)) / db - np.eye(N)
    U = U_matrix(T)
    vv = np.asarray(v, dtype=np.float64).reshape(T, N)
    vh = U @ vv                       # [omega][i]
    yh = np.zeros_like(vh)
    for w in range(T):
        if w < T // 2:
            NP, c = plan[w]
        else:
            NP, c = plan[T - 1 - w]
            c = np.conj(c)
        if trans:
            c = np.conj(c)
        yh[w] = kpm_block_apply(Amat, c, vh[w])
    y = U.conj().T @ yh
    assert np.max(np.abs(y.imag)) < 1e-9 * max(1.0, np.max(np.abs(y.real)))
    return y.real


def n_matvec_count(T: int, db: float, a1=1.0, a2=1.0) -> int:
    """N_mat-vec = 2 sum_{omega < T/2} (N_P(omega) - 1) (App. C E), with the
    unclamped floor as printed."""
    tot = 0
    for w in range(T // 2):
        tot += int(np.floor(db * (a1 / phi_omega(T, w) + a2))) - 1
    return 2 * tot


def n_matvec_bound(T: int, db: float, a1=1.0, a2=1.0) -> float:
    """Upper bound of Eq. (N_mv_bound)."""
    gamma = 0.5772156649015329
    return T * db * (a1 / np.pi * (gamma + np.log(2 * T)) + a2) - T


# ----------------------------------------------------------------------------
# Preconditioned CG, in the plain textbook form (Sec. VI A)
# ----------------------------------------------------------------------------
def pcg(m: Model, x, b, tol=1e-10, max_iter=5000, precond=False, a1=1.0, a2=1.0):
    """CG on M^T M v = b; with precond=True the preconditioner z = P^{-1} P^{-T} r
    (P^{-1} from the KPM approximation). Returns (v, iterations)."""
    M = fermion_matrix(m, x)
    A = M.T @ M
    bb = np.asarray(b, dtype=np.float64).reshape(-1)
    v = np.zeros_like(bb)
    r = bb.copy()

    def prec(r):
        if not precond:
            return r
        t = precond_inverse_apply(m, x, r, trans=True, a1=a1, a2=a2).reshape(-1)
        return precond_inverse_apply(m, x, t, trans=False, a1=a1, a2=a2).reshape(-1)

    z = prec(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(bb)
    for k in range(1, max_iter + 1):
        q = A @ p
        a = rz / (p @ q)
        v = v + a * p
        r = r - a * q
        if np.linalg.norm(bb - A @ v) / nb < tol:
            return v.reshape(m.Ltau, m.N), k
        z = prec(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return v.reshape(m.Ltau, m.N), max_iter


# ----------------------------------------------------------------------------
# Stochastic Green-function measurements (Sec. V)
# ----------------------------------------------------------------------------
def green_matrix(m: Model, x) -> np.ndarray:
    """G = M^{-1} (Sec. V A)."""
    return np.linalg.inv(fermion_matrix(m, x))


def extend(v) -> np.ndarray:
    """Q v = [v; -v] along tau (Eq. (G_def-1)): [T][N] -> [2T][N]."""
    v = np.asarray(v)
    return np.concatenate([v, -v], axis=0)


def _shift(v2: np.ndarray, L: int, dl: int, dy: int, dx: int) -> np.ndarray:
    """w_{(l,iy,ix)} = v_{(l+dl, iy+dy, ix+dx)} on the periodic doubled domain."""
    T2 = v2.shape[0]
    g = v2.reshape(T2, L, L)
    return np.roll(g, shift=(-dl, -dy, -dx), axis=(0, 1, 2))


def cross_corr_direct(a2: np.ndarray, b2: np.ndarray, L: int) -> np.ndarray:
    """(a star b)_Delta = sum_i a_i b_{i+Delta} over the periodic doubled
    domain (Eq. (cross_corr)), by direct summation. Output [2T][L][L] indexed
    [dl][dy][dx]."""
    T2 = a2.shape[0]
    out = np.zeros((T2, L, L))
    ag = a2.reshape(T2, L, L)
    for dl in range(T2):
        for dy in range(L):
            for dx in range(L):
                out[dl, dy, dx] = np.sum(ag * _shift(b2, L, dl, dy, dx))
    return out


def cross_corr_at(a2: np.ndarray, b2: np.ndarray, L: int, deltas) -> np.ndarray:
    """(a star b)_Delta = sum_i a_i b_{i+Delta} (Eq. (cross_corr)) over the
    periodic doubled domain, by direct summation at the listed offsets only.
    deltas: sequence of (dl, dy, dx). Returns one value per offset."""
    return np.array([np.sum(a2.reshape(-1) * _shift(b2, L, dl, dy, dx).reshape(-1))
                     for dl, dy, dx in deltas])


def green_average_at(m: Model, xi, Gxi, deltas) -> np.ndarray:
    """green_average at the listed offsets (dl, dy, dx) only:
    (1/N_rv) sum_n (1/(2 N T)) (Q xi_n star Q G xi_n)_Delta (Eqs. (G_avg-1),
    (G_def-1), (cross_corr), (G_approx_better))."""
    out = np.zeros(len(deltas))
    for v, gv in zip(xi, Gxi):
        out += cross_corr_at(extend(v), extend(gv), m.L, deltas)
    return out / (2.0 * m.n * len(xi))


def four_point_pairs_at(m: Model, xi, Gxi, deltas) -> np.ndarray:
    """four_point_pairs at the listed offsets only: the three pair-averaged
    Wick products of Sec. V C (Eq. (GG_approx_better)) over all pairs n < k,
    each by direct summation. Returns [3][len(deltas)]."""
    a = [extend(v) for v in xi]
    b = [extend(v) for v in Gxi]
    R = len(xi)
    out = np.zeros((3, len(deltas)))
    npairs = 0
    for n in range(R):
        for k in range(n + 1, R):
            out[0] += cross_corr_at(a[n] * a[k], b[n] * b[k], m.L, deltas)
            out[1] += cross_corr_at(a[n] * b[n], a[k] * b[k], m.L, deltas)
            out[2] += cross_corr_at(a[n] * b[k], a[k] * b[n], m.L, deltas)
            npairs += 1
    return out / (2.0 * m.n * npairs)


def green_average(m: Model, x, xi, Gxi=None) -> np.ndarray:
    """Space-time averaged Green function estimate, Eqs. (G_avg-1), (G_def-1), (cross_corr), averaged
    over the probe vectors (Eq. (G_approx_better)): (1/N_rv) sum_n (1/(2 N T)) (a_n star b_n)
    with a = Q xi, b = Q G xi. xi: [n_rv][T][N]."""
    xi = np.asarray(xi)
    if Gxi is None:
        G = green_matrix(m, x)
        Gxi = np.array([(G @ v.reshape(-1)).reshape(m.Ltau, m.N) for v in xi])
    out = np.zeros((2 * m.Ltau, m.L, m.L))
    for v, gv in zip(xi, Gxi):
        out += cross_corr_direct(extend(v), extend(gv), m.L)
    return out / (2.0 * m.n * len(xi))


def green_average_exact(m: Model, x) -> np.ndarray:
    """(1/(N T)) sum_{i in the original domain} G^ext_{i+Delta, i} (Eq. (G_avg-1)),
    from the dense G^ext = Q G Q^T."""
    N, T, L = m.N, m.Ltau, m.L
    G = green_matrix(m, x)
    Q = np.vstack([np.eye(N * T), -np.eye(N * T)])
    Gx = Q @ G @ Q.T
    out = np.zeros((2 * T, L, L))
    for l in range(T):
        for iy in range(L):
            for ix in range(L):
                i = l * N + site(ix, iy, L)
                for dl in range(2 * T):
                    for dy in range(L):
                        for dx in range(L):
                            j = ((l + dl) % (2 * T)) * N + site(ix + dx, iy + dy, L)
                            out[dl, dy, dx] += Gx[j, i]
    return out / (N * T)


def four_point_pairs(m: Model, x, xi, Gxi=None) -> np.ndarray:
    """Pair-averaged Wick 4-point estimators (Sec. V C products, Eq. (GG_approx_better)), over all
    pairs n < m of probe vectors, each normalised like the 2-point average:
    [0]: (xi_n . xi_m) star (Gxi_n . Gxi_m)
    [1]: (xi_n . Gxi_n) star (xi_m . Gxi_m)
    [2]: (xi_n . Gxi_m) star (xi_m . Gxi_n)
    ('.' is the element-wise product of the doubled vectors). Output [3][2T][L][L]."""
    xi = np.asarray(xi)
    if Gxi is None:
        G = green_matrix(m, x)
        Gxi = np.array([(G @ v.reshape(-1)).reshape(m.Ltau, m.N) for v in xi])
    a = [extend(v) for v in xi]
    b = [extend(v) for v in Gxi]
    R = len(xi)
    out = np.zeros((3, 2 * m.Ltau, m.L, m.L))
    npairs = 0
    for n in range(R):
        for k in range(n + 1, R):
            out[0] += cross_corr_direct(a[n] * a[k], b[n] * b[k], m.L)
            out[1] += cross_corr_direct(a[n] * b[n], a[k] * b[k], m.L)
            out[2] += cross_corr_direct(a[n] * b[k], a[k] * b[n], m.L)
            npairs += 1
    return out / (2.0 * m.n * npairs)


# ----------------------------------------------------------------------------
# Observables from the Green function (Sec. II, Eq. (Scdw) and P_s)
# ----------------------------------------------------------------------------
def observables_exact(m: Model, x) -> dict:
    """Per-configuration observables of the spin-degenerate model from the
    dense equal- and unequal-time G = M^{-1} (G_{ab} = <c_a c_b^dag>), by Wick's
    theorem for each spin (the two spins see the same x and are independent):
      <n> = 2 (1 - mean_a G_aa);
      C(r) = (1/(N T)) sum_{i, tau} <n_{i+r,tau} n_{i,tau}>, with
      <n_a n_b> = 4 (1 - G_aa)(1 - G_bb) + 2 (delta_ab - G_ba) G_ab;
      S_cdw = sum_r (-1)^(rx + ry) C(r)  (Eq. (Scdw));
      P_s = (dtau / (N T)) sum_{tau'} sum_l sum_{r, r'} G_{(r, tau'+l), (r', tau')}^2,
    the pair susceptibility with the imaginary-time integral as a sum over
    the T slices (G squared removes the antiperiodic sign)."""
    N, T, L = m.N, m.Ltau, m.L
    G = green_matrix(m, x)
    dG = np.diag(G).reshape(T, N)
    out_C = np.zeros((L, L))
    for tau in range(T):
        for iy in range(L):
            for ix in range(L):
                a = tau * N + site(ix, iy, L)
                for dy in range(L):
                    for dx in range(L):
                        b = tau * N + site(ix + dx, iy + dy, L)
                        nn = 4.0 * (1.0 - G[a, a]) * (1.0 - G[b, b]) + \
                            2.0 * ((1.0 if a == b else 0.0) - G[b, a]) * G[a, b]
                        out_C[dy, dx] += nn
    out_C /= N * T
    sign = np.array([[(-1.0) ** (dx + dy) for dx in range(L)] for dy in range(L)])
    ps = 0.0
    for t1 in range(T):
        for t0 in range(T):
            blk = G[t1 * N:(t1 + 1) * N, t0 * N:(t0 + 1) * N]
            ps += float(np.sum(blk * blk))
    ps *= m.dtau / (N * T)
    return {"density": 2.0 * (1.0 - float(np.mean(dG))), "C": out_C,
            "S_cdw": float(np.sum(sign * out_C)), "P_s": ps}


def observables_from_estimates(m: Model, G2, G4) -> dict:
    """The same observables from the space-time averaged 2-point function
    G2 [2T][L][L] and the pair-averaged Wick products G4 [3][2T][L][L]
    (Sec. V; index [dl][dy][dx]): g0 = G2[0, 0, 0] estimates mean G_aa;
    G4[1][0] (xi.Gxi star xi'.Gxi') estimates mean G_aa G_bb, G4[2][0]
    (xi.Gxi' star xi'.Gxi) mean G_ab G_ba, G4[0][l] (xi.xi' star Gxi.Gxi')
    mean G_{b,a}^2 at slice difference l."""
    G2 = np.asarray(G2)
    G4 = np.asarray(G4)
    L, T = m.L, m.Ltau
    g0 = float(G2[0, 0, 0])
    delta = np.zeros((L, L))
    delta[0, 0] = 1.0
    C = 4.0 * (1.0 - 2.0 * g0 + G4[1, 0]) + 2.0 * (delta * g0 - G4[2, 0])
    sign = np.array([[(-1.0) ** (dx + dy) for dx in range(L)] for dy in range(L)])
    ps = m.dtau * float(np.sum(G4[0, :T]))
    return {"density": 2.0 * (1.0 - g0), "C": C, "S_cdw": float(np.sum(sign * C)), "P_s": ps}


def wick_products_exact(m: Model, x) -> np.ndarray:
    """The expectations of the three pair estimators of four_point_pairs
    from the dense G^ext (no probes): [0] mean G_{i+D,i}^2, [1] mean
    G_{i,i} G_{i+D,i+D}, [2] mean G_{i,i+D} G_{i+D,i}, over the doubled
    domain (the extension's signs cancel in each product). [3][2T][L][L]."""
    N, T, L = m.N, m.Ltau, m.L
    G = green_matrix(m, x)
    Q = np.vstack([np.eye(N * T), -np.eye(N * T)])
    Gx = Q @ G @ Q.T
    out = np.zeros((3, 2 * T, L, L))
    idx = np.arange(2 * T * N)
    for dl in range(2 * T):
        for dy in range(L):
            for dx in range(L):
                l, r = idx // N, idx % N
                iy, ix = r // L, r % L
                j = ((l + dl) % (2 * T)) * N + ((iy + dy) % L) * L + (ix + dx) % L
                out[0, dl, dy, dx] = np.mean(Gx[j, idx] ** 2)
                out[1, dl, dy, dx] = np.mean(Gx[idx, idx] * Gx[j, j])
                out[2, dl, dy, dx] = np.mean(Gx[idx, j] * Gx[j, idx])
    return out
