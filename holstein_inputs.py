"""Seeded synthetic inputs for the Holstein HMC hot path.

This module is the only code shared by the oracle (``oracle/``) and the GPU
path (``paper_2203_01291_gb300``). It holds no arithmetic of the method: it
only names the workloads (lattice size, imaginary-time slices, couplings) and
draws the random numbers the method consumes -- phonon fields x[tau][i],
Gaussian vectors R (pseudofermion and momentum draws, Sec. III A, Eqs. (PhiSample-1), (sample_p) and
Algorithm 1), Z2 probe vectors xi (Sec. V B) and Metropolis uniforms.

Every array is FP64, C-contiguous, laid out as [..., tau, i] with the site
index i = ix + L * iy on the periodic L x L square lattice.

Workloads (the paper's benchmark parameters, Sec. II B: square lattice, t = 1,
mu = 0, dtau = 0.1):

* ``tiny``     L=4,  N=16,   Ltau=40,  beta=4,  omega0=1,   alpha=1
* ``hmc16``    L=16, N=256,  Ltau=160, beta=16, omega0=1,   alpha=1.5,
               x ~ N(0, 1/omega0^2) + 0.5
* ``big32``    L=32, N=1024, Ltau=200, beta=20, omega0=0.5, alpha=1,
               x ~ N(0, 1/omega0^2), 16 right-hand sides
* ``grad24``   L=24, N=576,  Ltau=160, beta=16, omega0=1,   alpha=1.2
* ``chains``   L in {8,...,28}, Ltau=120, beta=12, omega0=1, alpha=1

The paper samples equilibrium fields from long Markov chains; those are not
available, so i.i.d. Gaussian fields of the stated width stand in for them
(the worst case for the adiabatic preconditioner, Sec. VI B, because they are
not smooth in tau).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    Ltau: int
    dtau: float = 0.1
    t: float = 1.0
    mu: float = 0.0
    omega0: float = 1.0
    alpha: float = 1.0
    x_std: float = 1.0
    x_shift: float = 0.0
    n_rhs: int = 1
    seed: int = 1

    @property
    def N(self) -> int:
        return self.L * self.L

    @property
    def n(self) -> int:
        return self.N * self.Ltau

    @property
    def beta(self) -> float:
        return self.dtau * self.Ltau

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


WORKLOADS = {
    "tiny": Workload("tiny", L=4, Ltau=40, omega0=1.0, alpha=1.0, x_std=1.0),
    "hmc16": Workload("hmc16", L=16, Ltau=160, omega0=1.0, alpha=1.5,
                      x_std=1.0, x_shift=0.5, n_rhs=2),
    "big32": Workload("big32", L=32, Ltau=200, omega0=0.5, alpha=1.0,
                      x_std=2.0, n_rhs=16),
    "grad24": Workload("grad24", L=24, Ltau=160, omega0=1.0, alpha=1.2,
                       x_std=1.0),
}

CHAIN_SIZES = (8, 12, 16, 20, 24, 28)


def chain_workloads(per_size: int = 8, Ltau: int = 120):
    """The uneven multi-chain batch: ``per_size`` chains of each L."""
    out = []
    k = 0
    for L in CHAIN_SIZES:
        for _ in range(per_size):
            out.append(Workload(f"chain{k}", L=L, Ltau=Ltau, omega0=1.0,
                                alpha=1.0, x_std=1.0, seed=1000 + k))
            k += 1
    return out


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def phonon_field(w: Workload, seed: int | None = None) -> np.ndarray:
    """x[tau][i] ~ N(x_shift, x_std^2), i.i.d."""
    g = _rng(w.seed if seed is None else seed)
    x = g.standard_normal((w.Ltau, w.N)) * w.x_std + w.x_shift
    return np.ascontiguousarray(x, dtype=np.float64)


def phonon_field_ar1(w: Workload, corr: float, seed: int | None = None) -> np.ndarray:
    """x[tau][i]: for each site an AR(1) sequence along tau with lag-one
    correlation exp(-dtau/corr) and stationary law N(x_shift, x_std^2) (a
    generic tau-smooth input recipe; it is not periodic in tau)."""
    g = _rng(w.seed if seed is None else seed)
    rho = float(np.exp(-w.dtau / corr))
    e = g.standard_normal((w.Ltau, w.N))
    x = np.empty((w.Ltau, w.N))
    x[0] = e[0]
    s = np.sqrt(1.0 - rho * rho)
    for t in range(1, w.Ltau):
        x[t] = rho * x[t - 1] + s * e[t]
    return np.ascontiguousarray(x * w.x_std + w.x_shift, dtype=np.float64)


def phonon_field_prior(w: Workload, seed: int | None = None) -> np.ndarray:
    """x[tau][i] drawn from the free-phonon law exp(-S_B): per site, the
    Gaussian whose inverse covariance is the quadratic form of the discrete
    harmonic-oscillator action S_B = (dtau/2) sum_tau [omega0^2 x_tau^2 +
    ((x_{tau+1} - x_tau)/dtau)^2] (periodic in tau). That form is circulant
    in tau with eigenvalues q_k = dtau (omega0^2 + (2 - 2 cos(2 pi k/T))/dtau^2),
    so x = F^{-1} q^{-1/2} F R with R ~ N(0, 1) i.i.d. (numpy's FFT along
    tau), plus x_shift. tau-smooth, unlike phonon_field."""
    g = _rng(w.seed if seed is None else seed)
    R = g.standard_normal((w.Ltau, w.N))
    k = np.arange(w.Ltau)
    q = w.dtau * (w.omega0 ** 2 + (2.0 - 2.0 * np.cos(2.0 * np.pi * k / w.Ltau)) / w.dtau ** 2)
    x = np.fft.ifft(np.fft.fft(R, axis=0) / np.sqrt(q)[:, None], axis=0).real
    return np.ascontiguousarray(x + w.x_shift, dtype=np.float64)


def gaussian_vectors(w: Workload, count: int, seed: int) -> np.ndarray:
    """R[k][tau][i] ~ N(0, 1), i.i.d. (pseudofermion / momentum draws)."""
    g = _rng(seed)
    return np.ascontiguousarray(
        g.standard_normal((count, w.Ltau, w.N)), dtype=np.float64)


def site_vector(w: Workload, seed: int) -> np.ndarray:
    """v[i] ~ N(0, 1), i.i.d. over the N sites of one slice (a random start
    vector for the Arnoldi process)."""
    return np.ascontiguousarray(_rng(seed).standard_normal(w.N), dtype=np.float64)


def z2_vectors(w: Workload, count: int, seed: int) -> np.ndarray:
    """xi[k][tau][i] uniform in {-1, +1}, i.i.d. (stochastic probes)."""
    g = _rng(seed)
    bits = g.integers(0, 2, size=(count, w.Ltau, w.N))
    return np.ascontiguousarray(2.0 * bits - 1.0, dtype=np.float64)


def uniforms(count: int, seed: int) -> np.ndarray:
    """Metropolis uniforms in [0, 1)."""
    return _rng(seed).random(count)

