"""The seeded input generators shared by the oracle and the GPU path (no GPU):
determinism, shapes and layout, and the distributions the workloads state."""
import numpy as np
import pytest

import holstein_inputs as hi


@pytest.mark.parametrize("name", sorted(hi.WORKLOADS))
def test_workload_fields_have_the_stated_law(name):
    w = hi.WORKLOADS[name]
    x = hi.phonon_field(w)
    assert x.shape == (w.Ltau, w.N) and x.dtype == np.float64 and x.flags.c_contiguous
    assert np.array_equal(x, hi.phonon_field(w))            # seeded
    n = x.size
    assert abs(x.mean() - w.x_shift) < 5 * w.x_std / np.sqrt(n)
    assert abs(x.std() / w.x_std - 1.0) < 5 / np.sqrt(2 * n)
    assert abs(w.beta - w.dtau * w.Ltau) < 1e-15


def test_draws_are_seeded_distinct_and_well_formed():
    w = hi.WORKLOADS["tiny"]
    R = hi.gaussian_vectors(w, 3, seed=1)
    assert R.shape == (3, w.Ltau, w.N) and R.flags.c_contiguous
    assert np.array_equal(R, hi.gaussian_vectors(w, 3, seed=1))
    assert not np.array_equal(R, hi.gaussian_vectors(w, 3, seed=2))
    xi = hi.z2_vectors(w, 64, seed=3)
    assert set(np.unique(xi)) == {-1.0, 1.0}
    # <xi_i xi_j> = delta_ij (Sec. V B): the sample second moment is close to I
    X = xi.reshape(64, -1)
    assert abs((X * X).mean() - 1.0) == 0.0
    assert abs((X[:, :-1] * X[:, 1:]).mean()) < 5 / np.sqrt(X[:, 1:].size)
    u = hi.uniforms(1000, seed=4)
    assert u.min() >= 0.0 and u.max() < 1.0
    v = hi.site_vector(w, seed=5)
    assert v.shape == (w.N,)


def test_ar1_field_has_the_stated_lag_one_correlation():
    w = hi.Workload("a", L=16, Ltau=400, x_std=1.5, x_shift=0.2, seed=9)
    corr = 0.5
    x = hi.phonon_field_ar1(w, corr)
    rho = np.exp(-w.dtau / corr)
    z = (x - w.x_shift) / w.x_std
    r1 = (z[1:] * z[:-1]).mean() / (z * z).mean()
    assert abs(r1 - rho) < 0.02
    assert abs(z.std() - 1.0) < 0.05


def test_chain_batch_layout():
    ws = hi.chain_workloads(8, 120)
    assert len(ws) == 48
    assert sorted({w.L for w in ws}) == list(hi.CHAIN_SIZES)
    assert len({w.seed for w in ws}) == 48 and all(w.Ltau == 120 for w in ws)


def test_prior_field_has_the_free_phonon_covariance():
    """phonon_field_prior samples exp(-S_B): the sample covariance along tau
    matches the inverse of the action's quadratic form (built densely here
    from the stencil), and S_B averages N T / 2 (equipartition)."""
    w = hi.Workload("p", L=32, Ltau=20, omega0=0.7, dtau=0.1, seed=12)
    x = hi.phonon_field_prior(w)
    assert x.shape == (w.Ltau, w.N) and np.array_equal(x, hi.phonon_field_prior(w))
    T, dt = w.Ltau, w.dtau
    A = np.zeros((T, T))
    for t in range(T):
        A[t, t] += dt * w.omega0 ** 2 + 2.0 / dt
        A[t, (t + 1) % T] -= 1.0 / dt
        A[(t + 1) % T, t] -= 1.0 / dt
    C = np.linalg.inv(A)
    emp = x @ x.T / w.N
    assert np.abs(emp - C).max() < 6 * C.max() * np.sqrt(2.0 / w.N)
    SB = 0.5 * dt * np.sum(w.omega0 ** 2 * x * x + ((np.roll(x, -1, axis=0) - x) / dt) ** 2)
    assert abs(SB / (w.N * T / 2) - 1.0) < 5 * np.sqrt(2.0 / (w.N * T))
