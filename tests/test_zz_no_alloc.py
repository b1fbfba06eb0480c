"""The allocation-free entry point fermion_matvec_static, for callers that
cannot allocate device memory (their memory belongs to another allocator, or
they must avoid the synchronisation cudaMalloc can imply), against the
context-based fermion_matvec on the same inputs, through the C ABI.

Collected last on purpose (tests run in file order), so that a failure here
stops a `-x` run only after every other test has run. Two calls in a row
check that the shared static scratch carries nothing over between calls.
"""
import numpy as np
import pytest
import torch

import holstein_inputs as hi

pytestmark = pytest.mark.gpu

hg = pytest.importorskip("paper_2203_01291_gb300")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_static_scratch_operator_matches_context_operator():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hg.build.build()
    torch.cuda.set_device(0)
    w = hi.WORKLOADS["hmc16"]                      # N*T = 40960; 2 rhs fit the scratch
    params = hg.hol_params(w.L, w.Ltau, w.dtau, w.t, w.mu, w.alpha, w.omega0, 2)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        for call, (seed, op) in enumerate(((11, hg.HOL_OP_MTM), (12, hg.HOL_OP_MTM),
                                           (13, hg.HOL_OP_M), (14, hg.HOL_OP_MT))):
            x = torch.tensor(hi.phonon_field(w, seed=seed), device="cuda")
            v = torch.tensor(hi.gaussian_vectors(w, 2, seed=seed + 100), device="cuda")
            ctx.set_field(x)
            ref = torch.empty_like(v)
            ctx.fermion_matvec(op, v, ref)
            out = torch.full_like(v, float("nan"))
            hg.fermion_matvec_static(params, x, op, v, out, 2)
            torch.cuda.synchronize()
            assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-13, (call, op)


def test_static_scratch_operator_with_chemical_potential():
    """mu != 0 and a coupling other than 1: a sign or factor error in the
    exp(-dtau (alpha x - mu)) table of the static path would show here (the
    hmc16 workload above has mu = 0). Two calls in a row, all three ops."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hg.build.build()
    torch.cuda.set_device(0)
    w = hi.Workload("static_mu", L=12, Ltau=24, alpha=0.8, mu=0.35, omega0=1.0, x_std=1.0,
                    seed=61)
    params = hg.hol_params(w.L, w.Ltau, w.dtau, w.t, w.mu, w.alpha, w.omega0, 3)
    with hg.Context.from_workload(w, max_rhs=3) as ctx:
        x = torch.tensor(hi.phonon_field(w), device="cuda")
        ctx.set_field(x)
        for call in range(2):
            for op in (hg.HOL_OP_M, hg.HOL_OP_MT, hg.HOL_OP_MTM):
                v = torch.tensor(hi.gaussian_vectors(w, 3, seed=70 + 3 * call + op),
                                 device="cuda")
                ref = torch.empty_like(v)
                ctx.fermion_matvec(op, v, ref)
                out = torch.full_like(v, float("nan"))
                hg.fermion_matvec_static(params, x, op, v, out, 3)
                torch.cuda.synchronize()
                assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-13, (call, op)


def test_static_scratch_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    w = hi.WORKLOADS["big32"]                      # N*T = 204800: 5 M^T M rhs exceed 2^20
    params = hg.hol_params(w.L, w.Ltau, w.dtau, w.t, w.mu, w.alpha, w.omega0, 8)
    x = torch.zeros(w.Ltau, w.N, dtype=torch.float64, device="cuda")
    v = torch.zeros(8, w.Ltau, w.N, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HolError) as e:
        hg.fermion_matvec_static(params, x, hg.HOL_OP_MTM, v, torch.empty_like(v), 8)
    assert e.value.code == hg._abi.HOL_EINVAL
