"""Concurrent independent chains of uneven size (hmc_batch, measure_batch)
give exactly the results of running each chain alone. Marked gpu."""
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
SIZES = (8, 12, 16, 10, 8, 20)


def _chains():
    return [hi.Workload(f"c{k}", L=L, Ltau=20, omega0=1.0, alpha=1.0, seed=500 + k)
            for k, L in enumerate(SIZES)]


def test_hmc_batch_equals_sequential():
    ws = _chains()
    o = hg.md_opts(0.02, 3, 2, 1.0, force_tol=1e-10, action_tol=1e-10, prec=hg.HOL_F32)
    u = hi.uniforms(len(ws), seed=9)
    ctxs = [hg.Context.from_workload(w, max_rhs=2) for w in ws]
    ref_x, ref_dh = [], []
    for w, c, uk in zip(ws, ctxs, u):
        x = torch.tensor(hi.phonon_field(w), device=DEV)
        R = torch.tensor(hi.gaussian_vectors(w, 2, seed=w.seed + 1), device=DEV)
        Rp = torch.tensor(hi.gaussian_vectors(w, 1, seed=w.seed + 2)[0], device=DEV)
        acc, dh, _ = c.fourier_accel_leapfrog(x, R, Rp, o, uk)
        ref_x.append(x.cpu().numpy())
        ref_dh.append(dh)
    xs = [torch.tensor(hi.phonon_field(w), device=DEV) for w in ws]
    Rs = [torch.tensor(hi.gaussian_vectors(w, 2, seed=w.seed + 1), device=DEV) for w in ws]
    Rps = [torch.tensor(hi.gaussian_vectors(w, 1, seed=w.seed + 2)[0], device=DEV) for w in ws]
    acc, dh = hg.hmc_batch(ctxs, xs, Rs, Rps, o, u, n_threads=3)
    for k in range(len(ws)):
        assert dh[k] == ref_dh[k]
        assert np.array_equal(xs[k].cpu().numpy(), ref_x[k])
    for c in ctxs:
        c.close()


def test_measure_batch_equals_sequential():
    ws = _chains()[:4]
    opts = hg.hol_cg_opts(1e-10, 100000, 0, hg.HOL_F64, 50, 10)
    ctxs = [hg.Context.from_workload(w, max_rhs=4) for w in ws]
    xis, G2s, Gxis, refs = [], [], [], []
    for w, c in zip(ws, ctxs):
        c.set_field(torch.tensor(hi.phonon_field(w), device=DEV))
        xi = torch.tensor(hi.z2_vectors(w, 6, seed=w.seed + 3), device=DEV)
        Gxi = torch.empty_like(xi)
        G2 = torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=DEV)
        c.stochastic_measure(xi, Gxi, G2, tol=1e-10)
        refs.append(G2.cpu().numpy())
        xis.append(xi)
        Gxis.append(torch.empty_like(xi))
        G2s.append(torch.empty_like(G2))
    hg.measure_batch(ctxs, xis, Gxis, G2s, opts, n_threads=4)
    for k in range(len(ws)):
        assert np.array_equal(G2s[k].cpu().numpy(), refs[k])
    for c in ctxs:
        c.close()
