"""The paper's own nine models (Section 4, Table 1): truncated Gaussian kernel with
delta_hf = 0.25, eps^2 = 0.00178, tau = 0.01, the four-nuclei initial condition, meshes
h in {1/128, 1/88, 1/64} and horizons delta in {0.25, 0.1875, 0.125}, on the periodic lattice
with beta2 = 0.  h = 1/88 with delta = 0.1875 gives the non-integer delta/h = 16.5, served by
the generic kernel with the disc { |z| <= 16.5 }.  GPU against the FP64 oracle; tolerances
as in the periodic parity tests."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

# Table 1's model numbering: (1/h, delta)
PAPER_MODELS = [(128, 0.25), (128, 0.1875), (88, 0.1875), (88, 0.25), (128, 0.125), (88, 0.125),
                (64, 0.1875), (64, 0.25), (64, 0.125)]
GAUSS = dict(kernel=1, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, ic=2)


def gpu_solve(mf, g, seeds):
    import torch
    ns, n = len(seeds), g.n
    u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
    uT = torch.empty_like(u0)
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mf.mfmc_sample_eps(g, seeds), dtype=torch.float64, device="cuda")
    mf.mfmc_init_fields(g, seeds, u0)
    mf.mfmc_solve_fields(g, u0, ns, eps=eps, uT=uT, ooi=ooi)
    torch.cuda.synchronize()
    return u0.cpu().numpy().astype(np.float64), uT.cpu().numpy().astype(np.float64), ooi.cpu().numpy()


@pytest.mark.parametrize("path", ["DIRECT", "PLAIN"])
def test_noninteger_radius_constant_kernel_one_step_elementwise(gpu_lib, path):
    mf = gpu_lib
    n, delta = 64, 4.5 / 64
    g = mf.Model(n=n, delta=delta, eps=0.03, tau=5e-3, nsteps=1, ic=2, algo=getattr(mf, "ALGO_" + path))
    o = O.OracleModel(n=n, delta=delta, eps=0.03, tau=5e-3, nsteps=1, ic=2)
    assert g.info().disc_points == len(o.offsets()[0])
    u0, uT, _ = gpu_solve(mf, g, np.arange(3, dtype=np.uint64) + 40)
    for i in range(3):
        ref = o.step(u0[i], 0.03)
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max())


def test_noninteger_radius_gaussian_solve_and_auto_choice(gpu_lib):
    # model 3 of Table 1: h = 1/88, delta = 0.1875 (delta/h = 16.5), 20 steps
    mf = gpu_lib
    g = mf.Model(n=88, delta=0.1875, nsteps=20, **GAUSS)
    o = O.OracleModel(n=88, delta=0.1875, nsteps=20, **GAUSS)
    assert g.info().R == 16
    seeds = np.arange(2, dtype=np.uint64) + 3
    _, uT, f = gpu_solve(mf, g, seeds)
    # the candidates for a non-integer horizon: the generic direct kernel and the spectral form
    # (the disc enters only through K^); the spectral form is the faster by far here
    assert g.info().algo == mf.ALGO_SPECTRAL
    gd = mf.Model(n=88, delta=0.1875, nsteps=20, algo=mf.ALGO_DIRECT, **GAUSS)
    _, ud, fd = gpu_solve(mf, gd, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        for uu, ff in ((uT, f), (ud, fd)):
            assert abs(ff[i] - fr) <= 1e-5 * fr
            assert np.abs(uu[i] - ur).max() <= 20 * 4e-6 * math.exp(0.2)


@pytest.mark.parametrize("k", range(9))
def test_paper_model_short_solve_matches_oracle(gpu_lib, ooi_errors, k):
    mf = gpu_lib
    inv_h, delta = PAPER_MODELS[k]
    steps = 6
    g = mf.Model(n=inv_h, delta=delta, nsteps=steps, **GAUSS)
    o = O.OracleModel(n=inv_h, delta=delta, nsteps=steps, **GAUSS)
    seeds = np.arange(2, dtype=np.uint64) + 1000 + k
    _, uT, f = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        ooi_errors.add("the paper's nine Gaussian-kernel models, beta2 = 0, 6 steps, nuclei IC", f[i], fr,
                       field_err=np.abs(uT[i] - ur).max())
        assert abs(f[i] - fr) <= 1e-5 * fr, (k, i)
        assert np.abs(uT[i] - ur).max() <= steps * 4e-6 * math.exp(0.06)
