"""The beta2 > 0 step (MFMC_ALGO_ACTIVE_SET) against the FP64 oracle (oracle/beta2_oracle.py).

Both sides work in FP64 from the same FP32-rounded initial field and solve each step's
resolvent equation to max |F| <= 1e-11 (GPU: Newton with preconditioned CG; oracle: Newton with
sparse direct solves), so a step agrees to about 1e-11 / c_gamma; over k steps the map is
Lipschitz with constant about 1, so fields agree to k * 1e-9 and the OoI to 1e-8 relative.
The GPU forms the explicit disc sum directly for discs of fewer than 100 points and through an
FP64 cuFFT convolution otherwise; the cases below cover both sides."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import beta2_oracle as B2

pytestmark = pytest.mark.gpu


def gpu_solve(mf, g, seeds):
    import torch
    ns, n = len(seeds), g.n
    u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
    uT = torch.empty_like(u0)
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    ubar = torch.empty(ns, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mf.mfmc_sample_eps(g, seeds), dtype=torch.float64, device="cuda")
    mf.mfmc_init_fields(g, seeds, u0)
    mf.mfmc_solve_fields(g, u0, ns, eps=eps, uT=uT, ooi=ooi, ubar=ubar)
    torch.cuda.synchronize()
    return (u0.cpu().numpy().astype(np.float64), uT.cpu().numpy().astype(np.float64), ooi.cpu().numpy(),
            ubar.cpu().numpy())


CASES = [dict(n=32, delta=3 / 32, kernel=0, tau=0.01), dict(n=64, delta=4 / 64, kernel=0, tau=0.01),
         dict(n=64, delta=0.125, kernel=1, delta_hf=0.25, tau=0.01)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_active_set_one_step_elementwise(gpu_lib, case):
    mf = gpu_lib
    kw = dict(CASES[case], eps=0.04219, nsteps=1, ic=2, beta2=0.05)
    g = mf.Model(algo=mf.ALGO_ACTIVE_SET, **kw)
    okw = {k: v for k, v in kw.items() if k != "beta2"}
    o = O.OracleModel(**okw)
    u0, uT, _, _ = gpu_solve(mf, g, np.arange(3, dtype=np.uint64) + 11 * case)
    for i in range(3):
        ref, _, _ = B2.step(o, u0[i], 0.04219, 0.05)
        assert np.abs(uT[i] - ref).max() <= 1e-7   # uT is FP32: the FP64 fields agree to ~1e-11
        assert np.abs(uT[i]).max() <= 1.0
    assert (uT == -1.0).any() and (uT == 1.0).any()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_active_set_solve_matches_oracle(gpu_lib, ooi_errors, case):
    mf = gpu_lib
    steps = 15
    kw = dict(CASES[case], eps=0.04219, nsteps=steps, ic=2, beta2=0.05)
    g = mf.Model(**kw)                        # AUTO picks the active-set solver
    okw = {k: v for k, v in kw.items() if k != "beta2"}
    o = O.OracleModel(**okw)
    seeds = np.arange(2, dtype=np.uint64) + 100 + case
    _, uT, f, ubar = gpu_solve(mf, g, seeds)
    assert g.info().algo == mf.ALGO_ACTIVE_SET
    newton, cg = mf.mfmc_model_solver_stats(g)
    # per sample and step: the start, a few corrections and the confirming residual; each FP32
    # correction a few multigrid-preconditioned CG iterations
    assert 2 * len(seeds) * steps <= newton <= 12 * len(seeds) * steps
    assert newton - len(seeds) * steps <= cg <= 30 * (newton - len(seeds) * steps)
    for i, s in enumerate(seeds):
        fr, mean, ur, _ = B2.solve_sample(o, int(s), 0.05, steps)
        ooi_errors.add("beta2 = 0.05 active-set step (nuclei IC; direct and spectral disc sums)", f[i], fr,
                       ubar[i], mean, np.abs(uT[i] - ur).max())
        assert abs(f[i] - fr) <= 1e-8 * fr
        assert abs(ubar[i] - mean) <= 2e-8
        assert np.abs(uT[i] - ur).max() <= 1e-6


def test_active_set_small_beta2_approaches_the_projection_step(gpu_lib):
    # beta2 -> 0: the step tends to the beta2 = 0 projection step (difference O(beta2))
    mf = gpu_lib
    kw = dict(n=64, delta=4 / 64, eps=0.03, tau=5e-3, nsteps=10, ic=2)
    ga = mf.Model(beta2=1e-9, **kw)
    g0 = mf.Model(algo=mf.ALGO_DIRECT, **kw)
    seeds = np.arange(3, dtype=np.uint64) + 5
    _, ua, fa, _ = gpu_solve(mf, ga, seeds)
    _, u0, f0, _ = gpu_solve(mf, g0, seeds)
    assert np.abs(fa - f0).max() <= 1e-6
    assert np.abs(ua - u0).max() <= 1e-4


def test_active_set_stationary_batch_and_rejections(gpu_lib):
    import torch
    mf = gpu_lib
    kw = dict(n=32, delta=3 / 32, eps=0.03, tau=0.01, nsteps=5, ic=2, beta2=0.05)
    g = mf.Model(**kw)
    for c in (1.0, -1.0):
        u0 = torch.full((2, 32, 32), c, dtype=torch.float32, device="cuda")
        uT = torch.empty_like(u0)
        ooi = torch.empty(2, dtype=torch.float64, device="cuda")
        mf.mfmc_solve_fields(g, u0, 2, uT=uT, ooi=ooi)
        torch.cuda.synchronize()
        assert torch.all(uT == c)
    # the batch call (seeds in, OoIs out) against the oracle
    o = O.OracleModel(**{k: v for k, v in kw.items() if k != "beta2"})
    seeds = np.arange(3, dtype=np.uint64) + 900
    f, _ = mf.mfmc_solve_batch([g] * 3, seeds)
    for i, s in enumerate(seeds):
        fr, _, _, _ = B2.solve_sample(o, int(s), 0.05, 5)
        assert abs(f[i] - fr) <= 1e-8 * fr
    with pytest.raises(mf.MfmcError):      # the mixed-fidelity call serves beta2 = 0 only
        mf.mfmc_solve_batch_mixed([g], [1])


SUM_CASES = [dict(n=48, delta=5 / 48, kernel=0),                 # 81 disc points: direct sum
             dict(n=48, delta=6 / 48, kernel=0),                 # 113 points: own transforms, 48 = 4 4 3
             dict(n=88, delta=0.1875, kernel=1, delta_hf=0.25),  # delta/h = 16.5: own, 88 = 4 2 11
             dict(n=52, delta=6 / 52, kernel=0),                 # 52 = 4 13: through cuFFT
             dict(n=40, delta=6 / 40, kernel=1, delta_hf=0.25)]  # 113 points: own, 40 = 5 4 2


@pytest.mark.parametrize("case", range(len(SUM_CASES)))
def test_active_set_direct_and_spectral_disc_sums(gpu_lib, ooi_errors, case):
    mf = gpu_lib
    steps = 8
    kw = dict(SUM_CASES[case], eps=0.04219, tau=0.01, nsteps=steps, ic=2, beta2=0.05)
    g = mf.Model(**kw)
    o = O.OracleModel(**{k: v for k, v in kw.items() if k != "beta2"})
    seeds = np.arange(3, dtype=np.uint64) + 300 + 7 * case
    u0, uT, f, ubar = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, mean, ur, _ = B2.solve_sample(o, int(s), 0.05, steps)
        ooi_errors.add("beta2 = 0.05 active-set step (nuclei IC; direct and spectral disc sums)", f[i], fr,
                       ubar[i], mean, np.abs(uT[i] - ur).max())
        assert abs(f[i] - fr) <= 1e-8 * fr
        assert abs(ubar[i] - mean) <= 2e-8
        assert np.abs(uT[i] - ur).max() <= 1e-6
    one = mf.Model(**dict(kw, nsteps=1))
    u0, u1, _, _ = gpu_solve(mf, one, seeds[:1])
    ref, _, _ = B2.step(o, u0[0], 0.04219, 0.05)
    assert np.abs(u1[0] - ref).max() <= 1e-7


def test_newton_bound_reports_timeout_and_the_model_recovers(gpu_lib):
    # Failure detection in its safe form: an iteration bound set low by the host.  Every step
    # of these nuclei fields needs several Newton passes, so a bound of one pass is reached; the
    # kernel stops the sample and returns normally, the batch call reports MFMC_ETIMEOUT, and the
    # next call on the same model (default bounds again) runs on a usable context and matches
    # the oracle.
    mf = gpu_lib
    kw = dict(n=32, delta=3 / 32, eps=0.03, tau=0.01, nsteps=5, ic=2, beta2=0.05)
    g = mf.Model(**kw)
    seeds = np.arange(3, dtype=np.uint64) + 640
    g.set_iteration_limits(newton_max=1)
    with pytest.raises(mf.MfmcError) as e:
        mf.mfmc_solve_batch([g] * 3, seeds)
    assert e.value.status == mf.MFMC_ETIMEOUT
    with pytest.raises(mf.MfmcError) as e:
        g.set_iteration_limits(newton_max=-1)
    assert e.value.status == mf.MFMC_EINVAL
    g.set_iteration_limits()                  # 0, 0: the defaults
    f, _ = mf.mfmc_solve_batch([g] * 3, seeds)
    o = O.OracleModel(**{k: v for k, v in kw.items() if k != "beta2"})
    for i, s in enumerate(seeds):
        fr, _, _, _ = B2.solve_sample(o, int(s), 0.05, 5)
        assert abs(f[i] - fr) <= 1e-8 * fr
    # a CG bound of one iteration only makes each correction coarser: the Newton passes still
    # converge to the same tolerance within their default bound
    g.set_iteration_limits(cg_max=1)
    f1, _ = mf.mfmc_solve_batch([g] * 3, seeds)
    assert np.abs(f1 - f).max() <= 1e-8
