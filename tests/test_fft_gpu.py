"""The spectral (cuFFT) form of the disc sum, MFMC_ALGO_FFT, against the FP64 oracle.

The transforms round in FP32: the disc sum S of magnitude <= |D| max|u| carries an absolute
error of a few FP32 ulps of that magnitude, which the update scales by c1 (1e-5 .. 1e-2 here),
so the per-step bound of the other kernels, 4e-6 max|u|, still holds."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

GAUSS = dict(kernel=1, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, ic=2)


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


@pytest.mark.parametrize("n,R", [(64, 4), (68, 3), (128, 8), (256, 32)])
def test_fft_one_step_elementwise(gpu_lib, n, R):
    mf = gpu_lib
    kw = dict(n=n, delta=R / n, eps=0.03, tau=5e-3, nsteps=1, ic=2)
    g = mf.Model(algo=mf.ALGO_FFT, **kw)
    o = O.OracleModel(**kw)
    u0, uT, _, _ = gpu_solve(mf, g, np.arange(3, dtype=np.uint64) + n)
    for i in range(3):
        ref = o.step(u0[i], 0.03)
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max())


@pytest.mark.parametrize("inv_h,delta", [(128, 0.25), (88, 0.1875), (64, 0.125)])
def test_fft_paper_gaussian_models(gpu_lib, inv_h, delta):
    # Table 1's models 1, 3 (delta/h = 16.5) and 9: Gaussian weights, 12 steps of tau = 0.01
    mf = gpu_lib
    steps = 12
    g = mf.Model(n=inv_h, delta=delta, nsteps=steps, algo=mf.ALGO_FFT, **GAUSS)
    o = O.OracleModel(n=inv_h, delta=delta, nsteps=steps, **GAUSS)
    seeds = np.arange(2, dtype=np.uint64) + 17
    _, uT, f, _ = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert np.abs(uT[i] - ur).max() <= steps * 4e-6 * math.exp(0.12)


def test_fft_matches_the_prefix_kernel_over_a_solve(gpu_lib):
    # 256 x 256, R = 8, 200 steps, nuclei IC: the spectral and the register-tiled disc sums
    # give the same OoI to the accumulated rounding of the two FP32 forms
    mf = gpu_lib
    kw = dict(n=256, delta=8 / 256, eps=0.03, tau=5e-3, nsteps=200, ic=2)
    gf = mf.Model(algo=mf.ALGO_FFT, **kw)
    gt = mf.Model(algo=mf.ALGO_PREFIX_TMA, **kw)
    seeds = np.arange(8, dtype=np.uint64) + 90
    _, uf, ff, _ = gpu_solve(mf, gf, seeds)
    _, ut, ft, _ = gpu_solve(mf, gt, seeds)
    assert np.abs(ff - ft).max() <= 1e-5 * ft.max()
    assert np.abs(uf - ut).max() <= 200 * 4e-6 * math.exp(1.0)


def test_fft_batch_size_changes_and_rejections(gpu_lib):
    # the plans follow the batch size; a collar model cannot take the spectral path
    mf = gpu_lib
    kw = dict(n=64, delta=4 / 64, eps=0.03, tau=5e-3, nsteps=5, ic=2)
    g = mf.Model(algo=mf.ALGO_FFT, **kw)
    o = O.OracleModel(**kw)
    for ns in (3, 5, 3):
        seeds = np.arange(ns, dtype=np.uint64) + 7 * ns
        _, _, f, _ = gpu_solve(mf, g, seeds)
        for i, s in enumerate(seeds):
            fr, _, _, _ = o.solve_sample(int(s))
            assert abs(f[i] - fr) <= 1e-5 * fr
    with pytest.raises(mf.MfmcError):
        mf.Model(algo=mf.ALGO_FFT, bc=mf.BC_COLLAR, bc_value=-1.0, **kw)
