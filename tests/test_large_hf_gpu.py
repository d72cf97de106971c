"""The large high-fidelity configuration (1024 x 1024, delta = 32h: a 3209-point disc) against
the FP64 oracle for a bounded number of steps: the autotuned path, the plain FP32 disc sums of
the TMA tile kernel, the FP32-compensated (Kahan) sums, and the spectral forms on cuFFT and on
the library's own FFT kernels.  With |D| = 3209 FP32 adds per output
this is where accumulation error would show first; the per-step bound of the other parity
tests, 4e-6 max|u|, is the target for each of them."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def test_large_hf_fp32_kahan_and_fft_against_oracle(gpu_lib):
    import torch
    mf = gpu_lib
    n, R, steps = 1024, 32, 20
    kw = dict(n=n, delta=R / n, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=steps, ic=1, ic_amp=0.05)
    o = O.OracleModel(**kw)
    seeds = np.array([20231016 + 1000003 * 4], dtype=np.uint64)
    fr, _, ur, _ = o.solve_sample(int(seeds[0]))
    tol = steps * 4e-6 * 0.05 * math.e
    for algo in (mf.ALGO_AUTO, mf.ALGO_PREFIX_TMA, mf.ALGO_PREFIX_KAHAN, mf.ALGO_FFT, mf.ALGO_SPECTRAL):
        g = mf.Model(algo=algo, **kw)
        u0 = torch.empty((1, n, n), dtype=torch.float32, device="cuda")
        uT = torch.empty_like(u0)
        ooi = torch.empty(1, dtype=torch.float64, device="cuda")
        eps = torch.tensor(mf.mfmc_sample_eps(g, seeds), dtype=torch.float64, device="cuda")
        mf.mfmc_init_fields(g, seeds, u0)
        mf.mfmc_solve_fields(g, u0, 1, eps=eps, uT=uT, ooi=ooi)
        torch.cuda.synchronize()
        f = float(ooi.cpu()[0])
        assert abs(f - fr) <= 1e-9 * fr, algo
        assert np.abs(uT.cpu().numpy()[0].astype(np.float64) - ur).max() <= tol, algo


def _fixture():
    from tests.conftest import read_golden
    rows = read_golden("large_hf_1024_R32_100steps.txt")
    return [(int(r[1]), float(r[2]), float(r[3]), np.array([float(v) for v in r[4:]])) for r in rows]


@pytest.mark.slow
def test_large_hf_samples_0_to_3_100_steps_fp32_and_kahan(gpu_lib, ooi_errors):
    # samples 0..3 of the large configuration, 100 steps, against the FP64 oracle's solutions
    # stored by tests/golden/make_large_hf_fixture.py (OoI, mean and u at 512 fixed points):
    # the autotuned path (the own-FFT spectral form at this horizon), the plain FP32 prefix sums
    # and the compensated ones.  Bound on the field:
    # 100 x 4e-6 x max|u| e^{c_F T} with max|u| <= 0.05 e^{0.1}.
    import torch
    mf = gpu_lib
    n, R, steps = 1024, 32, 100
    kw = dict(n=n, delta=R / n, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=steps, ic=1, ic_amp=0.05)
    ref = _fixture()
    assert len(ref) == 4
    seeds = np.array([r[0] for r in ref], dtype=np.uint64)
    pts = np.random.default_rng(1024).integers(0, n, size=(512, 2))
    tol = steps * 4e-6 * 0.05 * math.exp(0.1) * math.exp(0.1)
    for algo in (mf.ALGO_AUTO, mf.ALGO_PREFIX_TMA, mf.ALGO_PREFIX_KAHAN):
        g = mf.Model(algo=algo, **kw)
        u0 = torch.empty((4, n, n), dtype=torch.float32, device="cuda")
        uT = torch.empty_like(u0)
        ooi = torch.empty(4, dtype=torch.float64, device="cuda")
        ubar = torch.empty(4, dtype=torch.float64, device="cuda")
        eps = torch.tensor(mf.mfmc_sample_eps(g, seeds), dtype=torch.float64, device="cuda")
        mf.mfmc_init_fields(g, seeds, u0)
        mf.mfmc_solve_fields(g, u0, 4, eps=eps, uT=uT, ooi=ooi, ubar=ubar)
        torch.cuda.synchronize()
        f, m, u = ooi.cpu().numpy(), ubar.cpu().numpy(), uT.cpu().numpy().astype(np.float64)
        for i, (_, fr, mr, ur) in enumerate(ref):
            ooi_errors.add("1024x1024, R=32, 100 steps (autotuned, FP32 prefix and compensated forms)", f[i], fr,
                           m[i], mr, np.abs(u[i][pts[:, 0], pts[:, 1]] - ur).max())
            assert abs(f[i] - fr) <= 1e-9 * fr, (algo, i)
            assert abs(m[i] - mr) <= 1e-5 * abs(mr) + 1e-9, (algo, i)
            assert np.abs(u[i][pts[:, 0], pts[:, 1]] - ur).max() <= tol, (algo, i)
        assert np.abs(u).max() <= 1.0
