"""The spectral step on the library's own FFT kernels (MFMC_ALGO_SPECTRAL: n = 1024 in two
passes per step, n = 64 and 128 resident in shared memory with register transforms, other even
n <= 128 resident with mixed-radix transforms) against the FP64 oracle's direct disc sums.

Tolerance: the transforms round in FP32.  A 1024-point transform by 32 x 32 with radix-2
stages has 10 rounded butterfly levels and FP32 twiddles, so each transform adds about
10 x 2^-24 relative to the RMS of its input; the disc sum S (|S| <= |D| max|u|) then carries an
absolute error of a few FP32 ulps of |D| max|u|, which the update multiplies by c1 (below 1e-2
here), so the per-step bound of the other kernels, 4e-6 max|u|, holds with a wide margin.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

N = 1024


def gpu_solve(mf, g, seeds, u0=None):
    import torch
    ns, n = len(seeds), g.n
    if u0 is None:
        u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
        mf.mfmc_init_fields(g, seeds, u0)
    uT = torch.empty_like(u0)
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    ubar = torch.empty(ns, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mf.mfmc_sample_eps(g, seeds), dtype=torch.float64, device="cuda")
    mf.mfmc_solve_fields(g, u0, ns, eps=eps, uT=uT, ooi=ooi, ubar=ubar)
    torch.cuda.synchronize()
    return (u0.cpu().numpy().astype(np.float64), uT.cpu().numpy().astype(np.float64), ooi.cpu().numpy(),
            ubar.cpu().numpy())


@pytest.mark.parametrize("R,kernel,ic", [(32, 0, 2), (8, 0, 1), (3, 0, 2), (20, 1, 2)])
def test_spectral_one_step_elementwise(gpu_lib, R, kernel, ic):
    # the horizon of the large configuration (3209 points), a small one, one that is not a
    # power of two, and the Gaussian kernel; nuclei ICs have the obstacle active, the smoothed
    # noise IC is nonzero at every row and column
    mf = gpu_lib
    kw = dict(n=N, delta=R / N, eps=0.02, tau=5e-3, nsteps=1, ic=ic, ic_amp=0.05)
    if kernel == 1:
        kw.update(kernel=1, delta_hf=R / N)
    g = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    o = O.OracleModel(**kw)
    seeds = np.arange(2, dtype=np.uint64) + 31 * R
    u0, uT, f, ubar = gpu_solve(mf, g, seeds)
    for i in range(len(seeds)):
        ref = o.step(u0[i], float(mf.mfmc_sample_eps(g, seeds)[i]))
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max()), i
        assert abs(ubar[i] - ref.mean()) <= 1e-5 * abs(ref.mean()) + 1e-9
    assert np.abs(uT).max() <= 1.0


def test_spectral_20_steps_large_configuration_against_oracle(gpu_lib):
    # 1024^2, delta = 32h, smoothed-noise IC of amplitude 0.05, eps = 0.02 U[0.8, 1.2]: the
    # large high-fidelity configuration, 20 steps, one sample
    mf = gpu_lib
    steps = 20
    kw = dict(n=N, delta=32 / N, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=steps, ic=1, ic_amp=0.05)
    g = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    o = O.OracleModel(**kw)
    seeds = np.array([20231016 + 1000003 * 4], dtype=np.uint64)
    fr, mr, ur, _ = o.solve_sample(int(seeds[0]))
    _, uT, f, ubar = gpu_solve(mf, g, seeds)
    assert abs(f[0] - fr) <= 1e-9 * fr
    assert abs(ubar[0] - mr) <= 1e-5 * abs(mr) + 1e-9
    assert np.abs(uT[0] - ur).max() <= steps * 4e-6 * 0.05 * math.e


def test_spectral_matches_the_cufft_path_and_is_deterministic(gpu_lib):
    # the same spectral product by cuFFT's transforms and by the own kernels: the two FP32
    # forms agree to their rounding over 50 steps; a repeated call is bitwise identical; odd
    # batch sizes (the last row pass and column tile are partly empty) and a batch that grows
    mf = gpu_lib
    kw = dict(n=N, delta=16 / N, eps=0.03, tau=5e-3, nsteps=50, ic=2)
    gs = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    gf = mf.Model(algo=mf.ALGO_FFT, **kw)
    for ns in (1, 3):
        seeds = np.arange(ns, dtype=np.uint64) + 700
        _, us, fs, _ = gpu_solve(mf, gs, seeds)
        _, uf, ff, _ = gpu_solve(mf, gf, seeds)
        _, us2, fs2, _ = gpu_solve(mf, gs, seeds)
        assert np.array_equal(us, us2) and np.array_equal(fs, fs2)
        assert np.abs(fs - ff).max() <= 1e-6 * ff.max()
        assert np.abs(us - uf).max() <= 50 * 4e-6 * math.exp(0.5)


def test_spectral_rejects_unsupported_models(gpu_lib):
    mf = gpu_lib
    # 512 and 136: neither 1024 nor <= 128; 52 = 4 x 13 (13 is not a radix); 36 with a disc wider
    # than the lattice; the collar boundary; beta2 > 0
    for kw in (dict(n=512, delta=8 / 512), dict(n=136, delta=8 / 136), dict(n=52, delta=8 / 52),
               dict(n=36, delta=18 / 36), dict(n=N, delta=8 / N, bc=mf.BC_COLLAR, bc_value=-1.0),
               dict(n=96, delta=8 / 96, bc=mf.BC_COLLAR, bc_value=-1.0), dict(n=N, delta=8 / N, beta2=0.05)):
        with pytest.raises(Exception):
            mf.Model(algo=mf.ALGO_SPECTRAL, nsteps=1, **kw)


GAUSS = dict(kernel=1, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, ic=2)


@pytest.mark.parametrize("n,R,kernel,ns", [(128, 32, 0, 2), (128, 8, 1, 3), (64, 8, 0, 5), (64, 16, 1, 4)])
def test_spectral_small_lattices_one_step(gpu_lib, n, R, kernel, ns):
    # the resident form (n = 128: one sample per CTA; n = 64: four, here also a partly empty CTA)
    mf = gpu_lib
    kw = dict(n=n, delta=R / n, eps=0.02, tau=5e-3, nsteps=1, ic=1, ic_amp=0.05)
    if kernel == 1:
        kw.update(kernel=1, delta_hf=R / n)
    g = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    o = O.OracleModel(**kw)
    seeds = np.arange(ns, dtype=np.uint64) + 11 * n + R
    u0, uT, f, ubar = gpu_solve(mf, g, seeds)
    eps = mf.mfmc_sample_eps(g, seeds)
    for i in range(ns):
        ref = o.step(u0[i], float(eps[i]))
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max()), i
        assert abs(ubar[i] - ref.mean()) <= 1e-5 * abs(ref.mean()) + 1e-9
        assert abs(f[i] - 0.5 * (1.0 + ref.mean())) <= 1e-5 * 0.5 * (1.0 + ref.mean())


@pytest.mark.parametrize("inv_h,delta", [(128, 0.25), (64, 0.125)])
def test_spectral_paper_gaussian_models(gpu_lib, inv_h, delta):
    # Table 1's models 1 (delta/h = 32, 3209 points) and 9: Gaussian weights, nuclei IC, 12 steps
    mf = gpu_lib
    steps = 12
    g = mf.Model(n=inv_h, delta=delta, nsteps=steps, algo=mf.ALGO_SPECTRAL, **GAUSS)
    o = O.OracleModel(n=inv_h, delta=delta, nsteps=steps, **GAUSS)
    seeds = np.arange(3, dtype=np.uint64) + 17
    _, uT, f, _ = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert np.abs(uT[i] - ur).max() <= steps * 4e-6 * math.exp(0.12)


@pytest.mark.parametrize("n", [64, 128])
def test_spectral_small_matches_cufft_and_repeats(gpu_lib, n):
    # 100 steps of the paper's finest horizon ratio on this lattice, 7 samples: the own resident
    # form against cuFFT's transforms (FP32 rounding of both), and bitwise repeatability
    mf = gpu_lib
    kw = dict(n=n, delta=0.25 if n == 128 else 0.125, nsteps=100, **GAUSS)
    gs = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    gf = mf.Model(algo=mf.ALGO_FFT, **kw)
    seeds = np.arange(7, dtype=np.uint64) + 900
    _, us, fs, _ = gpu_solve(mf, gs, seeds)
    _, uf, ff, _ = gpu_solve(mf, gf, seeds)
    _, us2, fs2, _ = gpu_solve(mf, gs, seeds)
    assert np.array_equal(us, us2) and np.array_equal(fs, fs2)
    assert np.abs(fs - ff).max() <= 1e-6 * ff.max()
    assert np.abs(us - uf).max() <= 100 * 4e-6 * math.exp(1.0)


def test_spectral_small_lattice_first_in_a_fresh_process(gpu_lib):
    # a process whose first (and only) spectral solve is on a small lattice: every table and
    # constant the resident form uses must be set up by that form itself
    import os
    import subprocess
    import sys
    code = (
        "import math, numpy as np, torch\n"
        "from paper_2310_10750_gb300 import mfmc\n"
        "kw = dict(n=128, delta=0.25, kernel=1, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, nsteps=20, ic=2)\n"
        "seeds = np.arange(3, dtype=np.uint64) + 5\n"
        "out = []\n"
        "for algo in (mfmc.ALGO_SPECTRAL, mfmc.ALGO_FFT):\n"
        "    g = mfmc.Model(algo=algo, **kw)\n"
        "    u0 = torch.empty((3, 128, 128), dtype=torch.float32, device='cuda')\n"
        "    mfmc.mfmc_init_fields(g, seeds, u0)\n"
        "    ooi = torch.empty(3, dtype=torch.float64, device='cuda')\n"
        "    mfmc.mfmc_solve_fields(g, u0, 3, ooi=ooi)\n"
        "    torch.cuda.synchronize()\n"
        "    out.append(ooi.cpu().numpy())\n"
        "print(float(np.abs(out[0] - out[1]).max() / out[1].max()))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert float(r.stdout.strip().splitlines()[-1]) <= 1e-6


@pytest.mark.parametrize("n,delta,kernel,ns", [(88, 11 / 88, 1, 3), (88, 0.1875, 1, 2), (96, 8 / 96, 0, 3),
                                               (120, 20 / 120, 0, 2), (44, 5 / 44, 1, 4), (100, 9 / 100, 0, 1),
                                               (56, 7 / 56, 1, 3)])
def test_spectral_mixed_radix_lattices_one_step(gpu_lib, n, delta, kernel, ns):
    # the resident mixed-radix form: radices 11 4 2 (88, also at the non-integer delta/h = 16.5),
    # 3 4 4 2 (96), 5 3 4 2 (120), 11 4 (44), 5 5 4 (100), 7 4 2 (56); nuclei IC (obstacle active)
    mf = gpu_lib
    kw = dict(n=n, delta=delta, eps=0.02, tau=5e-3, nsteps=1, ic=2)
    if kernel == 1:
        kw.update(kernel=1, delta_hf=0.25)
    g = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    o = O.OracleModel(**kw)
    seeds = np.arange(ns, dtype=np.uint64) + 3 * n
    u0, uT, f, ubar = gpu_solve(mf, g, seeds)
    eps = mf.mfmc_sample_eps(g, seeds)
    for i in range(ns):
        ref = o.step(u0[i], float(eps[i]))
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max()), i
        assert abs(f[i] - 0.5 * (1.0 + ref.mean())) <= 1e-5 * 0.5 * (1.0 + ref.mean())
    assert np.abs(uT).max() <= 1.0 and (uT == 1.0).any()   # the +1 bound is active around the nuclei


@pytest.mark.parametrize("delta", [0.1875, 0.25, 0.125])
def test_spectral_paper_88_models(gpu_lib, delta):
    # Table 1's models 3 (delta/h = 16.5), 4 and 6 on h = 1/88: 12 steps against the oracle;
    # 100 steps against cuFFT's transforms; a repeated call is bitwise identical
    mf = gpu_lib
    g = mf.Model(n=88, delta=delta, nsteps=12, algo=mf.ALGO_SPECTRAL, **GAUSS)
    o = O.OracleModel(n=88, delta=delta, nsteps=12, **GAUSS)
    seeds = np.arange(3, dtype=np.uint64) + 41
    _, uT, f, _ = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert np.abs(uT[i] - ur).max() <= 12 * 4e-6 * math.exp(0.12)
    kw = dict(n=88, delta=delta, nsteps=100, **GAUSS)
    gs = mf.Model(algo=mf.ALGO_SPECTRAL, **kw)
    gf = mf.Model(algo=mf.ALGO_FFT, **kw)
    seeds = np.arange(5, dtype=np.uint64) + 77
    _, us, fs, _ = gpu_solve(mf, gs, seeds)
    _, uf, ff, _ = gpu_solve(mf, gf, seeds)
    _, us2, fs2, _ = gpu_solve(mf, gs, seeds)
    assert np.array_equal(us, us2) and np.array_equal(fs, fs2)
    assert np.abs(fs - ff).max() <= 1e-6 * ff.max()
    assert np.abs(us - uf).max() <= 100 * 4e-6 * math.exp(1.0)
