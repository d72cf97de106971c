"""The volume-constrained collar boundary (MFMC_BC_COLLAR) on the GPU against the FP64
oracle's collar form (oracle.OracleModel with bc=1).

The collar lives in the TMA kernels' ghost frame (filled with the collar value, never
overwritten) and in the generic kernel's loads; the tolerances are those of the periodic
parity tests: per step |u_gpu - u_orc| <= 4e-6 max|u|, over k steps k times that bound times
e^{c_F T}, and |f_gpu - f_orc| <= 1e-5 f_orc on the output of interest.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

# name -> (algorithm, TMA tile variant or None)
PATHS = {"tma0": ("PREFIX_TMA", 0), "tma1": ("PREFIX_TMA", 1), "tma4": ("PREFIX_TMA", 4),
         "tma6": ("PREFIX_TMA", 6), "kahan": ("PREFIX_KAHAN", None), "direct": ("DIRECT", None),
         "plain": ("PLAIN", None)}


def pair(mf, n, R, steps, uI, path="tma4", ic=2, tau=5e-3, eps=0.03, kernel=0, delta_hf=0.0):
    algo, variant = PATHS[path] if path != "auto" else ("AUTO", None)
    kw = dict(n=n, delta=R / n, kernel=kernel, delta_hf=delta_hf, eps=eps, tau=tau, nsteps=steps, ic=ic,
              ic_amp=0.05)
    g = mf.Model(algo=getattr(mf, "ALGO_" + algo), bc=mf.BC_COLLAR, bc_value=uI, **kw)
    if variant is not None:
        g.set_tile_variant(variant)
    o = O.OracleModel(bc=1, bc_value=uI, **kw)
    return g, o


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


def seeds_of(k, base):
    return np.arange(k, dtype=np.uint64) + base


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("n,R,uI", [(64, 4, -1.0), (68, 3, 0.3), (132, 5, -1.0), (200, 8, 0.5), (160, 16, -1.0)])
def test_collar_one_step_elementwise(gpu_lib, path, n, R, uI):
    # ragged tiles (68, 132, 200), ghost width 4 (R = 3) and 16 (R = 16), collar values inside
    # (-1, 1) and at the obstacle
    mf = gpu_lib
    g, o = pair(mf, n, R, 1, uI, path)
    u0, uT, _, _ = gpu_solve(mf, g, seeds_of(3, 7 * n))
    for i in range(3):
        ref = o.step(u0[i], 0.03)
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max()), path
        assert np.abs(uT[i]).max() <= 1.0


@pytest.mark.parametrize("path", ["tma4", "tma0", "direct", "auto"])
def test_collar_solve_matches_oracle(gpu_lib, path):
    # nuclei initial condition, 60 steps of tau = 5e-3 with a -1 collar: the obstacle is
    # active inside and the collar erodes the +1 phase near the edges
    mf = gpu_lib
    steps = 60
    g, o = pair(mf, 128, 8, steps, -1.0, path)
    seeds = seeds_of(4, 321)
    _, uT, f, ubar = gpu_solve(mf, g, seeds)
    assert (uT == 1.0).any() and (uT == -1.0).any()
    tol = steps * 4e-6 * math.exp(steps * 5e-3)
    for i, s in enumerate(seeds):
        fr, mean, ur, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert abs(ubar[i] - mean) <= 2e-5 * fr
        assert np.abs(uT[i] - ur).max() <= tol


def test_collar_differs_from_periodic_only_near_the_edges(gpu_lib):
    # One step from the same field.  An output of tile variant 4 is the difference of running
    # row sums that start at the left end of its thread's window (columns 4 floor(x / 4) - R
    # to 4 floor(x / 4) + 3 + R), so where that window and the output's rows y - R .. y + R
    # stay inside the lattice, periodic and collar results agree bit for bit; elsewhere they
    # agree where the disc stays inside (to rounding) and differ at the edges.
    mf = gpu_lib
    n, R = 96, 6
    gc, _ = pair(mf, n, R, 1, -1.0, "tma4")
    gp = mf.Model(n=n, delta=R / n, eps=0.03, tau=5e-3, nsteps=1, ic=2, ic_amp=0.05, algo=mf.ALGO_PREFIX_TMA)
    gp.set_tile_variant(4)
    seeds = seeds_of(2, 5)
    _, uc, _, _ = gpu_solve(mf, gc, seeds)
    _, up, _, _ = gpu_solve(mf, gp, seeds)
    xb = 4 * (np.arange(n) // 4)
    cols = (xb - R >= 0) & (xb + 3 + R <= n - 1)
    assert np.array_equal(uc[:, R:n - R][:, :, cols], up[:, R:n - R][:, :, cols])
    assert np.abs(uc[:, R:n - R, R:n - R] - up[:, R:n - R, R:n - R]).max() <= 4e-6
    assert not np.array_equal(uc[:, :R], up[:, :R])


@pytest.mark.parametrize("uI", [-1.0, 0.0, 1.0])
def test_collar_pure_phase_matching_the_collar_is_stationary(gpu_lib, uI):
    import torch
    mf = gpu_lib
    for path in ("tma4", "direct", "kahan"):
        g, _ = pair(mf, 64, 4, 30, uI, path)
        u0 = torch.full((2, 64, 64), uI, dtype=torch.float32, device="cuda")
        uT = torch.empty_like(u0)
        ooi = torch.empty(2, dtype=torch.float64, device="cuda")
        mf.mfmc_solve_fields(g, u0, 2, uT=uT, ooi=ooi)
        torch.cuda.synchronize()
        assert torch.all(uT == uI)
        assert np.all(ooi.cpu().numpy() == 0.5 * (1 + uI))


def test_collar_gaussian_kernel_generic_path(gpu_lib):
    mf = gpu_lib
    eps = math.sqrt(0.00178)
    g, o = pair(mf, 64, 8, 20, -1.0, "direct", eps=eps, kernel=1, delta_hf=0.25, tau=1e-2)
    seeds = seeds_of(2, 9)
    _, uT, f, _ = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert np.abs(uT[i] - ur).max() <= 20 * 4e-6 * 1.3


def test_collar_batch_and_server_match_the_oracle(gpu_lib):
    import time
    mf = gpu_lib
    g, o = pair(mf, 128, 4, 40, -1.0, "auto")
    seeds = seeds_of(3, 77)
    f, _ = mf.mfmc_solve_batch([g] * 3, seeds)
    srv = mf.Server(1 << 30, 64)
    tickets = [srv.submit(g, int(s)) for s in seeds]
    got, t0 = {}, time.time()
    while len(got) < len(tickets):
        for t in tickets:
            if t not in got:
                r = srv.poll(t)
                if r is not None:
                    got[t] = r[0]
        assert time.time() - t0 < 120
        time.sleep(0.001)
    srv.close()
    assert g.info().algo in (mf.ALGO_PREFIX_TMA, mf.ALGO_DIRECT, mf.ALGO_PREFIX_KAHAN)
    for i, s in enumerate(seeds):
        fr, _, _, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert abs(got[tickets[i]] - fr) <= 1e-5 * fr


def test_collar_rejections(gpu_lib):
    mf = gpu_lib
    with pytest.raises(mf.MfmcError):       # collar value outside [-1, 1]
        mf.Model(n=64, delta=4 / 64, bc=mf.BC_COLLAR, bc_value=1.5)
    with pytest.raises(mf.MfmcError):       # unknown boundary
        mf.Model(n=64, delta=4 / 64, bc=7)
    for algo in (mf.ALGO_RESIDENT, mf.ALGO_ROWS, mf.ALGO_PREFIX):
        with pytest.raises(mf.MfmcError):   # periodic-only kernels
            mf.Model(n=64, delta=4 / 64, bc=mf.BC_COLLAR, algo=algo)
    g = mf.Model(n=128, delta=4 / 128, nsteps=4, bc=mf.BC_COLLAR, bc_value=-1.0)
    with pytest.raises(mf.MfmcError):       # the mixed-fidelity call is periodic only
        mf.mfmc_solve_batch_mixed([g], [1])


def test_collar_full_size_sampled(gpu_lib):
    # the benchmark's collar line: 256 x 256, delta = 8h, 1000 steps, 512 samples in one
    # launch configuration; the oracle checks samples 0 and 511 element by element
    import torch
    mf = gpu_lib
    n, R, steps, ns = 256, 8, 1000, 512
    kw = dict(n=n, delta=R / n, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=steps, ic=1, ic_amp=0.05)
    g = mf.Model(bc=mf.BC_COLLAR, bc_value=-1.0, **kw)
    o = O.OracleModel(bc=1, bc_value=-1.0, **kw)
    seeds = seeds_of(ns, 20231016 + 1000003)
    u0, uT, f, _ = gpu_solve(mf, g, seeds)
    assert np.abs(uT).max() <= 1.0
    # the -1 collar lowers the mean near the edges: every sample's mean drops below its start
    assert np.all(uT.mean(axis=(1, 2)) < u0.mean(axis=(1, 2)))
    tol = steps * 4e-6 * math.e
    for i in (0, ns - 1):
        fr, _, ur, _ = o.solve_sample(int(seeds[i]))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert np.abs(uT[i] - ur).max() <= tol
    del torch
