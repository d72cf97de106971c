"""The register-tiled weighted disc sum over TMA tiles (MFMC_ALGO_WEIGHTED) against the FP64
oracle: any radial kernel, both boundaries.  Tolerances as in the periodic parity tests
(per step 4e-6 max|u|; the OoI to 1e-5 relative)."""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n,R", [(64, 4), (68, 3), (132, 5), (160, 16), (128, 32)])
def test_weighted_one_step_elementwise(gpu_lib, kernel, bc, n, R):
    mf = gpu_lib
    kw = dict(n=n, delta=R / n, kernel=kernel, delta_hf=(R / n) if kernel else 0.0, eps=0.03, tau=5e-3,
              nsteps=1, ic=2)
    g = mf.Model(algo=mf.ALGO_WEIGHTED, bc=bc, bc_value=-1.0, **kw)
    o = O.OracleModel(bc=bc, bc_value=-1.0, **kw)
    u0, uT, _ = gpu_solve(mf, g, np.arange(2, dtype=np.uint64) + n + 7 * R)
    for i in range(2):
        ref = o.step(u0[i], 0.03)
        assert np.abs(uT[i] - ref).max() <= 4e-6 * max(1.0, np.abs(u0[i]).max())


@pytest.mark.parametrize("inv_h,delta", [(128, 0.25), (64, 0.125)])
def test_weighted_paper_gaussian_solves(gpu_lib, inv_h, delta):
    mf = gpu_lib
    steps = 20
    kw = dict(n=inv_h, delta=delta, kernel=1, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, nsteps=steps, ic=2)
    g = mf.Model(algo=mf.ALGO_WEIGHTED, **kw)
    o = O.OracleModel(**kw)
    seeds = np.arange(2, dtype=np.uint64) + 31
    _, uT, f = gpu_solve(mf, g, seeds)
    for i, s in enumerate(seeds):
        fr, _, ur, _ = o.solve_sample(int(s))
        assert abs(f[i] - fr) <= 1e-5 * fr
        assert np.abs(uT[i] - ur).max() <= steps * 4e-6 * math.exp(0.2)
