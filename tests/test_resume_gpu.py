"""Checkpoint and resume through the public calls: a solve of k1 steps, its final fields copied to
the host (the snapshot: the fields, the sample's eps and the steps done; the seed's random draws
are spent at the initial field), copied back and advanced k2 more steps, against one solve of
k1 + k2 steps on the same initial fields.

beta2 = 0: each step is a function of the previous field and the sample's coefficients alone, so
the resumed fields and OoIs equal the uninterrupted ones bit for bit, on every kernel family.
beta2 > 0: the first resumed step starts its Newton iteration from the beta2 = 0 step instead of
the previous step's w, so the two agree to the solver's tolerance (max|F| <= 1e-11 per step), not
bitwise.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GAUSS = dict(kernel=1, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, ic=2)


def _solve(mf, g, u0, eps):
    import torch
    ns = u0.shape[0]
    uT = torch.empty_like(u0)
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    mf.mfmc_solve_fields(g, u0, ns, eps=eps, uT=uT, ooi=ooi)
    torch.cuda.synchronize()
    return uT, ooi


# (description, model keywords): the benchmark's row-streaming kernel, the TMA tile kernel, the
# resident kernel, the register-transform and the mixed-radix spectral forms, the weighted form
CASES = [
    ("row streaming 256^2 R8", dict(n=256, delta=8 / 256, eps=0.02, tau=1e-3, ic=1, algo="ROWS")),
    ("TMA tile 96^2 R4", dict(n=96, delta=4 / 96, eps=0.03, tau=5e-3, ic=2, algo="PREFIX_TMA")),
    ("resident 64^2 R4", dict(n=64, delta=4 / 64, eps=0.03, tau=5e-3, ic=2, algo="RESIDENT")),
    ("spectral 128^2 Gaussian", dict(n=128, delta=0.25, algo="SPECTRAL", **GAUSS)),
    ("spectral 88^2 delta/h=16.5", dict(n=88, delta=0.1875, algo="SPECTRAL", **GAUSS)),
    ("weighted 64^2 Gaussian", dict(n=64, delta=0.125, algo="WEIGHTED", **GAUSS)),
]


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_resume_from_a_host_snapshot_is_bitwise(gpu_lib, case):
    import torch
    mf = gpu_lib
    kw = dict(CASES[case][1])
    algo = getattr(mf, "ALGO_" + kw.pop("algo"))
    k1, k2, ns = 7, 5, 6
    full = mf.Model(nsteps=k1 + k2, algo=algo, **kw)
    first = mf.Model(nsteps=k1, algo=algo, **kw)
    rest = mf.Model(nsteps=k2, algo=algo, **kw)
    seeds = np.arange(ns, dtype=np.uint64) + 123 + case
    n = kw["n"]
    u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
    mf.mfmc_init_fields(full, seeds, u0)
    eps = torch.tensor(mf.mfmc_sample_eps(full, seeds), dtype=torch.float64, device="cuda")
    u_full, f_full = _solve(mf, full, u0, eps)
    u_mid, _ = _solve(mf, first, u0, eps)
    snapshot = u_mid.cpu().numpy().copy()                 # to the host ...
    u_back = torch.from_numpy(snapshot).to("cuda")        # ... and back
    u_res, f_res = _solve(mf, rest, u_back, eps)
    assert torch.equal(u_res, u_full)
    assert torch.equal(f_res, f_full)


def test_resume_beta2_within_the_solver_tolerance(gpu_lib):
    import torch
    mf = gpu_lib
    kw = dict(n=64, delta=0.125, beta2=0.05, **GAUSS)
    k1, k2, ns = 6, 6, 3
    full = mf.Model(nsteps=k1 + k2, **kw)
    first = mf.Model(nsteps=k1, **kw)
    rest = mf.Model(nsteps=k2, **kw)
    seeds = np.arange(ns, dtype=np.uint64) + 5
    u0 = torch.empty((ns, 64, 64), dtype=torch.float32, device="cuda")
    mf.mfmc_init_fields(full, seeds, u0)
    eps = torch.tensor(mf.mfmc_sample_eps(full, seeds), dtype=torch.float64, device="cuda")
    u_full, f_full = _solve(mf, full, u0, eps)
    u_mid, _ = _solve(mf, first, u0, eps)
    u_res, f_res = _solve(mf, rest, torch.from_numpy(u_mid.cpu().numpy()).to("cuda"), eps)
    # the snapshot is FP32 (the FP64 iterate is rounded once), then each step is Lipschitz
    assert (f_res - f_full).abs().max().item() <= 1e-7
    assert (u_res - u_full).abs().max().item() <= 1e-5
