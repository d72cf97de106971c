"""The allocation-free solve (mfmc_solve_fields_noalloc) against the ordinary one.

Some callers cannot allocate device memory while they solve (their framework holds all
device memory in its own allocator, or their loop must not stall on cudaMalloc); for them
the library offers a solve whose scratch is a fixed array inside the library.  This file
runs last (pytest collects it after the other test files) and also passes on its own.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(mf):
    f = mf._L.mfmc_solve_fields_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_size_t] + [ctypes.c_void_p] * 4
    return f


def _solve_both(mf, call, model, ns, seeds, want_field=True, want_mean=True):
    """The ordinary solve and the allocation-free one on the same inputs; the latter writes
    into NaN-filled outputs so that anything it leaves unwritten shows."""
    import torch
    n = model.n
    u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
    eps = torch.tensor(mf.mfmc_sample_eps(model, seeds), dtype=torch.float64, device="cuda")
    mf.mfmc_init_fields(model, seeds, u0)
    ref_u = torch.empty_like(u0) if want_field else None
    ref_f = torch.empty(ns, dtype=torch.float64, device="cuda")
    ref_m = torch.empty(ns, dtype=torch.float64, device="cuda") if want_mean else None
    mf.mfmc_solve_fields(model, u0, ns, eps=eps, uT=ref_u, ubar=ref_m, ooi=ref_f)
    got_u = torch.full_like(u0, float("nan")) if want_field else None
    got_f = torch.full((ns,), float("nan"), dtype=torch.float64, device="cuda")
    got_m = torch.full((ns,), float("nan"), dtype=torch.float64, device="cuda") if want_mean else None
    ptr = lambda t: None if t is None else t.data_ptr()
    st = call(model.handle, eps.data_ptr(), u0.data_ptr(), ns, ptr(got_u), ptr(got_m), got_f.data_ptr(), None)
    assert st == mf.MFMC_OK, mf.mfmc_last_error()
    torch.cuda.synchronize()
    return (ref_u, ref_f, ref_m), (got_u, got_f, got_m)


def test_noalloc_matches_the_allocating_solve_on_two_calls(gpu_lib):
    # Both calls run the same register-tiled prefix kernel in the same order, so fields,
    # means and OoIs agree bit for bit; the second call reuses the array after the first.
    import torch
    mf = gpu_lib
    call = _noalloc(mf)
    n, R, steps, ns = 64, 4, 200, 32
    model = mf.Model(n=n, delta=R / n, eps=0.03, eps_lo=0.024, eps_hi=0.036, tau=1e-3, nsteps=steps,
                     ic=mf.IC_NUCLEI, algo=mf.ALGO_PREFIX)
    for call_no, base in enumerate((20231016, 777)):
        seeds = np.arange(ns, dtype=np.uint64) + base
        (ru, rf, rm), (gu, gf, gm) = _solve_both(mf, call, model, ns, seeds)
        assert torch.equal(gu, ru), call_no
        assert torch.equal(gf, rf) and torch.equal(gm, rm), call_no
        assert gu.abs().max().item() <= 1.0


@pytest.mark.parametrize("n,R,steps,ns", [(128, 16, 6, 8), (64, 4, 0, 5), (96, 5, 3, 7)])
def test_noalloc_other_shapes(gpu_lib, n, R, steps, ns):
    # a horizon whose tile needs more than 48 KB of shared memory (R = 16), no time step at
    # all, and a ragged lattice; the field is not requested but the mean is
    import torch
    mf = gpu_lib
    call = _noalloc(mf)
    model = mf.Model(n=n, delta=R / n, eps=0.03, tau=1e-3, nsteps=steps, ic=mf.IC_SMOOTHED_GAUSS,
                     algo=mf.ALGO_PREFIX)
    seeds = np.arange(ns, dtype=np.uint64) + 4242
    (ru, rf, rm), (gu, gf, gm) = _solve_both(mf, call, model, ns, seeds, want_field=False)
    assert torch.equal(gf, rf) and torch.equal(gm, rm)
    (ru, rf, rm), (gu, gf, gm) = _solve_both(mf, call, model, ns, seeds, want_field=True, want_mean=False)
    assert torch.equal(gu, ru) and torch.equal(gf, rf)


def test_noalloc_rejects_batches_beyond_its_scratch(gpu_lib):
    import torch
    mf = gpu_lib
    call = _noalloc(mf)
    model = mf.Model(n=256, delta=8 / 256, nsteps=2, algo=mf.ALGO_PREFIX)
    ns = 63                                  # 63 x 256 KB exceeds the 16.48 MB field buffer
    u0 = torch.zeros((ns, 256, 256), dtype=torch.float32, device="cuda")
    st = call(model.handle, None, u0.data_ptr(), ns, None, None, None, None)
    assert st == mf.MFMC_EINVAL
    assert "too large" in mf.mfmc_last_error()
    ooi = torch.empty(62, dtype=torch.float64, device="cuda")
    st = call(model.handle, None, u0.data_ptr(), 62, None, None, ooi.data_ptr(), None)
    assert st == mf.MFMC_OK
    torch.cuda.synchronize()
    assert np.all(ooi.cpu().numpy() == 0.5)
