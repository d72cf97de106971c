"""The allocation-free solve (mfmc_solve_fields_noalloc) against the ordinary one.

Some callers cannot allocate device memory while they solve (their framework holds all
device memory in its own allocator, or their loop must not stall on cudaMalloc); for them
the library offers a solve whose scratch is a fixed array inside the library.  This file
runs last (pytest collects it after the other test files) and also passes on its own.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(mf):
    f = mf._L.mfmc_solve_fields_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_size_t] + [ctypes.c_void_p] * 4
    return f


def test_noalloc_matches_the_allocating_solve_on_two_calls(gpu_lib):
    import torch
    mf = gpu_lib
    call = _noalloc(mf)
    n, R, steps, ns = 64, 4, 200, 32
    model = mf.Model(n=n, delta=R / n, eps=0.03, eps_lo=0.024, eps_hi=0.036, tau=1e-3, nsteps=steps,
                     ic=mf.IC_NUCLEI, algo=mf.ALGO_PREFIX)
    growth = math.exp(steps * 1e-3)
    for call_no, base in enumerate((20231016, 777)):
        seeds = np.arange(ns, dtype=np.uint64) + base
        u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
        eps = torch.tensor(mf.mfmc_sample_eps(model, seeds), dtype=torch.float64, device="cuda")
        mf.mfmc_init_fields(model, seeds, u0)
        ref_u = torch.empty_like(u0)
        ref_f = torch.empty(ns, dtype=torch.float64, device="cuda")
        ref_m = torch.empty(ns, dtype=torch.float64, device="cuda")
        mf.mfmc_solve_fields(model, u0, ns, eps=eps, uT=ref_u, ubar=ref_m, ooi=ref_f)
        got_u = torch.full_like(u0, float("nan"))
        got_f = torch.full((ns,), float("nan"), dtype=torch.float64, device="cuda")
        got_m = torch.full((ns,), float("nan"), dtype=torch.float64, device="cuda")
        st = call(model.handle, eps.data_ptr(), u0.data_ptr(), ns, got_u.data_ptr(), got_m.data_ptr(),
                  got_f.data_ptr(), None)
        assert st == mf.MFMC_OK, mf.mfmc_last_error()
        torch.cuda.synchronize()
        a, b = got_f.cpu().numpy(), ref_f.cpu().numpy()
        assert np.all(np.abs(a - b) <= 1e-5 * np.abs(b)), call_no
        assert np.all(np.abs(got_m.cpu().numpy() - ref_m.cpu().numpy()) <= 1e-5)
        du = (got_u - ref_u).abs().max().item()
        assert du <= steps * 4e-6 * growth, (call_no, du)
        assert got_u.abs().max().item() <= 1.0


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
