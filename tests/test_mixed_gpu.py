"""The one-launch-per-step hierarchy solve (mfmc_solve_batch_mixed) against the FP64 oracle
and against the per-model solves.

Tolerances as in the single-fidelity parity tests: a k-step solve agrees with the oracle to
|f_gpu - f_orc| <= 1e-5 f_orc.  Against the per-model solves with the same kernels (the TMA
prefix kernel for the queued models, the resident kernel for models that fit in shared
memory) the fields are the same FP32 values (each output is formed by the same sequence of
operations whatever the tile shape), so the OoI differs only by the FP64 summation order of
the tile partials.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

COMMON = dict(eps=0.03, eps_lo=0.024, eps_hi=0.036, tau=5e-3, ic=2, ic_amp=0.05)
# (n, R): every R the mixed kernel serves, ragged tiles at 96 (64 x 64 tiles) and 160
# (128 x 64 tiles for R = 16), a field smaller than one R = 8 tile (64 x 128) at 64.
HIERARCHY = [(160, 16), (64, 8), (96, 4), (64, 2)]


def models(mf, steps=40, algo=None):
    out = []
    for n, R in HIERARCHY:
        g = mf.Model(n=n, delta=R / n, nsteps=steps, algo=algo if algo is not None else mf.ALGO_AUTO, **COMMON)
        out.append(g)
    return out


def oracle_model(n, R, steps):
    return O.OracleModel(n=n, delta=R / n, nsteps=steps, **COMMON)


def test_mixed_batch_matches_oracle(gpu_lib):
    mf = gpu_lib
    gs = models(mf)
    pick = [0, 1, 2, 3, 3, 2, 1, 0, 2, 3]
    seeds = np.arange(len(pick), dtype=np.uint64) + 777
    f, ubar = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    for i, k in enumerate(pick):
        n, R = HIERARCHY[k]
        fr, mean, _, _ = oracle_model(n, R, 40).solve_sample(int(seeds[i]))
        assert abs(f[i] - fr) <= 1e-5 * fr, (i, n, R, f[i], fr)
        assert abs(ubar[i] - mean) <= 2e-5 * fr


def reference_models(mf, steps):
    """Per-model solves with the algorithm the mixed call uses for that model: the resident
    kernel where it fits, else the TMA prefix kernel (4 columns per thread)."""
    out = []
    for n, R in HIERARCHY:
        try:
            g = mf.Model(n=n, delta=R / n, nsteps=steps, algo=mf.ALGO_RESIDENT, **COMMON)
        except mf.MfmcError:
            g = mf.Model(n=n, delta=R / n, nsteps=steps, algo=mf.ALGO_PREFIX_TMA, **COMMON)
        out.append(g)
    return out


def test_mixed_batch_matches_per_model_solves(gpu_lib):
    mf = gpu_lib
    gs = models(mf, steps=30)
    ref = reference_models(mf, 30)
    kinds = {g.info().algo for g in ref}
    assert mf.ALGO_PREFIX_TMA in kinds and mf.ALGO_RESIDENT in kinds
    pick = [k for k in range(4) for _ in range(5)]
    seeds = np.arange(len(pick), dtype=np.uint64) + 4242
    f, ubar = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    fr, ur = mf.mfmc_solve_batch([ref[k] for k in pick], seeds)
    np.testing.assert_allclose(f, fr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(ubar, ur, rtol=0, atol=2e-13)


def test_mixed_queue_of_four_streamed_models(gpu_lib):
    # four models too large for the resident kernel: all of them share the step queue
    # (ragged tiles for every shape: 64 x 64, 64 x 128 and 128 x 64 tiles on n = 132..160)
    mf = gpu_lib
    shapes = [(160, 16), (136, 8), (132, 4), (140, 2)]
    gs = [mf.Model(n=n, delta=R / n, nsteps=12, **COMMON) for n, R in shapes]
    tma = [mf.Model(n=n, delta=R / n, nsteps=12, algo=mf.ALGO_PREFIX_TMA, **COMMON) for n, R in shapes]
    pick = [3, 2, 1, 0, 0, 1, 2, 3, 1]
    seeds = np.arange(len(pick), dtype=np.uint64) + 555
    f, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    fr, _ = mf.mfmc_solve_batch([tma[k] for k in pick], seeds)
    np.testing.assert_allclose(f, fr, rtol=0, atol=1e-13)
    for i in (0, 3, 5):
        n, R = shapes[pick[i]]
        fo, _, _, _ = oracle_model(n, R, 12).solve_sample(int(seeds[i]))
        assert abs(f[i] - fo) <= 1e-5 * fo


def test_mixed_per_sample_steps(gpu_lib):
    mf = gpu_lib
    gs = models(mf, steps=12)
    pick = [0, 1, 2, 3, 0, 3]
    steps = [12, 3, 1, 7, 5, 12]
    seeds = np.arange(len(pick), dtype=np.uint64) + 99
    p = mf.make_params(len(pick), nsteps=steps)
    f, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds, params=p)
    for i, k in enumerate(pick):
        n, R = HIERARCHY[k]
        fr, _, _, _ = oracle_model(n, R, steps[i]).solve_sample(int(seeds[i]))
        assert abs(f[i] - fr) <= 1e-5 * fr, (i, steps[i])


def test_mixed_graph_replay_and_repeat(gpu_lib):
    # the second call of a shape replays the captured step loop with new inputs
    mf = gpu_lib
    gs = models(mf, steps=20)
    pick = [3, 2, 1, 0]
    s1 = np.arange(4, dtype=np.uint64) + 1
    s2 = np.arange(4, dtype=np.uint64) + 1001
    a1, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], s1)
    a2, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], s2)
    b1, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], s1)
    assert np.array_equal(a1, b1)
    assert not np.array_equal(a1, a2)
    for i, k in enumerate(pick):
        n, R = HIERARCHY[k]
        fr, _, _, _ = oracle_model(n, R, 20).solve_sample(int(s2[i]))
        assert abs(a2[i] - fr) <= 1e-5 * fr


def test_mixed_single_model_single_sample(gpu_lib):
    mf = gpu_lib
    g = mf.Model(n=64, delta=4 / 64, nsteps=5, **COMMON)
    f, _ = mf.mfmc_solve_batch_mixed([g], [31337])
    fr, _, _, _ = oracle_model(64, 4, 5).solve_sample(31337)
    assert abs(f[0] - fr) <= 1e-5 * fr


def test_mixed_rejects_unsupported(gpu_lib):
    mf = gpu_lib
    gs = models(mf, steps=4)
    extra = mf.Model(n=128, delta=8 / 128, nsteps=4, **COMMON)
    with pytest.raises(mf.MfmcError):   # five distinct models
        mf.mfmc_solve_batch_mixed(gs + [extra], np.arange(5, dtype=np.uint64))
    r3 = mf.Model(n=136, delta=3 / 136, nsteps=4, **COMMON)
    with pytest.raises(mf.MfmcError):   # R outside {2, 4, 8, 16} and n > 128
        mf.mfmc_solve_batch_mixed([r3], [1])
    gauss = mf.Model(n=144, delta=8 / 144, kernel=1, delta_hf=0.25, nsteps=4, **COMMON)
    with pytest.raises(mf.MfmcError):   # Gaussian kernel and n > 128
        mf.mfmc_solve_batch_mixed([gauss], [1])
    many = [mf.Model(n=64, delta=(3 + k) / 64, nsteps=4, **COMMON) for k in range(17)]
    with pytest.raises(mf.MfmcError):   # 17 models for the resident spectral queue (at most 16)
        mf.mfmc_solve_batch_mixed(many, np.arange(17, dtype=np.uint64))
    b2 = mf.Model(n=64, delta=8 / 64, beta2=0.05, nsteps=4, **COMMON)
    with pytest.raises(mf.MfmcError):   # beta2 > 0
        mf.mfmc_solve_batch_mixed([b2], [1])
    zero = mf.Model(n=64, delta=4 / 64, nsteps=0, **COMMON)
    with pytest.raises(mf.MfmcError):   # no step to take
        mf.mfmc_solve_batch_mixed([zero], [1])
    # the library stays usable after the rejections
    f, _ = mf.mfmc_solve_batch_mixed([gs[3]], [5])
    fr, _, _, _ = oracle_model(64, 2, 4).solve_sample(5)
    assert abs(f[0] - fr) <= 1e-5 * fr


# The paper's hierarchy (Section 4, Table 1): Gaussian kernel, h in {1/128, 1/88, 1/64} x delta in
# {0.25, 0.1875, 0.125} (delta/h = 16.5 on h = 1/88), nuclei IC.  The TMA queue does not serve it;
# every model fits the resident spectral form, so one launch runs the samples of all nine.
PAPER = [(128, 0.25), (128, 0.1875), (88, 0.1875), (88, 0.25), (128, 0.125), (88, 0.125),
         (64, 0.1875), (64, 0.25), (64, 0.125)]
GAUSS = dict(kernel=1, delta_hf=0.25, eps=0.0421900462, tau=0.01, ic=2)


def test_mixed_paper_hierarchy_matches_oracle(gpu_lib):
    mf = gpu_lib
    steps = 15
    gs = [mf.Model(n=n, delta=d, nsteps=steps, **GAUSS) for n, d in PAPER]
    pick = [8, 0, 2, 5, 1, 7, 3, 6, 4, 0, 2, 8]
    seeds = np.arange(len(pick), dtype=np.uint64) + 2023
    f, ubar = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    for i, k in enumerate(pick):
        n, d = PAPER[k]
        fr, mean, _, _ = O.OracleModel(n=n, delta=d, nsteps=steps, **GAUSS).solve_sample(int(seeds[i]))
        assert abs(f[i] - fr) <= 1e-5 * fr, (i, n, d, f[i], fr)
        assert abs(ubar[i] - mean) <= 2e-5 * fr


def test_mixed_paper_hierarchy_matches_per_model_spectral_solves(gpu_lib):
    # against per-model MFMC_ALGO_SPECTRAL solves: on h = 1/88 the same resident mixed-radix
    # kernel (identical results); on 1/64 and 1/128 the register-transform form (FP32 rounding of
    # two different transforms); per-sample step counts; a repeated call is bitwise identical
    mf = gpu_lib
    steps = 40
    gs = [mf.Model(n=n, delta=d, nsteps=steps, **GAUSS) for n, d in PAPER]
    ref = [mf.Model(n=n, delta=d, nsteps=steps, algo=mf.ALGO_SPECTRAL, **GAUSS) for n, d in PAPER]
    pick = [k for k in range(9) for _ in range(3)]
    seeds = np.arange(len(pick), dtype=np.uint64) + 9000
    f, ubar = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    fr, ur = mf.mfmc_solve_batch([ref[k] for k in pick], seeds)
    for i, k in enumerate(pick):
        if PAPER[k][0] == 88:
            assert f[i] == fr[i] and ubar[i] == ur[i], i
        else:
            assert abs(f[i] - fr[i]) <= 1e-6 * fr[i], i
    f2, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    assert np.array_equal(f, f2)
    steps_ps = [1 + (7 * i) % steps for i in range(len(pick))]
    p = mf.make_params(len(pick), nsteps=steps_ps)
    fp, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds, params=p)
    for i in (0, 4, 8, 13, 20, 26):
        n, d = PAPER[pick[i]]
        fo, _, _, _ = O.OracleModel(n=n, delta=d, nsteps=steps_ps[i], **GAUSS).solve_sample(int(seeds[i]))
        assert abs(fp[i] - fo) <= 1e-5 * fo, (i, steps_ps[i])
