"""Per-work-item trace (mfmc_trace_enable / mfmc_trace_read) of the queue kernels: one record
per item, each item exactly once, timestamps ordered, SM ids in range, no change to any result,
and the ring's overflow and read-out rules."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GAUSS = dict(kernel=1, delta_hf=0.25, eps=0.0421900462, tau=0.01, ic=2)
SMALL = [(128, 0.25), (88, 0.1875), (64, 0.125)]
PICK = [0] * 4 + [1] * 6 + [2] * 9          # 19 samples: 128^2 first (heaviest), then 88^2, 64^2
ITEMS = 4 + 6 + 3                            # one 128^2 or 88^2 sample an item, four 64^2 samples


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_trace_of_the_resident_spectral_queue(gpu_lib):
    mf = gpu_lib
    gs = [mf.Model(n=n, delta=d, nsteps=5, **GAUSS) for n, d in SMALL]
    seeds = np.arange(len(PICK), dtype=np.uint64) + 5
    f0, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in PICK], seeds)      # untraced
    mf.mfmc_trace_enable(1024)
    try:
        f1, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in PICK], seeds)
        rec, dropped = mf.mfmc_trace_read()
        again, _ = mf.mfmc_trace_read()
    finally:
        mf.mfmc_trace_enable(0)
    assert np.array_equal(f0, f1)                   # tracing changes no result
    assert dropped == 0 and len(again) == 0         # a read empties the ring
    assert len(rec) == ITEMS and np.all(rec["kind"] == mf.TRACE_SPECTRAL_QUEUE)
    assert sorted(rec["item"].tolist()) == list(range(ITEMS))
    assert np.all(rec["t1_ns"] > rec["t0_ns"])
    assert np.all(rec["sm"] < _sms()) and len(set(rec["sm"].tolist())) > 1


def test_trace_of_the_mixed_step_queue_and_its_graph(gpu_lib):
    # the step queue's launches are replayed from a captured graph: a shape first captured
    # untraced is captured again once tracing is on; every step's items appear exactly once
    mf = gpu_lib
    common = dict(eps=0.03, tau=5e-3, ic=2, nsteps=3)
    gs = [mf.Model(n=n, delta=R / n, **common) for n, R in [(160, 16), (136, 8)]]
    pick = [0, 1, 1, 0, 1]
    seeds = np.arange(len(pick), dtype=np.uint64) + 71
    f0, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
    mf.mfmc_trace_enable(1 << 16)
    try:
        f1, _ = mf.mfmc_solve_batch_mixed([gs[k] for k in pick], seeds)
        rec, dropped = mf.mfmc_trace_read()
    finally:
        mf.mfmc_trace_enable(0)
    assert np.array_equal(f0, f1) and dropped == 0
    assert len(rec) > 0 and np.all(rec["kind"] == mf.TRACE_MIXED_STEP)
    per_step = [sorted(rec["item"][rec["step"] == s].tolist()) for s in (1, 2, 3)]
    assert per_step[0] == list(range(len(per_step[0]))) and per_step[0] == per_step[1] == per_step[2]
    assert len(rec) == 3 * len(per_step[0])
    # the steps are separate launches in stream order
    assert rec["t1_ns"][rec["step"] == 1].max() <= rec["t0_ns"][rec["step"] == 2].min()
    assert rec["t1_ns"][rec["step"] == 2].max() <= rec["t0_ns"][rec["step"] == 3].min()


def test_trace_of_the_active_set_solver(gpu_lib):
    mf = gpu_lib
    g = mf.Model(n=32, delta=3 / 32, eps=0.03, tau=0.01, nsteps=4, ic=2, beta2=0.05)
    seeds = np.arange(3, dtype=np.uint64) + 640
    mf.mfmc_trace_enable(64)
    try:
        mf.mfmc_solve_batch([g] * 3, seeds)
        rec, dropped = mf.mfmc_trace_read()
    finally:
        mf.mfmc_trace_enable(0)
    assert dropped == 0 and len(rec) == 3
    assert np.all(rec["kind"] == mf.TRACE_ACTIVE_SET) and np.all(rec["step"] == 4)
    assert sorted(rec["item"].tolist()) == [0, 1, 2]


def test_trace_ring_overflow_and_off(gpu_lib):
    mf = gpu_lib
    gs = [mf.Model(n=n, delta=d, nsteps=2, **GAUSS) for n, d in SMALL]
    seeds = np.arange(len(PICK), dtype=np.uint64) + 9
    mf.mfmc_trace_enable(8)
    try:
        mf.mfmc_solve_batch_mixed([gs[k] for k in PICK], seeds)
        rec, dropped = mf.mfmc_trace_read()
        few, dropped_few = None, None
        mf.mfmc_solve_batch_mixed([gs[k] for k in PICK], seeds)
        few, dropped_few = mf.mfmc_trace_read(max_records=3)
    finally:
        mf.mfmc_trace_enable(0)
    assert len(rec) == 8 and dropped == ITEMS - 8            # the newest 8 of 13
    assert len(set(rec["item"].tolist())) == 8
    assert len(few) == 3 and dropped_few == ITEMS - 3
    with pytest.raises(mf.MfmcError) as e:                   # off: nothing to read
        mf.mfmc_trace_read()
    assert e.value.status == mf.MFMC_EINVAL
