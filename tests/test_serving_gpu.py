"""Continuous-batching serving: results are the same alone and in a mix of concurrent
requests, admission respects the slot and memory limits, per-request step counts are
honoured, and the results agree with the oracle."""
import time

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

COMMON = dict(eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=5e-3, ic=2)


def models(mf):
    return {64: mf.Model(n=64, delta=2 / 64, nsteps=60, **COMMON),
            128: mf.Model(n=128, delta=4 / 128, nsteps=60, **COMMON),
            256: mf.Model(n=256, delta=8 / 256, nsteps=60, **COMMON)}


def wait(srv, tickets, timeout=120):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout
        time.sleep(0.001)
    return out


def test_alone_and_in_the_mix_are_identical(gpu_lib, ooi_errors):
    mf = gpu_lib
    ms = models(mf)
    probe = [(64, 1234), (128, 99), (256, 7)]
    alone = {}
    for n, seed in probe:
        srv = mf.Server(8 << 30, 64)
        t = srv.submit(ms[n], seed)
        alone[(n, seed)] = wait(srv, [t])[t][0]
        srv.close()
    srv = mf.Server(8 << 30, 256)
    rng = np.random.default_rng(0)
    tickets = {}
    # a long request first (6000 steps): every later request is admitted while it runs
    long_t = srv.submit(ms[256], 4242, params=mf.make_params(1, nsteps=[6000])[0])
    for i in range(120):
        n = int(rng.choice([64, 128, 256], p=[0.5, 0.3, 0.2]))
        tickets[srv.submit(ms[n], 5000 + i)] = (n, 5000 + i)
        if i in (10, 60, 100):
            for pn, ps in probe:
                tickets[srv.submit(ms[pn], ps)] = (pn, ps)
        if i % 20 == 0:
            time.sleep(0.002)   # later requests arrive while earlier ones run
    res = wait(srv, list(tickets) + [long_t])
    st = srv.stats()
    times = {t: srv.times(t) for t in list(tickets) + [long_t]}
    srv.close()
    # a sample's arithmetic does not depend on the cohort it runs in (per-sample tiles or rows
    # summed in a fixed order, the OoI from fixed-order partials): identical OoIs
    for t, (n, seed) in tickets.items():
        if (n, seed) in alone:
            assert res[t][0] == alone[(n, seed)], (n, seed)
    assert st["completed"] == len(tickets) + 1
    # continuous batching, not a queue: requests of different cohorts ran on the device at the
    # same time, and every probe in the mix was admitted while some other request was in flight
    assert st["peak_inflight"] > 1
    for t, (n, seed) in tickets.items():
        if (n, seed) in alone:
            _, a0, d0 = times[t]
            assert any(u != t and a1 < a0 < d1 for u, (_, a1, d1) in times.items()), (n, seed)
    _, a_long, d_long = times[long_t]
    assert sum(1 for t, (_, a, d) in times.items() if t != long_t and a_long < a < d_long) >= 100
    with pytest.raises(mf.MfmcError) as e:
        mf.Server(1 << 20, 2).times(12345)
    assert e.value.status == mf.MFMC_ENOTFOUND
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    # spot check against the oracle
    for t, (n, seed) in list(tickets.items())[:3]:
        o = O.OracleModel(n=n, delta=(n // 32) / n, nsteps=60, **COMMON)
        fr = o.solve_sample(seed)[0]
        ooi_errors.add("served requests in a continuous-batching mix (64^2-256^2, 60 steps)", res[t][0], fr)
        assert abs(res[t][0] - fr) <= 1e-5 * fr


def test_admission_limits(gpu_lib):
    mf = gpu_lib
    ms = models(mf)
    field = 256 * 256 * 4
    budget = 3 * (field + 2 * 272 * 272 * 4 + 4096)   # room for about three 256^2 requests
    srv = mf.Server(budget, 5)
    ts = [srv.submit(ms[256], 10 + i) for i in range(12)] + [srv.submit(ms[64], 50 + i) for i in range(12)]
    wait(srv, ts)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 24
    assert st["peak_bytes"] <= budget
    assert st["peak_inflight"] <= 5


def test_per_request_step_counts(gpu_lib):
    mf = gpu_lib
    ms = models(mf)
    srv = mf.Server(8 << 30, 64)
    steps = [5, 60, 17, 33, 60, 1]
    tickets = []
    for i, k in enumerate(steps):
        p = mf.make_params(1, nsteps=[k])
        tickets.append((srv.submit(ms[256 if i % 2 else 64], 900 + i, params=p[0]), i, k))
    res = wait(srv, [t for t, _, _ in tickets])
    srv.close()
    for t, i, k in tickets:
        n = 256 if i % 2 else 64
        o = O.OracleModel(n=n, delta=(n // 32) / n, nsteps=k, **COMMON)
        fr = o.solve_sample(900 + i)[0]
        assert abs(res[t][0] - fr) <= 1e-5 * fr
    # the batch call honours per-sample step counts too
    p = mf.make_params(len(steps), nsteps=steps)
    f, _ = mf.mfmc_solve_batch([ms[64]] * len(steps), np.arange(len(steps)) + 900, params=p)
    for i, k in enumerate(steps):
        o = O.OracleModel(n=64, delta=2 / 64, nsteps=k, **COMMON)
        assert abs(f[i] - o.solve_sample(900 + i)[0]) <= 1e-5


def test_unknown_ticket_and_bad_requests(gpu_lib):
    mf = gpu_lib
    srv = mf.Server(1 << 20, 4)
    with pytest.raises(mf.MfmcError) as e:
        srv.poll(12345)
    assert e.value.status == mf.MFMC_ENOTFOUND
    big = mf.Model(n=1024, delta=32 / 1024, nsteps=10)
    with pytest.raises(mf.MfmcError) as e:
        srv.submit(big, 1)         # larger than the 1 MiB budget
    assert e.value.status == mf.MFMC_EINVAL
    gauss = mf.Model(n=64, delta=8 / 64, kernel=1, delta_hf=0.25, nsteps=10)
    with pytest.raises(mf.MfmcError):
        srv.submit(gauss, 1)
    srv.close()
