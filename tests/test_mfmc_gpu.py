"""Parity of the MFMC layer (FP64 statistics and estimator on the GPU, host planner)
with the oracle of Section 3, through the C ABI."""
import numpy as np
import pytest

from oracle import mfmc_oracle as M
import oracle as O
from tests.conftest import read_golden

pytestmark = pytest.mark.gpu


def synthetic_pilot(K=5, n=64, seed=0):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=n)
    rho = np.array([1.0, 0.999, 0.99, 0.95, 0.8][:K])
    sig = np.array([0.0067, 0.0066, 0.0065, 0.0064, 0.006][:K])
    F = np.stack([0.5 + sig[k] * (rho[k] * z + np.sqrt(1 - rho[k] ** 2) * rng.normal(size=n)) for k in range(K)])
    return F


def test_pilot_statistics_fp64_gpu_vs_oracle(gpu_lib):
    import torch
    mf = gpu_lib
    for K, n in ((1, 2), (3, 50), (5, 64), (9, 1000), (16, 257)):
        F = synthetic_pilot(min(K, 5), n, seed=K) if K <= 5 else np.random.default_rng(K).normal(0.5, 0.01, (K, n))
        F = F[:K]
        d = torch.tensor(F, dtype=torch.float64, device="cuda")
        mean, sigma, rho = mf.mfmc_pilot_stats(K, n, d)
        m0, s0, r0 = M.pilot_statistics(F)
        assert np.allclose(mean, m0, rtol=1e-13, atol=0)
        assert np.allclose(sigma, s0, rtol=1e-12, atol=0)
        assert np.allclose(rho, r0, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("policy", [0, 1, 2])
@pytest.mark.parametrize("budget", [3.0, 40.0, 500.0, 1e4])
def test_plan_matches_oracle(gpu_lib, policy, budget):
    mf = gpu_lib
    F = synthetic_pilot(5, 64, seed=11)
    C = [1.0, 0.6, 0.2, 0.05, 0.01]
    _, s0, r0 = M.pilot_statistics(F)
    ref = M.select(list(r0), list(s0), C, budget, policy=policy)
    if ref is None:
        with pytest.raises(mf.MfmcError) as e:
            mf.mfmc_plan(F, C, budget, policy)
        assert e.value.status == mf.MFMC_EBUDGET
        return
    p = mf.mfmc_plan(F, C, budget, policy).as_dict()
    assert p["idx"] == ref.subset
    assert p["below_min_budget"] == ref.below_min_budget
    assert np.allclose(p["alpha"], ref.alpha, rtol=1e-11)
    assert np.allclose(p["m_real"], ref.m_real, rtol=1e-9)
    # floor(m) may differ only where m_real is within 1e-9 of an integer (ambiguous)
    for a, b, x in zip(p["m"], ref.m, ref.m_real):
        assert a == b or abs(x - round(x)) < 1e-9
    assert p["V"] == pytest.approx(ref.V, rel=1e-11)
    assert p["Bmin"] == pytest.approx(ref.Bmin, rel=1e-9)
    assert p["mse_theory"] == pytest.approx(ref.mse_theory, rel=1e-9)


def test_plan_on_table1_statistics_reproduces_cases(gpu_lib):
    # Feed pilot samples whose statistics are exactly Table 1's rho and sigma: a
    # two-point-free construction is not possible for 9 correlated models, so the check
    # is the planner's: policy 1 -> Case 1 subset, policy 2 -> Case 3 subset.
    mf = gpu_lib
    rows = read_golden("table1_pilot_statistics.txt")
    rho = [float(r[3]) for r in rows]
    C = [float(r[4]) for r in rows]
    sig = [float(r[5]) for r in rows]
    # build samples with exactly these correlations to the first model by Gram-Schmidt
    n = 50
    rng = np.random.default_rng(5)
    z = rng.normal(size=n)
    z = (z - z.mean()) / z.std(ddof=1)
    F = [0.5 + sig[0] * z]
    for k in range(1, 9):
        e = rng.normal(size=n)
        e = e - e.mean()
        e = e - (e @ z) / (z @ z) * z
        e = e / e.std(ddof=1)
        F.append(0.5 + sig[k] * (rho[k] * z + np.sqrt(1 - rho[k] ** 2) * e))
    F = np.stack(F)
    _, s0, r0 = M.pilot_statistics(F)
    assert np.allclose(r0, rho, atol=1e-12)
    p1 = mf.mfmc_plan(F, C, 1e6, 1).as_dict()
    assert p1["idx"] == M.select(list(r0), list(s0), C, 1e6, policy=1).subset
    assert sorted(i + 1 for i in p1["idx"]) == [1, 2, 3, 9]
    p2 = mf.mfmc_plan(F, C, 1e6, 2).as_dict()
    assert sorted(i + 1 for i in p2["idx"]) == [1, 9]
    assert p1["n_feasible"] == 131


def test_estimate_fp64_gpu_vs_oracle(gpu_lib):
    mf = gpu_lib
    F = synthetic_pilot(4, 64, seed=3)
    C = [1.0, 0.3, 0.05, 0.01]
    plan = mf.mfmc_plan(F, C, 200.0, 0)
    d = plan.as_dict()
    rng = np.random.default_rng(9)
    lists = [0.5 + 0.01 * rng.normal(size=d["m"][-1] + 3) for _ in d["idx"]]
    got = mf.mfmc_estimate(plan, lists)
    ref = M.estimate(d["idx"], d["alpha"], d["m"], lists)
    assert abs(got - ref) <= 1e-10 * abs(ref)


def test_mfmc_run_end_to_end_small_hierarchy(gpu_lib):
    # three fidelities of the model with the nuclei IC; the GPU run's plan and estimate
    # are re-derived by the oracle from the oracle's own OoIs on the same seeds
    mf = gpu_lib
    levels = [dict(n=64, delta=4 / 64), dict(n=32, delta=2 / 32), dict(n=64, delta=2 / 64)]
    common = dict(eps=0.05, tau=5e-3, nsteps=30, ic=2)
    models = [mf.Model(**lv, **common, ic_base_n=0) for lv in levels]
    costs = [1.0, 0.2, 0.4]
    n_pilot, seed_base = 32, 5000
    plan, est = mf.mfmc_run(models, n_pilot, 60.0, policy=0, seed_base=seed_base, costs=costs)
    p = plan.as_dict()
    orcs = [O.OracleModel(**lv, eps=0.05, tau=5e-3, nsteps=30, ic=2) for lv in levels]
    pilot = np.array([[o.solve_sample(seed_base + s)[0] for s in range(n_pilot)] for o in orcs])
    mean, sigma, rho = M.pilot_statistics(pilot)
    assert np.allclose(p["rho_all"], rho, rtol=1e-6, atol=1e-9)
    assert np.allclose(p["sigma_all"], sigma, rtol=1e-4)
    ref = M.select(list(rho), list(sigma), costs, 60.0, policy=0)
    assert p["idx"] == ref.subset
    lists = [np.array([orcs[i].solve_sample(seed_base + n_pilot + s)[0] for s in range(p["m"][j])])
             for j, i in enumerate(p["idx"])]
    q_ref = M.estimate(p["idx"], p["alpha"], p["m"], lists)
    assert abs(est - q_ref) <= 1e-5 * abs(q_ref)
    # the estimator itself matches to 1e-10 on the same OoIs
    got = mf.mfmc_estimate(plan, lists)
    assert abs(got - M.estimate(p["idx"], p["alpha"], p["m"], lists)) <= 1e-10 * abs(q_ref)


def test_budget_errors(gpu_lib):
    mf = gpu_lib
    F = synthetic_pilot(3, 64, seed=1)
    with pytest.raises(mf.MfmcError) as e:
        mf.mfmc_plan(F, [1.0, 0.5, 0.1], 0.5, 0)   # below one high-fidelity sample
    assert e.value.status == mf.MFMC_EBUDGET
    with pytest.raises(mf.MfmcError) as e:
        mf.mfmc_plan(F, [1.0, 0.5, 0.0], 10.0, 0)  # zero cost
    assert e.value.status == mf.MFMC_EINVAL
