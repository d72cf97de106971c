"""Pins of the MFMC oracle (oracle/mfmc_oracle.py): the printed Tables 1 and 2 and
Cases 1-5 of Section 4, the optimality of the allocation against the estimator
variance obtained by expanding Eq. (MFMC_estimator), and brute-force replication."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mfmc_oracle as M
from tests.conftest import read_golden

C1_SECONDS = 63.089


def table1():
    rows = read_golden("table1_pilot_statistics.txt")
    rho = [float(r[3]) for r in rows]
    C = [float(r[4]) for r in rows]
    sigma = [float(r[5]) for r in rows]
    return rho, C, sigma


def as_ordered(members, rho):
    """1-based paper model numbers -> 0-based subset in the order of Eq. (conditiona)."""
    order = M.order_models(rho)
    s = [m - 1 for m in members]
    return [0] + sorted(s[1:], key=order.index)


def test_subset_counts():
    rho, C, _ = table1()
    everything, feas = M.enumerate_subsets(rho, C)
    assert len(everything) == 2 ** 8 - 1 == 255
    assert len(feas) == 131


def test_table2_rows():
    rho, C, _ = table1()
    _, feas = M.enumerate_subsets(rho, C)
    by_v = sorted(feas, key=lambda s: M.variance_reduction_ratio(s, rho, C))
    by_b = sorted(feas, key=lambda s: M.min_budget(s, rho, C))
    highlighted = {1, 2, 28, 93, 126}
    for rank_v, members, V, bmin, rank_b in read_golden("table2_subsets.txt"):
        nums = [int(x) for x in members.split(",")]
        s = as_ordered(nums, rho)
        assert s in feas
        # V is insensitive to the 7-digit rounding of rho: 1e-3 relative.  rho_7 and
        # rho_8 differ by 1e-6, below that rounding, and several unhighlighted rows
        # match with the labels f_7 and f_8 exchanged; either labelling is accepted.
        swapped = as_ordered([{7: 8, 8: 7}.get(x, x) for x in nums], rho)
        cands = [M.variance_reduction_ratio(s, rho, C)]
        if int(rank_v) not in highlighted and (7 in nums or 8 in nums):
            cands.append(M.variance_reduction_ratio(swapped, rho, C))
        assert any(abs(c / float(V) - 1) < 1.5e-3 for c in cands)
        if 1 not in [m - 1 for m in [int(x) for x in members.split(",")]]:
            # B_min of subsets without f_2 is pinned to 0.3 %; with f_2, 1 - rho_2^2 ~ 2e-7
            # is below the printed precision of rho_2 and B_min is unpinned.
            assert M.min_budget(s, rho, C) == pytest.approx(float(bmin), rel=3e-3)
        if int(rank_v) in highlighted:
            assert by_v.index(s) + 1 == int(rank_v)
            assert by_b.index(s) + 1 == int(rank_b)


def test_cases_in_seconds_and_v_ratios():
    rho, C, _ = table1()
    cases = read_golden("cases_bmin_seconds.txt")
    V = {}
    for case, members, v, bsec in cases:
        s = as_ordered([int(x) for x in members.split(",")], rho)
        V[int(case)] = M.variance_reduction_ratio(s, rho, C)
        if int(case) in (2, 3, 4):
            assert M.min_budget(s, rho, C) * C1_SECONDS == pytest.approx(float(bsec), rel=3e-3)
    # Section 4: Case 2 costs a 0.50 % larger V than Case 1, Case 3 a 3.65 % larger one
    assert V[2] / V[1] - 1 == pytest.approx(0.0050, abs=0.0006)
    assert V[3] / V[1] - 1 == pytest.approx(0.0365, abs=0.0006)
    # selection policies: 1 -> Case 1, 2 -> Case 3
    _, _, sigma = table1()
    p1 = M.select(rho, sigma, C, 1e6, policy=1)
    assert p1.subset == as_ordered([1, 2, 3, 9], rho)
    p2 = M.select(rho, sigma, C, 1e6, policy=2)
    assert p2.subset == as_ordered([1, 9], rho)
    # policy 0 at B = 100 C_1: Case 1 needs ~712-795 C_1, Case 2 (36.2 C_1) is next by V
    p0 = M.select(rho, sigma, C, 100.0, policy=0)
    assert p0.subset == as_ordered([1, 3, 9], rho) and not p0.below_min_budget


def test_section3_example_enumeration():
    # Section 3.1 example: four ordered models give the 7 subsets
    # {1,2},{1,3},{1,4},{1,2,3},{1,2,4},{1,3,4},{1,2,3,4} in that order; when {1,4} and
    # {1,2,4} fail Eq. (conditionb) the 5 listed remain, re-indexed in order.  The
    # statistics below (found by a seeded search) realise exactly that case.
    rho = [1.0, 0.991, 0.98, 0.501]
    C = [1.0, 0.787, 6.792, 2.188]
    everything, feas = M.enumerate_subsets(rho, C)
    assert everything == [[0, 1], [0, 2], [0, 3], [0, 1, 2], [0, 1, 3], [0, 2, 3], [0, 1, 2, 3]]
    assert feas == [[0, 1], [0, 2], [0, 1, 2], [0, 2, 3], [0, 1, 2, 3]]
    # the failing subsets violate the condition at a named j
    assert not M.feasible([0, 3], rho, C) and not M.feasible([0, 1, 3], rho, C)


def test_alpha_is_regression_slope():
    # alpha_j = rho sigma_1 / sigma_j is the least-squares slope of f_1 on f_j
    rng = np.random.default_rng(1)
    x = rng.normal(size=5000)
    f1 = 2.0 + 0.3 * x + 0.05 * rng.normal(size=5000)
    f2 = -1.0 + 0.7 * x + 0.02 * rng.normal(size=5000)
    _, sigma, rho = M.pilot_statistics(np.stack([f1, f2]))
    alpha = M.coefficients([0, 1], rho, sigma)
    slope = np.polyfit(f2, f1, 1)[0]
    assert alpha[1] == pytest.approx(slope, rel=1e-10)
    assert rho[1] == pytest.approx(np.corrcoef(f1, f2)[0, 1], rel=1e-12)


def test_allocation_is_optimal_for_the_expanded_variance():
    # At the real-valued allocation of Eqs. (alpha, rk, samples) the variance of the
    # estimator (expanded from Eq. MFMC_estimator) equals V sigma_1^2 C_1 / B, which
    # Eq. (error_theory) restates; and perturbing m along the budget constraint
    # cannot lower it.
    rho, C, sigma = table1()
    _, feas = M.enumerate_subsets(rho, C)
    B = 3000.0
    for s in feas[::7]:
        p = M.plan(s, rho, sigma, C, B)
        if p.below_min_budget:
            continue
        m = p.m_real
        assert sum(C[i] * m[j] for j, i in enumerate(s)) == pytest.approx(B, rel=1e-12)
        assert p.r[0] == pytest.approx(1.0, rel=1e-12)
        var = M.estimator_variance(s, p.alpha, m, rho, sigma)
        s1 = sigma[0]
        assert var == pytest.approx(p.V * s1 * s1 * C[0] / B, rel=1e-6)
        assert p.mse_theory == pytest.approx(var, rel=1e-6)
        assert M.min_budget(s, rho, C) == pytest.approx(B / m[0], rel=1e-10)
        rng = np.random.default_rng(len(s))
        for _ in range(5):
            d = rng.normal(size=len(s)) * 0.01
            mm = [m[j] * (1 + d[j]) for j in range(len(s))]
            scale = B / sum(C[i] * mm[j] for j, i in enumerate(s))
            mm = [x * scale for x in mm]
            if all(mm[j] >= mm[j - 1] for j in range(1, len(s))):
                assert M.estimator_variance(s, p.alpha, mm, rho, sigma) >= var * (1 - 1e-9)


def test_below_min_budget_invariants():
    rho, C, sigma = table1()
    s = as_ordered([1, 3, 9], rho)
    bmin = M.min_budget(s, rho, C)
    need = sum((l + 1) * C[i] for l, i in enumerate(s))
    assert M.below_min_budget(s, rho, C, need * 0.999) is None
    assert M.plan(s, rho, sigma, C, need * 0.999) is None
    prev = None
    for B in np.linspace(need, bmin * 0.999999, 25):
        m = M.below_min_budget(s, rho, C, B)
        assert sum(m[j] * C[i] for j, i in enumerate(s)) <= B * (1 + 1e-12)
        assert all(m[j] >= j + 1 - 1e-12 for j in range(len(s)))
        assert all(m[j] >= m[j - 1] for j in range(1, len(s)))
        prev = m
    # continuity with the closed form as B -> B_min from below
    closed, _ = M.allocation(s, rho, C, bmin)
    assert prev[0] == pytest.approx(1.0)
    assert np.allclose(prev, closed, rtol=1e-4)


def test_mc_and_identical_model_special_cases():
    rng = np.random.default_rng(2)
    f = rng.normal(size=1000)
    assert M.estimate([0], [1.0], [100], [f]) == pytest.approx(M.mc_estimate(f, 100))
    # identical surrogate with alpha = 1: the telescoping sum collapses to the mean
    # of f over the last m
    q = M.estimate([0, 1, 2], [1.0, 1.0, 1.0], [10, 50, 400], [f, f, f])
    assert q == pytest.approx(np.mean(f[:400]), rel=1e-12)


def test_estimator_unbiased_and_variance_by_replication():
    # Synthetic correlated models with known mean: E f_1 = 0.5; 20000 replicates.
    rng = np.random.default_rng(3)
    s = [0, 1, 2]
    rho_true = np.array([1.0, 0.95, 0.8])
    sig = np.array([0.01, 0.012, 0.02])
    C = [1.0, 0.1, 0.01]
    # build f_k = mu_k + sig_k (rho_k z + sqrt(1-rho_k^2) e_k)
    mu = np.array([0.5, 0.45, 0.52])
    alpha = M.coefficients(s, rho_true, sig)
    p = M.plan(s, list(rho_true), list(sig), C, 60.0)
    m = p.m
    reps = 20000
    N = m[-1]
    z = rng.normal(size=(reps, N))
    est = np.empty(reps)
    for rI in range(reps):
        fs = [mu[k] + sig[k] * (rho_true[k] * z[rI] + math.sqrt(1 - rho_true[k] ** 2)
                                * rng.normal(size=N)) for k in s]
        est[rI] = M.estimate(s, alpha, m, fs)
    se = est.std(ddof=1) / math.sqrt(reps)
    assert abs(est.mean() - 0.5) <= 4 * se
    var_theory = M.estimator_variance(s, alpha, m, rho_true, sig)
    assert est.var(ddof=1) == pytest.approx(var_theory, rel=0.05)
    mse = M.mse(0.5, est)
    assert mse == pytest.approx(var_theory, rel=0.06)


@pytest.mark.slow
def test_unbiased_on_the_model_hierarchy_by_permutation():
    # Three fidelities of the nonlocal model on tiny lattices (16^2 R=2, 8^2 R=1 and
    # 16^2 R=1), a pool of seeds, and random permutations of the pool: the mean of
    # the MFMC estimates equals the pool mean of f_1 up to sampling error.
    levels = [O.OracleModel(n=16, delta=2 / 16, eps=0.05, nsteps=30, ic=2, tau=5e-3),
              O.OracleModel(n=16, delta=1 / 16, eps=0.05, nsteps=30, ic=2, tau=5e-3),
              O.OracleModel(n=8, delta=1 / 8, eps=0.05, nsteps=30, ic=2, tau=5e-3)]
    pool = 400
    F = np.array([[lv.solve_sample(1000 + s)[0] for s in range(pool)] for lv in levels])
    _, sigma, rho = M.pilot_statistics(F)
    C = [1.0, 0.4, 0.1]
    order = M.order_models(rho)
    s = [0] + [k for k in order if k != 0]
    if not M.feasible(s, rho, C):
        s = [0, order[1]]
    p = M.plan(s, rho, sigma, C, 40.0)
    rng = np.random.default_rng(4)
    reps = 10000
    est = np.empty(reps)
    for r in range(reps):
        perm = rng.permutation(pool)
        est[r] = M.estimate(s, p.alpha, p.m, [F[k][perm] for k in s])
    se = est.std(ddof=1) / math.sqrt(reps)
    assert abs(est.mean() - F[0].mean()) <= 4 * se
