"""MFMC oracle (test infrastructure only): plain FP64 Python of Section 3.

Follows the paper's steps in its order and notation:
  pilot statistics sigma_k, rho_{1,k}             (Section 3.1, the three bullet items)
  ordering by decreasing rho_{1,k}^2              (Eq. conditiona)
  enumeration of subsets containing f_1 and the
  feasibility test                                (Eq. conditionb)
  variance reduction ratio V                      (Eq. variance_reduction_ratio)
  coefficients alpha_j, ratios r_j, samples m_j   (Eqs. alpha, rk, samples)
  minimum budget B_min                            (Eq. bmin)
  rounding down of m_j                            (the Remark after Eq. bmin)
  below-minimum-budget allocation                 (the modified algorithm of Section 4,
                                                   Eq. below_min_budget)
  the telescoping estimator                       (Eq. MFMC_estimator)
  empirical and theoretical MSE                   (Eqs. mse_error, error_theory)

Readings where the paper is silent (the choices this oracle makes):
  * ties in rho^2 are broken by model index (stable sort);
  * a zero denominator in Eq. (conditionb) makes the subset infeasible;
  * variances use the n-1 convention (rho and alpha do not depend on it);
  * in the below-minimum-budget loop the budget already spent on the fixed models
    is sum_{l<=j} m_l C_{i_l} with the current values of m_l; this equals the
    printed sum_{l<=j} l C_{i_l} whenever the loop fixes j = 1, 2, ... in turn;
  * model i_j is evaluated on the first m_j samples of one shared sample sequence
    (nested samples), and Q^{(i_j)}_{m_{j-1}} uses the first m_{j-1} of them.
Model indices here are 0-based: model 0 is the high-fidelity model f_1.
"""
from dataclasses import dataclass
from itertools import combinations
from typing import List, Optional, Sequence

import numpy as np


def pilot_statistics(F: np.ndarray):
    """F[k, s] = OoI of model k on pilot sample s.  Returns (mean, sigma, rho_1k)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[1]
    mean = F.mean(axis=1)
    D = F - mean[:, None]
    var = (D * D).sum(axis=1) / (n - 1)
    sigma = np.sqrt(var)
    cov1 = (D[0][None, :] * D).sum(axis=1) / (n - 1)
    rho = cov1 / (sigma[0] * sigma)
    return mean, sigma, rho


def order_models(rho: Sequence[float]) -> List[int]:
    """Eq. (conditiona): indices sorted by decreasing rho^2, ties by index."""
    rho = np.asarray(rho, dtype=np.float64)
    return sorted(range(len(rho)), key=lambda k: (-(rho[k] ** 2), k))


def _rho2_next(rho2: Sequence[float], j: int) -> float:
    return rho2[j + 1] if j + 1 < len(rho2) else 0.0


def feasible(subset: Sequence[int], rho, C) -> bool:
    """Eq. (conditionb) for j = 2..|S| (1-based), rho_{i_{|S|+1}} = 0."""
    r2 = [rho[i] ** 2 for i in subset]
    for j in range(1, len(subset)):
        num = r2[j - 1] - r2[j]
        den = r2[j] - _rho2_next(r2, j)
        if den <= 0.0:
            return False
        if not (C[subset[j - 1]] / C[subset[j]] > num / den):
            return False
    return True


def variance_reduction_ratio(subset: Sequence[int], rho, C) -> float:
    """Eq. (variance_reduction_ratio)."""
    r2 = [rho[i] ** 2 for i in subset]
    s = 0.0
    for j, i in enumerate(subset):
        s += np.sqrt(C[i] / C[subset[0]] * (r2[j] - _rho2_next(r2, j)))
    return s * s


def min_budget(subset: Sequence[int], rho, C) -> float:
    """Eq. (bmin): B_min = C_1 sqrt(V / (1 - rho_{1,i_2}^2))."""
    V = variance_reduction_ratio(subset, rho, C)
    return C[subset[0]] * np.sqrt(V / (1.0 - rho[subset[1]] ** 2))


def enumerate_subsets(rho, C):
    """All 2^(K-1)-1 subsets {f_1} + nonempty set of surrogates, members in the order
    of Eq. (conditiona).  Returns (all_subsets, feasible_subsets)."""
    order = order_models(rho)
    assert order[0] == 0, "model 0 must be the high-fidelity model (rho = 1)"
    surr = order[1:]
    everything = []
    for size in range(1, len(surr) + 1):
        for comb in combinations(surr, size):
            everything.append([0] + list(comb))
    keep = [s for s in everything if feasible(s, rho, C)]
    return everything, keep


def coefficients(subset, rho, sigma):
    """Eq. (alpha): alpha_j = rho_{1,i_j} sigma_1 / sigma_{i_j} (alpha_1 unused, = 1)."""
    return [1.0] + [rho[i] * sigma[subset[0]] / sigma[i] for i in subset[1:]]


def ratios(subset, rho, C):
    """Eq. (rk)."""
    r2 = [rho[i] ** 2 for i in subset]
    denom = 1.0 - r2[1]
    return [np.sqrt(C[subset[0]] * (r2[j] - _rho2_next(r2, j)) / (C[i] * denom))
            for j, i in enumerate(subset)]


def allocation(subset, rho, C, B):
    """Eq. (samples): real-valued m_j (before rounding)."""
    r = ratios(subset, rho, C)
    m1 = B / sum(C[i] * r[j] for j, i in enumerate(subset))
    return [m1 * rj for rj in r], r


def below_min_budget(subset, rho, C, B):
    """The below-minimum-budget allocation of Section 4 (steps 1-5 of the modified
    algorithm).  Returns real-valued m_j, or None when B < sum_l l C_{i_l}."""
    k = len(subset)
    if B < sum((l + 1) * C[i] for l, i in enumerate(subset)):
        return None
    r2 = [rho[i] ** 2 for i in subset]
    m, _ = allocation(subset, rho, C, B)                       # step 1
    while True:
        bad = [j for j in range(k - 1) if m[j] < j + 1]         # step 2 (1-based j <= |S|-1)
        if not bad:
            break
        j = bad[0]                                             # step 3
        m[j] = float(j + 1)
        jp = j + 1                                             # 0-based index of i_{j+1}
        r = [0.0] * k
        for l in range(jp, k):                                 # step 4
            r[l] = np.sqrt(C[subset[jp]] * (r2[l] - _rho2_next(r2, l)) /
                           (C[subset[l]] * (r2[jp] - _rho2_next(r2, jp))))
        spent = sum(m[q] * C[subset[q]] for q in range(jp))    # step 5 (reading)
        m_next = (B - spent) / sum(C[subset[l]] * r[l] for l in range(jp, k))
        for l in range(jp, k):
            m[l] = m_next * r[l]
    return m


@dataclass
class Plan:
    subset: List[int]
    alpha: List[float]
    r: List[float]
    m_real: List[float]
    m: List[int]
    V: float
    Bmin: float
    below_min_budget: bool
    mse_theory: float


def plan(subset, rho, sigma, C, B) -> Optional[Plan]:
    """Coefficients and sample counts for one subset and budget B."""
    V = variance_reduction_ratio(subset, rho, C)
    Bmin = min_budget(subset, rho, C)
    alpha = coefficients(subset, rho, sigma)
    m_real, r = allocation(subset, rho, C, B)
    m1_star = m_real[0]
    below = B < Bmin
    if below:
        m_real = below_min_budget(subset, rho, C, B)
        if m_real is None:
            return None
    m = [int(np.floor(x)) for x in m_real]                     # Remark: round down
    s1 = sigma[subset[0]]
    mse = s1 * s1 * (1.0 - rho[subset[1]] ** 2) * B / (m1_star * m1_star * C[subset[0]])
    return Plan(list(subset), alpha, r, m_real, m, V, Bmin, below, mse)


def select(rho, sigma, C, B, policy=0, explicit=None) -> Optional[Plan]:
    """Subset selection. 0: smallest V with B >= B_min, else the smallest-V subset that
    admits the below-minimum-budget branch; 1: smallest V regardless of B_min;
    2: smallest B_min; 3: the explicit subset."""
    _, feas = enumerate_subsets(rho, C)
    if policy == 3:
        return plan(list(explicit), rho, sigma, C, B)
    if policy == 1:
        best = min(feas, key=lambda s: variance_reduction_ratio(s, rho, C))
        return plan(best, rho, sigma, C, B)
    if policy == 2:
        best = min(feas, key=lambda s: min_budget(s, rho, C))
        return plan(best, rho, sigma, C, B)
    by_v = sorted(feas, key=lambda s: variance_reduction_ratio(s, rho, C))
    for s in by_v:
        if B >= min_budget(s, rho, C):
            return plan(s, rho, sigma, C, B)
    for s in by_v:
        p = plan(s, rho, sigma, C, B)
        if p is not None:
            return p
    return None


def estimate(subset, alpha, m, samples: Sequence[np.ndarray]) -> float:
    """Eq. (MFMC_estimator).  samples[j] holds model i_j on the shared sample sequence
    (at least m_j values); Q^{(i_j)}_{m} is the mean of its first m values."""
    q = float(np.mean(np.asarray(samples[0][:m[0]], dtype=np.float64)))
    for j in range(1, len(subset)):
        x = np.asarray(samples[j], dtype=np.float64)
        q += alpha[j] * (float(np.mean(x[:m[j]])) - float(np.mean(x[:m[j - 1]])))
    return q


def mc_estimate(f: np.ndarray, M: int) -> float:
    """Eq. (mc)."""
    return float(np.mean(np.asarray(f[:M], dtype=np.float64)))


def mse(q_ref: float, estimates: Sequence[float]) -> float:
    """Eq. (mse_error) over the given replicate estimates."""
    e = np.asarray(estimates, dtype=np.float64)
    return float(np.mean((q_ref - e) ** 2))


def estimator_variance(subset, alpha, m, rho, sigma) -> float:
    """Variance of Eq. (MFMC_estimator) for nested samples, by expanding the
    telescoping sum: sigma_1^2/m_1 + sum_j (1/m_{j-1} - 1/m_j)
    (alpha_j^2 sigma_j^2 - 2 alpha_j rho_j sigma_1 sigma_j)."""
    s1 = sigma[subset[0]]
    v = s1 * s1 / m[0]
    for j in range(1, len(subset)):
        i = subset[j]
        v += (1.0 / m[j - 1] - 1.0 / m[j]) * (alpha[j] ** 2 * sigma[i] ** 2
                                              - 2.0 * alpha[j] * rho[i] * s1 * sigma[i])
    return v
