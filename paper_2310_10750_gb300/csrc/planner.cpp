// Host-side MFMC model selection and sample allocation in FP64 (Section 3):
// ordering (Eq. conditiona), subset feasibility (Eq. conditionb), variance reduction
// ratio (Eq. variance_reduction_ratio), alpha / r / m (Eqs. alpha, rk, samples), B_min
// (Eq. bmin), rounding down (the Remark after Eq. bmin), the below-minimum-budget
// allocation of Section 4 (Eq. below_min_budget) and the theoretical MSE
// (Eq. error_theory).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mfmc_internal.h"

namespace mfmc {

namespace {

struct Stats {
    std::vector<double> rho2, C;
};

double rho2_after(const std::vector<int> &S, const Stats &st, size_t j) {
    return j + 1 < S.size() ? st.rho2[S[j + 1]] : 0.0;
}

bool is_feasible(const std::vector<int> &S, const Stats &st) {
    for (size_t j = 1; j < S.size(); ++j) {
        const double num = st.rho2[S[j - 1]] - st.rho2[S[j]];
        const double den = st.rho2[S[j]] - rho2_after(S, st, j);
        if (!(den > 0.0)) return false;
        if (!(st.C[S[j - 1]] / st.C[S[j]] > num / den)) return false;
    }
    return true;
}

double ratio_V(const std::vector<int> &S, const Stats &st) {
    double s = 0.0;
    for (size_t j = 0; j < S.size(); ++j)
        s += std::sqrt(st.C[S[j]] / st.C[S[0]] * (st.rho2[S[j]] - rho2_after(S, st, j)));
    return s * s;
}

double budget_min(const std::vector<int> &S, const Stats &st) {
    return st.C[S[0]] * std::sqrt(ratio_V(S, st) / (1.0 - st.rho2[S[1]]));
}

std::vector<double> closed_form_r(const std::vector<int> &S, const Stats &st) {
    std::vector<double> r(S.size());
    const double den = 1.0 - st.rho2[S[1]];
    for (size_t j = 0; j < S.size(); ++j)
        r[j] = std::sqrt(st.C[S[0]] * (st.rho2[S[j]] - rho2_after(S, st, j)) / (st.C[S[j]] * den));
    return r;
}

std::vector<double> closed_form_m(const std::vector<int> &S, const Stats &st, double B) {
    std::vector<double> r = closed_form_r(S, st), m(S.size());
    double cr = 0.0;
    for (size_t j = 0; j < S.size(); ++j) cr += st.C[S[j]] * r[j];
    for (size_t j = 0; j < S.size(); ++j) m[j] = B / cr * r[j];
    return m;
}

// Section 4 branch for B < B_min.  Returns false if B < sum_l l C_{i_l}.  The budget
// already spent on the fixed models is sum_{l<=j} m_l C_{i_l} with their current values.
bool below_branch(const std::vector<int> &S, const Stats &st, double B, std::vector<double> &m) {
    const size_t k = S.size();
    double need = 0.0;
    for (size_t l = 0; l < k; ++l) need += (double)(l + 1) * st.C[S[l]];
    if (B < need) return false;
    m = closed_form_m(S, st, B);
    for (;;) {
        size_t j = k;
        for (size_t q = 0; q + 1 < k; ++q)
            if (m[q] < (double)(q + 1)) {
                j = q;
                break;
            }
        if (j == k) break;
        m[j] = (double)(j + 1);
        const size_t jp = j + 1;
        std::vector<double> r(k, 0.0);
        const double den = st.rho2[S[jp]] - rho2_after(S, st, jp);
        for (size_t l = jp; l < k; ++l)
            r[l] = std::sqrt(st.C[S[jp]] * (st.rho2[S[l]] - rho2_after(S, st, l)) / (st.C[S[l]] * den));
        double spent = 0.0, cr = 0.0;
        for (size_t q = 0; q < jp; ++q) spent += m[q] * st.C[S[q]];
        for (size_t l = jp; l < k; ++l) cr += st.C[S[l]] * r[l];
        const double mn = (B - spent) / cr;
        for (size_t l = jp; l < k; ++l) m[l] = mn * r[l];
    }
    return true;
}

}  // namespace

mfmc_status plan_from_stats(int K, const double *mean, const double *sigma, const double *rho,
                            const double *costs, double budget, int policy, const int *explicit_idx,
                            int explicit_len, mfmc_plan_t *out) {
    if (K < 1 || K > MFMC_MAX_MODELS) return fail(MFMC_EINVAL, "K must be in [1, %d]", MFMC_MAX_MODELS);
    if (!(budget > 0)) return fail(MFMC_EINVAL, "budget must be > 0");
    for (int k = 0; k < K; ++k)
        if (!(costs[k] > 0)) return fail(MFMC_EINVAL, "cost of model %d must be > 0", k);
    if (policy < 0 || policy > 3) return fail(MFMC_EINVAL, "unknown policy");
    Stats st;
    st.rho2.resize(K);
    st.C.assign(costs, costs + K);
    for (int k = 0; k < K; ++k) st.rho2[k] = rho[k] * rho[k];

    std::memset(out, 0, sizeof(*out));
    out->n_models = K;
    out->budget = budget;
    for (int k = 0; k < K; ++k) {
        out->rho_all[k] = rho[k];
        out->sigma_all[k] = sigma[k];
        out->mean_all[k] = mean[k];
    }

    std::vector<int> best;
    if (K == 1) {
        // Monte Carlo (Eq. mc): the whole budget on f_1
        out->K_sel = 1;
        out->idx[0] = 0;
        out->rho[0] = 1.0;
        out->sigma[0] = sigma[0];
        out->cost[0] = costs[0];
        out->alpha[0] = 1.0;
        out->r[0] = 1.0;
        out->m_real[0] = budget / costs[0];
        out->m[0] = (int64_t)std::floor(out->m_real[0]);
        out->V = 1.0;
        out->Bmin = costs[0];
        out->mse_theory = sigma[0] * sigma[0] / out->m_real[0];
        if (out->m[0] < 1) return fail(MFMC_EBUDGET, "budget below one high-fidelity sample");
        return MFMC_OK;
    }

    // Eq. (conditiona): surrogates by decreasing rho^2, ties by model index
    std::vector<int> order;
    for (int k = 1; k < K; ++k) order.push_back(k);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return st.rho2[a] > st.rho2[b]; });

    // every subset {f_1} + nonempty set of surrogates, by size then lexicographic position
    std::vector<std::vector<int>> feas;
    const int m_s = K - 1;
    for (int size = 1; size <= m_s; ++size) {
        std::vector<int> pos(size);
        for (int i = 0; i < size; ++i) pos[i] = i;
        for (;;) {
            std::vector<int> S{0};
            for (int p : pos) S.push_back(order[p]);
            if (is_feasible(S, st)) feas.push_back(S);
            int i = size - 1;
            while (i >= 0 && pos[i] == m_s - size + i) --i;
            if (i < 0) break;
            ++pos[i];
            for (int q = i + 1; q < size; ++q) pos[q] = pos[q - 1] + 1;
        }
    }
    out->n_feasible = (int)feas.size();

    std::vector<double> m_real;
    bool below = false;
    auto try_plan = [&](const std::vector<int> &S) -> bool {
        if (budget >= budget_min(S, st)) {
            m_real = closed_form_m(S, st, budget);
            below = false;
            return true;
        }
        below = true;
        return below_branch(S, st, budget, m_real);
    };

    if (policy == 3) {
        if (!explicit_idx || explicit_len < 2 || explicit_len > K || explicit_idx[0] != 0)
            return fail(MFMC_EINVAL, "explicit subset must start with model 0 and hold 2..K models");
        std::vector<int> S(explicit_idx, explicit_idx + explicit_len);
        for (int v : S)
            if (v < 0 || v >= K) return fail(MFMC_EINVAL, "explicit subset index out of range");
        std::vector<int> tail(S.begin() + 1, S.end());
        std::stable_sort(tail.begin(), tail.end(), [&](int a, int b) { return st.rho2[a] > st.rho2[b]; });
        S.assign(1, 0);
        S.insert(S.end(), tail.begin(), tail.end());
        if (!try_plan(S)) return fail(MFMC_EBUDGET, "budget below sum_l l C_{i_l} for the explicit subset");
        best = S;
    } else {
        if (feas.empty()) return fail(MFMC_EBUDGET, "no feasible subset");
        if (policy == 1 || policy == 2) {
            size_t bi = 0;
            for (size_t i = 1; i < feas.size(); ++i) {
                const double a = policy == 1 ? ratio_V(feas[i], st) : budget_min(feas[i], st);
                const double b = policy == 1 ? ratio_V(feas[bi], st) : budget_min(feas[bi], st);
                if (a < b) bi = i;
            }
            best = feas[bi];
            if (!try_plan(best)) return fail(MFMC_EBUDGET, "budget below sum_l l C_{i_l} for the selected subset");
        } else {
            std::vector<size_t> byv(feas.size());
            for (size_t i = 0; i < feas.size(); ++i) byv[i] = i;
            std::stable_sort(byv.begin(), byv.end(),
                             [&](size_t a, size_t b) { return ratio_V(feas[a], st) < ratio_V(feas[b], st); });
            for (size_t i : byv)
                if (budget >= budget_min(feas[i], st)) {
                    best = feas[i];
                    break;
                }
            if (best.empty())
                for (size_t i : byv) {
                    std::vector<double> tmp;
                    if (below_branch(feas[i], st, budget, tmp)) {
                        best = feas[i];
                        break;
                    }
                }
            if (best.empty()) return fail(MFMC_EBUDGET, "the budget admits no subset");
            try_plan(best);
        }
    }

    const std::vector<double> r = closed_form_r(best, st);
    const std::vector<double> m_star = closed_form_m(best, st, budget);
    out->K_sel = (int)best.size();
    out->V = ratio_V(best, st);
    out->Bmin = budget_min(best, st);
    out->below_min_budget = below ? 1 : 0;
    for (size_t j = 0; j < best.size(); ++j) {
        const int i = best[j];
        out->idx[j] = i;
        out->rho[j] = rho[i];
        out->sigma[j] = sigma[i];
        out->cost[j] = costs[i];
        out->alpha[j] = j == 0 ? 1.0 : rho[i] * sigma[0] / sigma[i];
        out->r[j] = r[j];
        out->m_real[j] = m_real[j];
        out->m[j] = (int64_t)std::floor(m_real[j]);
    }
    const double s1 = sigma[0];
    out->mse_theory = s1 * s1 * (1.0 - st.rho2[best[1]]) * budget / (m_star[0] * m_star[0] * costs[0]);
    return MFMC_OK;
}

}  // namespace mfmc
