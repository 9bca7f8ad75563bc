// Noise budget of the Leuvenshtein DP and the refresh plan (host code).
//
// Section 3.1.3 ("Limiting the noise growth"): in units of the variance of a
// fresh bootstrap output, each M and each EQ9 is an independent unit noise,
// dv_out = M - dh_in and dh_out = M - dv_in, and the key
// (1 - dv_in) + 3 (1 + dh_in) + EQ9 of Eq. eq_keyeq2 has variance
//   var(dv_in) + 9 var(dh_in) - 6 cov(dv_in, dh_in) + 1.
// When a key would exceed the budget, the dv / dh of an earlier anti-diagonal
// are refreshed by a bootstrap (they become fresh units).  A refreshed cell
// computes dv_out = PBS(key; LUT_V) and dh_out = PBS(key'; LUT_V), key' being
// the key with dv_in and dh_in exchanged, so its swapped key must fit the
// budget too.
//
// The plan propagates, per cell c, var(v_c), var(h_c) and cov(v_c, h_c).  For
// c = (i, j) with left neighbour L = (i, j-1), upper neighbour U = (i-1, j) and
// diagonal neighbour D = (i-1, j-1):
//   cov(v_L, h_U) = cov(h_D, v_D) if L and U are both ordinary cells, else 0
// (v_L = M_L - h_D and h_U = M_U - v_D; the M are independent), and for an
// ordinary cell var(v_c) = 1 + var(h_U), var(h_c) = 1 + var(v_L),
// cov(v_c, h_c) = 1 + cov(h_U, v_L).  Boundary cells and cells outside the
// band are noiseless constants; refreshed cells output two fresh units.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lvs_internal.hpp"

namespace lvs {

namespace {

struct CellNoise {
    double vv = 0, vh = 0, x = 0;   // var(v), var(h), cov(v, h)
    uint8_t kind = 0;               // 0 constant, 1 ordinary, 2 refreshed
};

struct Planner {
    size_t m, n;
    long band;
    // three anti-diagonals (d - 2, d - 1, d), indexed by i
    std::vector<CellNoise> dg[3];

    Planner(size_t m_, size_t n_, long band_) : m(m_), n(n_), band(band_)
    {
        for (auto &v : dg) v.assign(m + 2, CellNoise{});
    }
    bool computed(size_t i, size_t j) const
    {
        if (i < 1 || j < 1 || i > m || j > n) return false;
        if (band < 0) return true;
        const long k = (long)j - (long)i, delta = (long)n - (long)m;
        return std::min(0L, delta) - band <= k && k <= std::max(0L, delta) + band;
    }
    // cell (i, d - i) of slot s (0: d-2, 1: d-1, 2: d)
    const CellNoise &at(int s, size_t i, size_t d) const
    {
        static const CellNoise none{};
        if (i < 1 || i > m || d < i + 1 || !computed(i, d - i)) return none;
        return dg[s][i];
    }
    // key and swapped-key variances of (i, j) on diagonal d (slots 0, 1 hold d-2, d-1)
    void key_var(size_t i, size_t d, double &vk, double &vs) const
    {
        const CellNoise &L = at(1, i, d - 1), &U = at(1, i - 1, d - 1), &D = at(0, i - 1, d - 2);
        const double c = (L.kind == 1 && U.kind == 1) ? D.x : 0.0;
        vk = L.vv + 9.0 * U.vh - 6.0 * c + 1.0;
        vs = 9.0 * L.vv + U.vh - 6.0 * c + 1.0;
    }
    // outputs of diagonal d into slot 2
    void outputs(size_t d, bool refreshed)
    {
        for (size_t i = 1; i <= m; ++i) {
            CellNoise o;
            if (d >= i + 1 && d - i <= n && computed(i, d - i)) {
                if (refreshed) {
                    o.vv = o.vh = 1.0;
                    o.x = 0.0;
                    o.kind = 2;
                } else {
                    const CellNoise &L = at(1, i, d - 1), &U = at(1, i - 1, d - 1), &D = at(0, i - 1, d - 2);
                    const double c = (L.kind == 1 && U.kind == 1) ? D.x : 0.0;
                    o.vv = 1.0 + U.vh;
                    o.vh = 1.0 + L.vv;
                    o.x = 1.0 + c;
                    o.kind = 1;
                }
            }
            dg[2][i] = o;
        }
    }
    double diag_cost(size_t d) const
    {
        double worst = 0;
        for (size_t i = std::max<size_t>(1, d > n ? d - n : 1); i <= m && i + 1 <= d; ++i) {
            if (!computed(i, d - i)) continue;
            double vk, vs;
            key_var(i, d, vk, vs);
            worst = std::max(worst, std::max(vk, vs));
        }
        return worst;
    }
    void shift()
    {
        std::swap(dg[0], dg[1]);
        std::swap(dg[1], dg[2]);
    }
};

double tuniform_var(uint32_t b) { return (std::ldexp(1.0, 2 * (int)b + 1) + 1.0) / 6.0; }
double digit_sq(uint32_t base_log) { const double B = std::ldexp(1.0, (int)base_log); return (B * B + 2.0) / 12.0; }

}  // namespace

lvs_status noise_plan(size_t m, size_t n, long band, double budget, std::vector<uint8_t> *refresh, double *worst_out)
{
    if (refresh) refresh->assign(m + n + 1, 0);
    double worst = 0;
    if (m == 0 || n == 0) {
        if (worst_out) *worst_out = 0;
        return LVS_OK;
    }
    Planner pl(m, n, band);
    // diagonal d's keys depend on d-1 and d-2; decide d's refresh by looking at d+1
    for (size_t d = 2; d <= m + n; ++d) {
        // slots: 0 = d-2, 1 = d-1 (already final)
        const double cost = pl.diag_cost(d);
        if (budget > 0 && cost > budget)
            return set_error(LVS_ERR_NOISE_BUDGET, "noise budget " + std::to_string(budget) +
                                                        " too small: a key needs " + std::to_string(cost));
        worst = std::max(worst, cost);
        pl.outputs(d, false);
        if (budget > 0 && d < m + n) {
            pl.shift();
            const double next = pl.diag_cost(d + 1);
            // undo the shift to keep slot 2 = d while deciding
            std::swap(pl.dg[1], pl.dg[2]);
            std::swap(pl.dg[0], pl.dg[1]);
            if (next > budget) {
                pl.outputs(d, true);
                if (refresh) (*refresh)[d] = 1;
            }
        }
        pl.shift();
    }
    if (worst_out) *worst_out = worst;
    return LVS_OK;
}

namespace {
struct BootstrapVariances {
    double pbs, ks, ms;   // torus Z_2^64, binary keys of expected weight half their length
};

BootstrapVariances bootstrap_variances(const lvs_params &p)
{
    BootstrapVariances v;
    const double big = (double)p.k * p.N;
    const int beta_pbs = (int)(p.pbs_level * p.pbs_base_log);
    const double r_pbs = std::ldexp(1.0, 2 * (63 - beta_pbs)) / 3.0;
    v.pbs = (p.n / 2.0) * (1.0 + big / 2.0) * r_pbs +
            (double)p.n * (p.k + 1) * p.pbs_level * p.N * digit_sq(p.pbs_base_log) * tuniform_var(p.glwe_noise_log2);
    const int beta_ks = (int)(p.ks_level * p.ks_base_log);
    v.ks = (big / 2.0) * std::ldexp(1.0, 2 * (63 - beta_ks)) / 3.0 +
           big * p.ks_level * digit_sq(p.ks_base_log) * tuniform_var(p.lwe_noise_log2);
    const double step = std::ldexp(1.0, 64) / (2.0 * p.N);
    v.ms = (1.0 + p.n / 2.0) * step * step / 12.0;
    return v;
}
}  // namespace

double noise_budget(const lvs_params &p, double log2_pfail)
{
    const BootstrapVariances v = bootstrap_variances(p);
    // z with erfc(z / sqrt 2) = 2^log2_pfail
    const double target = std::exp2(log2_pfail);
    double lo = 0, hi = 40;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (std::erfc(mid / std::sqrt(2.0)) > target) lo = mid;
        else hi = mid;
    }
    const double z = 0.5 * (lo + hi);
    const double room = std::pow(std::ldexp(1.0, 58) / z, 2) - v.ks - v.ms;
    return room / v.pbs;
}

// log2 of the probability that a key of key_var PBS-output variances (plus the
// key-switch and modulus-switch noise) leaves the half-step 2^58: erfc(2^58 / (sigma sqrt 2))
double noise_log2_pfail(const lvs_params &p, double key_var)
{
    const BootstrapVariances v = bootstrap_variances(p);
    const double sigma = std::sqrt(key_var * v.pbs + v.ks + v.ms);
    const double x = std::ldexp(1.0, 58) / (sigma * std::sqrt(2.0));
    const double pf = std::erfc(x);
    if (pf > 0) return std::log2(pf);
    // erfc(x) ~ exp(-x^2) / (x sqrt(pi)) for large x
    return (-x * x - std::log(x * std::sqrt(3.14159265358979323846))) / std::log(2.0);
}

lvs_status plan_refresh(const lvs_ctx *ctx, int32_t refresh_budget, PairRows &P)
{
    P.refresh.clear();
    if (refresh_budget < 0 || P.m == 0 || P.n == 0) return LVS_OK;
    const double budget = refresh_budget > 0 ? (double)refresh_budget : noise_budget(ctx->P.p, -64.0);
    if (budget < 1.0) return set_error(LVS_ERR_NOISE_BUDGET, "the parameter set leaves no noise budget");
    // full matrix: the largest key is 14 (min(m, n) - 1) + 10 (+ the swapped key's symmetric term)
    if (P.band < 0 && 14.0 * ((double)std::min(P.m, P.n) - 1.0) + 10.0 <= budget) return LVS_OK;
    std::vector<uint8_t> r;
    lvs_status st = noise_plan(P.m, P.n, P.band, budget, &r, nullptr);
    if (st != LVS_OK) return st;
    if (std::find(r.begin(), r.end(), 1) != r.end()) P.refresh = std::move(r);
    return LVS_OK;
}

}  // namespace lvs

using namespace lvs;

extern "C" {

lvs_status lvs_noise_budget(const lvs_params *p, double log2_pfail, double *budget)
{
    if (!p || !budget) return set_error(LVS_ERR_ARG, "lvs_noise_budget: NULL argument");
    lvs_status st = check_params(*p);
    if (st != LVS_OK) return st;
    if (!(log2_pfail < 0) || log2_pfail < -1000) return set_error(LVS_ERR_ARG, "lvs_noise_budget: log2_pfail out of range");
    *budget = noise_budget(*p, log2_pfail);
    return LVS_OK;
}

lvs_status lvs_noise_pfail(const lvs_params *p, double key_var, double *log2_pfail)
{
    if (!p || !log2_pfail) return set_error(LVS_ERR_ARG, "lvs_noise_pfail: NULL argument");
    lvs_status st = check_params(*p);
    if (st != LVS_OK) return st;
    if (!(key_var >= 0)) return set_error(LVS_ERR_ARG, "lvs_noise_pfail: negative variance");
    *log2_pfail = noise_log2_pfail(*p, key_var);
    return LVS_OK;
}

lvs_status lvs_noise_plan(size_t m, size_t n, int32_t band, double budget, uint8_t *refresh, double *max_key_var)
{
    std::vector<uint8_t> r;
    double worst = 0;
    lvs_status st = noise_plan(m, n, band, budget, &r, &worst);
    if (st != LVS_OK) return st;
    if (refresh) std::copy(r.begin(), r.end(), refresh);
    if (max_key_var) *max_key_var = worst;
    return LVS_OK;
}

}  // extern "C"
