"""The library's refresh plan and noise budget (host code of the C ABI,
Section 3.1.3) against the oracle's exact tracker and variance models -- no
GPU needed."""
import math

import pytest

from oracle import noise as Nz
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L

CASES = [(20, 20, -1, 25), (20, 20, -1, 60), (15, 22, -1, 40), (22, 15, -1, 33), (16, 16, 5, 30),
         (16, 16, 2, 11), (12, 12, -1, 11), (30, 30, -1, 0), (9, 9, 3, 0), (1, 1, -1, 5), (1, 17, -1, 12),
         (17, 1, -1, 12), (25, 25, 8, 100), (12, 20, 3, 30), (20, 9, 2, 25), (7, 15, 0, 0)]


@pytest.mark.parametrize("m,n,band,budget", CASES)
def test_plan_matches_oracle(m, n, band, budget):
    ob = None if budget <= 0 else budget
    oband = None if band < 0 else band
    want, worst = Nz.refresh_schedule(m, n, oband, ob)
    got, gworst = L.lvs_noise_plan(m, n, band, budget)
    assert got == want
    assert gworst == worst


def test_plan_rejects_small_budget():
    with pytest.raises(ValueError):
        Nz.refresh_schedule(12, 12, None, 10)
    with pytest.raises(L.LvsError) as ei:
        L.lvs_noise_plan(12, 12, -1, 10)
    assert ei.value.status == L.LVS_ERR_NOISE_BUDGET


@pytest.mark.parametrize("which", ["default", "test"])
def test_budget_matches_oracle(which):
    p = L.lvs_params_default() if which == "default" else L.lvs_params_test()
    op = (T.params_lvs() if which == "default" else T.params_test()).as_dict()
    for lp in (-64.0, -40.0, -10.0):
        a = L.lvs_noise_budget(p, lp)
        b = Nz.noise_budget(op, lp)
        assert abs(a / b - 1) < 1e-9, (lp, a, b)
    # 256 characters need no refresh at the default parameters
    assert 14 * 255 + 10 < L.lvs_noise_budget(L.lvs_params_default(), -64.0)
    assert math.isfinite(L.lvs_noise_budget(p, -64.0))


@pytest.mark.parametrize("which", ["default", "test"])
def test_pfail_matches_oracle(which):
    p = L.lvs_params_default() if which == "default" else L.lvs_params_test()
    op = (T.params_lvs() if which == "default" else T.params_test()).as_dict()
    for kv in (1.0, 3580.0, 1e5, 1e6, 9e6):
        want = math.log2(max(Nz.pfail_of(op, kv), 1e-300))
        assert abs(L.lvs_noise_pfail(p, kv) - want) < 1e-6
    # at the budget for 2^-64 the failure probability is 2^-64
    assert abs(L.lvs_noise_pfail(p, L.lvs_noise_budget(p, -64.0)) + 64) < 1e-6
