"""Pins for the noise accounting of the oracle (oracle/noise.py) -- no GPU.

- the exact linear tracker against the closed form worked out by hand from
  the recursion of Section 3.1.3, and against a Monte-Carlo propagation of
  independent unit noises through the cell equations (a different algorithm);
- the refresh table LUT_V against the cell equations on all 18 inputs, and
  the refreshed encrypted DP against Wagner-Fischer;
- the greedy refresh schedule: every key within the budget, each refresh
  needed, infeasible budgets rejected;
- the key-switch and modulus-switch variance models against the CPU TFHE
  oracle's own key switch and modulus switch on real ciphertexts, and the
  normal tail used for the failure probability against textbook values.
"""
import math

import numpy as np
import pytest

from oracle import noise as Nz
from oracle import plain as P
from oracle import tfhe as T


@pytest.mark.parametrize("m,n", [(1, 1), (1, 7), (7, 1), (6, 6), (9, 5), (4, 11)])
def test_tracker_equals_closed_form(m, n):
    var = Nz.key_variances(m, n)
    assert set(var) == {(i, j) for i in range(1, m + 1) for j in range(1, n + 1)}
    for (i, j), (vk, vs) in var.items():
        assert vk == Nz.key_variance_closed_form(i, j)
        # the swapped key is the key of the transposed problem
        assert vs == Nz.key_variance_closed_form(j, i)


def test_closed_form_paper_count():
    """Section 3.1.3: with Eq. eq_keyeq2, a diagonal step contributes
    N_H + 4 N_M + 9 N_L = 1 + 4 + 9, plus 1 for EQ9."""
    assert Nz.key_variance_closed_form(1, 1) == 1
    assert Nz.key_variance_closed_form(2, 2) - Nz.key_variance_closed_form(1, 1) == 14
    assert Nz.key_variance_closed_form(256, 256) == 14 * 255 + 1


def _monte_carlo(m, n, band, refresh, trials, seed):
    rng = np.random.default_rng(seed)
    zero = np.zeros(trials)
    v, h, out = {}, {}, {}
    for d in range(2, m + n + 1):
        for i in range(max(1, d - n), min(m, d - 1) + 1):
            j = d - i
            if band is not None and abs(i - j) > band:
                continue
            dv, dh = v.get((i, j - 1), zero), h.get((i - 1, j), zero)
            eq9 = rng.standard_normal(trials)
            out[(i, j)] = (np.var(-dv + 3 * dh + eq9), np.var(3 * dv - dh + eq9))
            if d in refresh:
                v[(i, j)], h[(i, j)] = rng.standard_normal(trials), rng.standard_normal(trials)
            else:
                M = rng.standard_normal(trials)
                v[(i, j)], h[(i, j)] = M - dh, M - dv
    return out


@pytest.mark.parametrize("m,n,band,refresh", [(7, 7, None, ()), (8, 5, None, (6,)), (8, 8, 2, (5, 9)),
                                              (6, 9, None, (4, 5, 11))])
def test_tracker_against_monte_carlo(m, n, band, refresh):
    exact = Nz.key_variances(m, n, band, frozenset(refresh))
    mc = _monte_carlo(m, n, band, frozenset(refresh), 20000, 3)
    assert set(exact) == set(mc)
    for c in exact:
        for a, b in zip(exact[c], mc[c]):
            assert abs(b / a - 1) < 0.08, (c, a, b)


def test_refresh_lut_matches_cell_equations():
    for eq in (0, 1):
        for dh in (-1, 0, 1):
            for dv in (-1, 0, 1):
                want_v, want_h = P.lvs_cell(dv, dh, eq)
                key = P.key_eq2(dv, dh, eq)
                key_sw = P.key_eq2_swapped(dv, dh, eq)
                assert P.lookup(P.LUT_V, key) == want_v % 32
                assert P.lookup(P.LUT_V, key_sw) == want_h % 32


def test_schedule_properties():
    for (m, n, band, budget) in [(20, 20, None, 25), (20, 20, None, 60), (15, 22, None, 40), (16, 16, 5, 30),
                                 (12, 12, None, 11)]:
        chosen, worst = Nz.refresh_schedule(m, n, band, budget)
        var = Nz.key_variances(m, n, band, frozenset(chosen))
        assert worst == max(max(x) for x in var.values()) <= budget
        for d in chosen:
            # as late as possible: without refreshing d, diagonal d + 1 exceeds the budget
            others = frozenset(c for c in chosen if c != d)
            var2 = Nz.key_variances(m, n, band, others)
            assert max(max(x) for (i, j), x in var2.items() if i + j == d + 1) > budget
    chosen, worst = Nz.refresh_schedule(30, 30, None, None)
    assert chosen == [] and worst == 14 * 29 + 1     # at (30, 30)
    big = Nz.refresh_schedule(30, 30, None, 10 ** 6)
    assert big == ([], 14 * 29 + 1)
    with pytest.raises(ValueError):
        Nz.refresh_schedule(12, 12, None, 10)


@pytest.fixture(scope="module")
def keys():
    return T.Keys(T.params_test(), 0)


def test_refreshed_encrypted_dp_matches_wf(keys):
    a, b = "kitt", "sitn"
    chosen, _ = Nz.refresh_schedule(4, 4, None, 25)
    assert chosen
    xa = T.encrypt_string(keys, a, P.ALPHA_ASCII7, 9, 0)
    yb = T.encrypt_string(keys, b, P.ALPHA_ASCII7, 9, 1)
    r1 = T.lvs_encrypted(keys, xa, yb, P.ALPHA_ASCII7, parallel=True, refresh=set(chosen))
    assert T.decrypt_distance(keys, r1["h_row"], 4) == P.wf_distance(a, b)
    ncells = sum(1 for i in range(1, 5) for j in range(1, 5) if i + j in chosen)
    assert r1["pbs"] == 3 * 16 + ncells
    r2 = T.lvs_encrypted(keys, xa, yb, P.ALPHA_ASCII7, parallel=False, refresh=set(chosen))
    for x, y in zip(r1["h_row"], r2["h_row"]):
        assert np.array_equal(x, y)


def _signed(x):
    x = int(x) % 2**64
    return x - 2**64 if x >= 2**63 else x


def test_keyswitch_and_modswitch_variance_models(keys):
    p = keys.params
    pd = p.as_dict()
    count = 1500
    ks_err, ms_err = [], []
    step = 2**64 // (2 * p.N)
    for t in range(count):
        mu = t % 32
        ct = T.encrypt(keys, mu, 77, 3, t)
        small = T.keyswitch(keys, ct)
        ph_small = (int(small[-1]) - sum(int(a) * int(s) for a, s in zip(small[:-1], keys.lwe_key))) % 2**64
        ks_err.append(_signed(ph_small - T.phase(keys, ct)))
        ms = T.modswitch(keys, small)
        ph_ms = (int(ms[-1]) - sum(int(a) * int(s) for a, s in zip(ms[:-1], keys.lwe_key))) * step % 2**64
        ms_err.append(_signed(ph_ms - ph_small))
    ks_err = np.array(ks_err, dtype=np.float64)
    ms_err = np.array(ms_err, dtype=np.float64)
    w_big = int(np.sum(keys.glwe_key))
    w_small = int(np.sum(keys.lwe_key))
    r_ks = np.mean(ks_err ** 2) / Nz.var_keyswitch(pd, w_big)
    r_ms = np.mean(ms_err ** 2) / Nz.var_modswitch(pd, w_small)
    assert 0.85 < r_ks < 1.15, r_ks
    assert 0.85 < r_ms < 1.15, r_ms


def test_normal_tail_textbook_values():
    assert abs(Nz.z_for_pfail(-1) - 0.6744897501960817) < 1e-9       # median of |X|
    assert abs(math.erfc(Nz.z_for_pfail(math.log2(0.05)) / math.sqrt(2)) - 0.05) < 1e-12
    assert abs(Nz.z_for_pfail(math.log2(0.05)) - 1.959963984540054) < 1e-9


def test_budget_and_pfail_consistent():
    p = T.params_lvs().as_dict()
    b = Nz.noise_budget(p, -64)
    assert abs(math.log2(Nz.pfail_of(p, b)) + 64) < 1e-6
    # the configurations (at most 256 characters) stay far inside the budget
    assert Nz.key_variance_closed_form(256, 256) < b
    assert Nz.pfail_of(p, 14 * 255 + 10) < 2.0 ** -80


def test_output_variances_closed_form():
    """dv_out = M - dh_in and dh_out = M - dv_in: along the diagonal each step
    adds two unit terms, so for a full matrix var h[i][j] = 2j - 1 (i >= j) or
    2i (i < j), and var v[i][j] = 2i - 1 (j >= i) or 2j (j < i)."""
    out = Nz.output_variances(9, 7)
    for (i, j), (vv, vh) in out.items():
        assert vh == (2 * j - 1 if i >= j else 2 * i)
        assert vv == (2 * i - 1 if j >= i else 2 * j)


def test_pbs_output_variance_model(keys):
    """var_pbs (Section 2.2's bootstrap noise) against the oracle's own
    bootstraps: the phase error of 768 PBS outputs, with the keys' actual
    weights, has the predicted variance (the gadget rounding term dominates at
    this parameter set, the key-noise term is checked by the full-size GPU
    measurement)."""
    p = keys.params
    pd = p.as_dict()
    count = 768
    msgs = [t % 16 for t in range(count)]
    lut = [(3 * x + 1) % 16 for x in range(16)]
    cts = np.stack([T.encrypt(keys, m, 91, 4, t) for t, m in enumerate(msgs)])
    out = T.pbs_many(keys, cts, np.tile(np.asarray(lut, np.uint32), (count, 1)))
    err = np.array([_signed(T.phase(keys, out[t]) - lut[m] * T.DELTA) for t, m in enumerate(msgs)],
                   dtype=np.float64)
    w_lwe, w_glwe = int(np.sum(keys.lwe_key)), int(np.sum(keys.glwe_key))
    ratio = np.mean(err ** 2) / Nz.var_pbs(pd, w_lwe, w_glwe)
    assert 0.8 < ratio < 1.2, ratio
    # the expected-weight form is the same model at weights n/2 and kN/2
    assert Nz.var_pbs(pd) == Nz.var_pbs(pd, p.n / 2, p.k * p.N / 2)


def test_modswitch_body_term():
    """A ciphertext with a zero mask leaves only the body's rounding to a
    multiple of 2^64 / 2N: variance step^2 / 12, the weight-0 case of the
    modulus-switch model."""
    K = T.Keys(T.params_test(), 2)
    p = K.params
    step = 2**64 // (2 * p.N)
    rng = np.random.default_rng(5)
    bodies = rng.integers(0, 2**63, size=4000, dtype=np.int64).astype(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=4000, dtype=np.int64).astype(np.uint64)
    err = []
    for b in bodies:
        small = np.zeros(p.n + 1, dtype=np.uint64)
        small[-1] = b
        ms = T.modswitch(K, small)
        assert not ms[:-1].any()
        err.append(_signed(int(ms[-1]) * step - int(b)))
    ratio = np.mean(np.array(err, dtype=np.float64) ** 2) / Nz.var_modswitch(p.as_dict(), 0)
    assert 0.93 < ratio < 1.07, ratio


@pytest.mark.parametrize("level,base_log", [(1, 3), (2, 3), (5, 3), (2, 4), (3, 5)])
def test_balanced_digit_second_moment_by_enumeration(level, base_log):
    """Every value of the top level * base_log bits, decomposed by the oracle:
    all digits lie in [-B/2, B/2) and their mean square is the model's E[d^2]."""
    beta = level * base_log
    B = 2 ** base_log
    sq, cnt = 0, 0
    for v in range(2 ** beta):
        d = T.decompose(v << (64 - beta), level, base_log)
        assert all(-B // 2 <= x < B // 2 for x in d)
        sq += sum(x * x for x in d)
        cnt += level
    assert abs(sq / cnt - Nz.balanced_digit_sq(base_log)) < 1e-12
