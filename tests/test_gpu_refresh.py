"""Refresh of dv / dh by bootstrapping (Section 3.1.3) on the GPU.

With a small noise budget (the paper's example parameter set allows 25
additions) the library refreshes the anti-diagonals its plan chooses; the
result must be bit-exact with the oracle's Algorithm algo_complete run with
the same refreshed anti-diagonals (oracle plan), decrypt to Wagner-Fischer,
and take one extra PBS per refreshed cell.  Also through the band taps, the
DNA pipeline and the preprocessed path; the budget derived from the
parameters refreshes nothing at these lengths.
"""
import random

import numpy as np
import pytest

from oracle import noise as Nz
from oracle import plain as P
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L
from paper_2508_14568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALPHA = {P.ALPHA_ASCII7: L.LVS_ALPHA_ASCII7, P.ALPHA_DNA4: L.LVS_ALPHA_DNA4, P.ALPHA_27: L.LVS_ALPHA_27}


@pytest.fixture(scope="module")
def small():
    ck, sk = L.lvs_keygen(L.lvs_params_test(), 0)
    return ck, L.lvs_ctx_create(sk, 0), T.Keys(T.params_test(), 0)


def _run(ck, ctx, pairs, alpha, seed, budget, band=-1):
    A = [L.lvs_encrypt_string(ck, a, ALPHA[alpha], seed, 2 * k) for k, (a, b) in enumerate(pairs)]
    B = [L.lvs_encrypt_string(ck, b, ALPHA[alpha], seed, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
    pbs0 = L.lvs_ctx_pbs_count(ctx)
    r = L.lvs_edit_distance_batch(ctx, A, B, L.lvs_opts_default(band=band, refresh_budget=budget))
    return r, L.lvs_decrypt_all(ck, r), L.lvs_ctx_pbs_count(ctx) - pbs0


def _refreshed_cells(m, n, diags, band=None):
    return sum(1 for i in range(1, m + 1) for j in range(1, n + 1)
               if i + j in diags and (band is None or abs(i - j) <= band))


@pytest.mark.parametrize("alpha", [P.ALPHA_ASCII7, P.ALPHA_DNA4])
def test_refreshed_rows_bit_exact_vs_oracle(small, alpha):
    ck, ctx, K = small
    pairs = [("kitten!", "sitting"), ("abcd", "dcbaab")] if alpha == P.ALPHA_ASCII7 else \
        [("GATTACAG", "GCATGCTA"), ("ACG", "TTGCA")]
    r, d, npbs = _run(ck, ctx, pairs, alpha, 61, 25)
    extra = 0
    for k, (a, b) in enumerate(pairs):
        diags, _ = Nz.refresh_schedule(len(a), len(b), None, 25)
        assert diags, "the small budget must refresh something"
        extra += _refreshed_cells(len(a), len(b), set(diags))
        xa = T.encrypt_string(K, a, alpha, 61, 2 * k)
        yb = T.encrypt_string(K, b, alpha, 61, 2 * k + 1)
        res = T.lvs_encrypted(K, xa, yb, alpha, parallel=True, refresh=set(diags))
        assert np.array_equal(L.lvs_result_export(r, k, K.big_dim), np.stack(res["h_row"]))
    assert d == [P.wf_distance(a, b) for a, b in pairs]
    per = P.eq_pbs_per_cell(alpha) + 1
    assert npbs == sum(per * len(a) * len(b) for a, b in pairs) + extra


def test_refresh_many_pairs_and_budgets(small):
    ck, ctx, _ = small
    pairs = W.random_pairs(31, 20, W.PRINTABLE[:6], 1, 14)
    for budget in (11, 25, 60, -1, 0):
        r, d, npbs = _run(ck, ctx, pairs, P.ALPHA_ASCII7, 62, budget)
        assert d == [P.wf_distance(a, b) for a, b in pairs]
        extra = 0
        if budget > 0:
            for a, b in pairs:
                diags, _ = Nz.refresh_schedule(len(a), len(b), None, budget)
                extra += _refreshed_cells(len(a), len(b), set(diags))
        assert npbs == sum(3 * len(a) * len(b) for a, b in pairs) + extra


def test_refresh_with_band_taps_bit_exact(small):
    ck, ctx, K = small
    a, b = "kittens!", "sittings"
    for band in (2, 4):
        diags, _ = Nz.refresh_schedule(8, 8, band, 21)
        assert diags
        r, d, _ = _run(ck, ctx, [(a, b)], P.ALPHA_ASCII7, 63, 21, band=band)
        xa = T.encrypt_string(K, a, P.ALPHA_ASCII7, 63, 0)
        yb = T.encrypt_string(K, b, P.ALPHA_ASCII7, 63, 1)
        res = T.lvs_encrypted(K, xa, yb, P.ALPHA_ASCII7, parallel=True, band=band, refresh=set(diags))
        assert np.array_equal(L.lvs_result_export(r, 0, K.big_dim), np.stack(res["diag"]))
        if band == 4:
            assert d[0] == P.wf_distance(a, b)


def test_refresh_preprocessed_path(small):
    ck, ctx, _ = small
    rng = random.Random(5)
    qs = [("".join(rng.choice(W.ALPHA27[:5]) for _ in range(rng.randint(3, 12))),
           "".join(rng.choice(W.ALPHA27[:5]) for _ in range(rng.randint(3, 12)))) for _ in range(6)]
    tables = [L.lvs_preprocess(ctx, L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_27, 64, k)) for k, (a, _) in enumerate(qs)]
    pbs0 = L.lvs_ctx_pbs_count(ctx)
    r = L.lvs_edit_distance_preprocessed_batch(ctx, tables, [b for _, b in qs], L.lvs_opts_default(refresh_budget=25))
    assert L.lvs_decrypt_all(ck, r) == [P.wf_distance(a, b) for a, b in qs]
    extra = sum(_refreshed_cells(len(a), len(b), set(Nz.refresh_schedule(len(a), len(b), None, 25)[0]))
                for a, b in qs)
    assert L.lvs_ctx_pbs_count(ctx) - pbs0 == sum(len(a) * len(b) for a, b in qs) + extra


def test_budget_too_small_is_an_error(small):
    ck, ctx, _ = small
    with pytest.raises(L.LvsError) as ei:
        _run(ck, ctx, [("abcdefgh", "hgfedcba")], P.ALPHA_ASCII7, 65, 10)
    assert ei.value.status == L.LVS_ERR_NOISE_BUDGET


def test_refresh_full_parameters_long_pair():
    """Refresh at the full parameter set on a longer DNA pair with a small
    budget: exact distance, one extra PBS per refreshed cell."""
    ck, sk = L.lvs_keygen(L.lvs_params_default(), 2)
    ctx = L.lvs_ctx_create(sk, 0)
    rng = random.Random(8)
    a = "".join(rng.choice(W.DNA) for _ in range(40))
    b = W.mutate_rate(rng, a, W.DNA, 0.15)
    pairs = [(a, b)]
    r, d, npbs = _run(ck, ctx, pairs, P.ALPHA_DNA4, 66, 30)
    diags, worst = Nz.refresh_schedule(len(a), len(b), None, 30)
    assert worst <= 30 and len(diags) > 5
    assert d == [P.wf_distance(a, b)]
    assert npbs == 2 * len(a) * len(b) + _refreshed_cells(len(a), len(b), set(diags))
    L.lvs_ctx_free(ctx)


def test_split_launches_keep_refreshed_cells_together(small):
    """Steps split over launches of at most `cap` PBS, the split falling at
    many offsets of each step's job list: ciphertexts bit-exact with whole
    steps, distances equal to Wagner-Fischer, the same PBS count.  The two
    LUT_V lookups of a refreshed cell share a launch (the second reads the v
    row the first one writes)."""
    ck, ctx, K = small
    pairs = [("kitten!", "sitting"), ("abcd", "dcbaab"), ("flaw", "lawns")]
    r0, d0, n0 = _run(ck, ctx, pairs, P.ALPHA_ASCII7, 71, 25)
    assert d0 == [P.wf_distance(a, b) for a, b in pairs]
    base = [L.lvs_result_export(r0, k, K.big_dim) for k in range(len(pairs))]
    launches = []
    for cap in (2, 3, 5, 7):
        L.lvs_ctx_set_max_launch_jobs(ctx, cap)
        assert L.lvs_ctx_max_launch_jobs(ctx) == cap
        l0 = L.lvs_ctx_launch_count(ctx)
        r, d, n = _run(ck, ctx, pairs, P.ALPHA_ASCII7, 71, 25)
        launches.append(L.lvs_ctx_launch_count(ctx) - l0)
        assert n == n0 and d == d0, cap
        for k in range(len(pairs)):
            assert np.array_equal(L.lvs_result_export(r, k, K.big_dim), base[k]), (cap, k)
    L.lvs_ctx_set_max_launch_jobs(ctx, 0)
    assert L.lvs_ctx_max_launch_jobs(ctx) == 65536
    assert launches[0] > launches[-1]
    with pytest.raises(L.LvsError):
        L.lvs_ctx_set_max_launch_jobs(ctx, 1)
