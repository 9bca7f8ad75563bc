"""Banded Leuvenshtein (Algorithm alg_levenshtein's |i - j| <= band, Section
3.2: "Exact Skip" with band = floor(m/2), approximate with smaller bands; for
m != n the band widened to the diagonals between 0 and n - m) on the GPU: the
readout path is bit-exact with the oracle's banded run, the distance equals
Wagner-Fischer for the exact bands and the plaintext banded oracle otherwise,
and fewer PBS run."""
import numpy as np
import pytest

from oracle import plain as P
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L
from paper_2508_14568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALPHA = {P.ALPHA_ASCII7: L.LVS_ALPHA_ASCII7, P.ALPHA_DNA4: L.LVS_ALPHA_DNA4}


@pytest.fixture(scope="module")
def small():
    ck, sk = L.lvs_keygen(L.lvs_params_test(), 0)
    return ck, L.lvs_ctx_create(sk, 0), T.Keys(T.params_test(), 0)


def _banded_plain(a, b, band):
    m = len(a)
    E9 = [[0] * (m + 1) for _ in range(m + 1)]
    for i in range(1, m + 1):
        for j in range(1, m + 1):
            E9[i][j] = 9 if a[i - 1] == b[j - 1] else 0
    h, v = P.lvs_on_eq9(E9, m, m, band=band)
    return P.readout_diagonal(h, v, m)


def _run(ck, ctx, pairs, alpha, band, seed):
    A = [L.lvs_encrypt_string(ck, a, ALPHA[alpha], seed, 2 * k) for k, (a, b) in enumerate(pairs)]
    B = [L.lvs_encrypt_string(ck, b, ALPHA[alpha], seed, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
    pbs0 = L.lvs_ctx_pbs_count(ctx)
    r = L.lvs_edit_distance_batch(ctx, A, B, L.lvs_opts_default(band=band))
    d = L.lvs_decrypt_all(ck, r)
    return r, d, L.lvs_ctx_pbs_count(ctx) - pbs0


@pytest.mark.parametrize("alpha,pool", [(P.ALPHA_ASCII7, W.PRINTABLE[:6]), (P.ALPHA_DNA4, W.DNA)])
def test_exact_skip_band_equals_wf(small, alpha, pool):
    ck, ctx, _ = small
    import random
    rng = random.Random(7)
    pairs = []
    for _ in range(24):
        m = rng.randint(1, 12)
        pairs.append(("".join(rng.choice(pool) for _ in range(m)), "".join(rng.choice(pool) for _ in range(m))))
    for band_of in (lambda m: m // 2, lambda m: m):
        bands = {band_of(len(a)) for a, _ in pairs}
        for band in bands:
            sel = [p for p in pairs if band_of(len(p[0])) == band]
            r, d, npbs = _run(ck, ctx, sel, alpha, band, 11)
            assert d == [P.wf_distance(a, b) for a, b in sel]
            per = P.eq_pbs_per_cell(alpha) + 1
            assert npbs == sum(per * P.band_cells(len(a), band) for a, _ in sel)


def test_approximate_band_matches_plain_oracle(small):
    ck, ctx, _ = small
    pairs = W.random_pairs(5, 30, W.PRINTABLE[:5], 6, 6) + [("abcdefgh", "hgfedcba"), ("aaaaaaaa", "bbbbbbbb")]
    pairs = [(a, b[:len(a)].ljust(len(a), "a")) for a, b in pairs]
    for band in (0, 1, 2):
        r, d, _ = _run(ck, ctx, pairs, P.ALPHA_ASCII7, band, 12)
        assert d == [_banded_plain(a, b, band) for a, b in pairs]
        assert all(x >= P.wf_distance(a, b) for x, (a, b) in zip(d, pairs))


def test_band_path_bit_exact_vs_oracle(small):
    ck, ctx, K = small
    pairs = [("kitten", "sittin"), ("GATC", "GTTC")]
    for k, (a, b) in enumerate(pairs):
        alpha = P.ALPHA_DNA4 if k == 1 else P.ALPHA_ASCII7
        for band in (1, 3):
            r, d, _ = _run(ck, ctx, [(a, b)], alpha, band, 13)
            xa = T.encrypt_string(K, a, alpha, 13, 0)
            yb = T.encrypt_string(K, b, alpha, 13, 1)
            res = T.lvs_encrypted(K, xa, yb, alpha, parallel=True, band=band)
            got = L.lvs_result_export(r, 0, K.big_dim)
            assert np.array_equal(got, np.stack(res["diag"]))
            assert d[0] == T.decrypt_path(K, res["diag"])


def test_non_square_band_bit_exact_and_exact(small):
    """m != n: the band widened to the diagonals between 0 and n - m
    (plain.in_band) with the path readout; exact from band ceil(min/2) on,
    bit-exact with the oracle's banded run, and PBS only inside the band."""
    ck, ctx, K = small
    cases = [("kitten", "sitting!!", P.ALPHA_ASCII7), ("GATTACAGA", "GCAT", P.ALPHA_DNA4),
             ("ab", "abcdefg", P.ALPHA_ASCII7), ("TTTTTTT", "T", P.ALPHA_DNA4)]
    for k, (a, b, alpha) in enumerate(cases):
        m, n = len(a), len(b)
        for band in sorted({0, 1, (min(m, n) + 1) // 2}):
            r, d, npbs = _run(ck, ctx, [(a, b)], alpha, band, 15 + k)
            xa = T.encrypt_string(K, a, alpha, 15 + k, 0)
            yb = T.encrypt_string(K, b, alpha, 15 + k, 1)
            res = T.lvs_encrypted(K, xa, yb, alpha, parallel=True, band=band)
            assert np.array_equal(L.lvs_result_export(r, 0, K.big_dim), np.stack(res["path"]))
            E9 = [[9 if i and j and a[i - 1] == b[j - 1] else 0 for j in range(n + 1)] for i in range(m + 1)]
            h, v = P.lvs_on_eq9(E9, m, n, band=band)
            assert d[0] == P.readout_path(h, v, m, n) == T.decrypt_path(K, res["path"])
            assert d[0] >= P.wf_distance(a, b)
            if band >= (min(m, n) + 1) // 2:
                assert d[0] == P.wf_distance(a, b)
            assert npbs == (P.eq_pbs_per_cell(alpha) + 1) * P.band_cells_general(m, n, band)


def test_non_square_band_batch_mixed_lengths(small):
    ck, ctx, _ = small
    import random
    rng = random.Random(21)
    pairs = []
    for _ in range(30):
        m, n = rng.randint(1, 11), rng.randint(1, 11)
        pairs.append(("".join(rng.choice("abcd") for _ in range(m)), "".join(rng.choice("abcd") for _ in range(n))))
    band = 6    # >= ceil(min(m, n) / 2) for every pair: exact
    r, d, npbs = _run(ck, ctx, pairs, P.ALPHA_ASCII7, band, 22)
    assert d == [P.wf_distance(a, b) for a, b in pairs]
    assert npbs == sum(3 * P.band_cells_general(len(a), len(b), band) for a, b in pairs)


def test_preprocessed_path_with_band(small):
    """The band (and its path readout) on the preprocessed path of Section 5:
    exact from ceil(min(m,n)/2), the plaintext banded oracle otherwise."""
    ck, ctx, _ = small
    import random
    rng = random.Random(33)
    qs = [("".join(rng.choice(W.ALPHA27[:5]) for _ in range(rng.randint(2, 10))),
           "".join(rng.choice(W.ALPHA27[:5]) for _ in range(rng.randint(2, 10)))) for _ in range(8)]
    tables = L.lvs_preprocess_batch(ctx, [L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_27, 34, k)
                                          for k, (a, _) in enumerate(qs)])
    for band in (1, 5):
        pbs0 = L.lvs_ctx_pbs_count(ctx)
        r = L.lvs_edit_distance_preprocessed_batch(ctx, tables, [b for _, b in qs], L.lvs_opts_default(band=band))
        d = L.lvs_decrypt_all(ck, r)
        want = []
        for a, b in qs:
            m, n = len(a), len(b)
            E9 = [[9 if i and j and a[i - 1] == b[j - 1] else 0 for j in range(n + 1)] for i in range(m + 1)]
            h, v = P.lvs_on_eq9(E9, m, n, band=band)
            want.append(P.readout_path(h, v, m, n))
        assert d == want
        if band == 5:
            assert d == [P.wf_distance(a, b) for a, b in qs]
        assert L.lvs_ctx_pbs_count(ctx) - pbs0 == sum(P.band_cells_general(len(a), len(b), band) for a, b in qs)
