"""Pins for the CPU TFHE oracle (oracle/tfhe_oracle.c) -- no GPU.

The oracle is checked against: the published SplitMix64 output, exact
enumeration of the TUniform sampler, polynomial products over Python integers,
algebraic identities of X^N = -1, the gadget recomposition bound, closed forms
of blind rotation and sample extraction, decryption of keys and PBS outputs, and
the LUT tables printed in the paper (tests/golden/).
"""
import random

import numpy as np
import pytest

from oracle import plain as P
from oracle import tfhe as T
from tests.conftest import golden_lines

MASK = 2**64 - 1


@pytest.fixture(scope="module")
def keys():
    return T.Keys(T.params_test(), 0)


def test_splitmix64_published_value():
    # first output of SplitMix64 seeded with 0 (reference implementation)
    assert T.sm64(0) == 0xE220A8397B1DCDAF
    # c-th output from state K is mix(K + (c+1) * gamma): consecutive outputs
    assert T.word(0, 0) == 0xE220A8397B1DCDAF
    assert T.word(0, 1) == T.sm64(0x9E3779B97F4A7C15)


def test_tuniform_exact_distribution():
    b = 3
    counts = {}
    for w in range(1 << (b + 2)):
        e = T.tuniform(w, b)
        counts[e] = counts.get(e, 0) + 1
    assert sorted(counts) == list(range(-(1 << b), (1 << b) + 1))
    assert counts[-(1 << b)] == counts[1 << b] == 1
    assert all(counts[e] == 2 for e in range(-(1 << b) + 1, 1 << b))
    # only the low b+2 bits matter
    assert T.tuniform(0xFFFF0000_00000005, b) == T.tuniform(5, b)


def _poly_mul_ints(a, b, N):
    full = [0] * (2 * N)
    for i in range(N):
        for j in range(N):
            full[i + j] += int(a[i]) * int(b[j])
    return [(full[t] - full[t + N]) % 2**64 for t in range(N)]


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_negacyclic_mul_against_integer_product(N):
    rng = random.Random(N)
    for _ in range(5):
        a = np.array([rng.getrandbits(64) for _ in range(N)], dtype=np.uint64)
        b = np.array([rng.getrandbits(64) for _ in range(N)], dtype=np.uint64)
        assert [int(x) for x in T.negacyclic_mul(a, b)] == _poly_mul_ints(a, b, N)


def test_rotation_identities():
    N = 16
    rng = random.Random(1)
    a = np.array([rng.getrandbits(64) for _ in range(N)], dtype=np.uint64)
    # X^N = -1
    assert [int(x) for x in T.poly_rotate(a, N)] == [(-int(x)) % 2**64 for x in a]
    for r in range(2 * N):
        mono = np.zeros(N, dtype=np.uint64)
        if r < N:
            mono[r] = 1
        else:
            mono[r - N] = np.uint64(MASK)       # -1
        assert np.array_equal(T.poly_rotate(a, r), T.negacyclic_mul(a, mono))
        back = T.poly_rotate(T.poly_rotate(a, r), (2 * N - r) % (2 * N))
        assert np.array_equal(back, a)


@pytest.mark.parametrize("level,base_log", [(2, 13), (5, 3), (1, 23)])
def test_decomposition_recomposes_within_rounding(level, base_log):
    rng = random.Random(level * 100 + base_log)
    beta = level * base_log
    for _ in range(2000):
        a = rng.getrandbits(64)
        d = T.decompose(a, level, base_log)
        B = 1 << base_log
        assert all(-B // 2 <= x < B // 2 for x in d)
        rec = sum(x * (1 << (64 - (lev + 1) * base_log)) for lev, x in enumerate(d)) % 2**64
        err = (a - rec) % 2**64
        err = err - 2**64 if err >= 2**63 else err
        assert abs(err) <= 1 << (63 - beta)
    # exact multiples of the last gadget recompose exactly
    for _ in range(200):
        a = (rng.getrandbits(beta) << (64 - beta)) % 2**64
        d = T.decompose(a, level, base_log)
        rec = sum(x * (1 << (64 - (lev + 1) * base_log)) for lev, x in enumerate(d)) % 2**64
        assert rec == a


def test_keygen_deterministic_and_seeded():
    p = T.params_test()
    k1, k2, k3 = T.Keys(p, 7), T.Keys(p, 7), T.Keys(p, 8)
    for f in ("lwe_key", "glwe_key", "bsk", "ksk"):
        assert np.array_equal(getattr(k1, f), getattr(k2, f))
        assert not np.array_equal(getattr(k1, f), getattr(k3, f))
    assert set(np.unique(k1.lwe_key)) <= {0, 1} and set(np.unique(k1.glwe_key)) <= {0, 1}
    assert 0.3 < k1.lwe_key.mean() < 0.7 and 0.4 < k1.glwe_key.mean() < 0.6


def test_bsk_rows_decrypt_to_gadget_messages(keys):
    """Each GGSW row r = j*l + lev-1 of BSK_i is a GLWE whose phase polynomial
    is s_i * q / B^lev on coefficient 0 of component j (j < k: the mask part
    contributes -s_i * g * S_j), plus TUniform noise."""
    p = keys.params
    N, k, l = p.N, p.k, p.pbs_level
    bsk = keys.bsk.reshape(p.n, (k + 1) * l, k + 1, N)
    S = keys.glwe_key.reshape(k, N)
    for i in (0, 1, p.n - 1):
        for j in range(k + 1):
            for lev in range(1, l + 1):
                row = bsk[i, j * l + lev - 1]
                ph = row[k].copy()
                for jj in range(k):
                    ph = ph - T.negacyclic_mul(row[jj], S[jj])
                g = 1 << (64 - lev * p.pbs_base_log)
                msg = np.zeros(N, dtype=np.uint64)
                if j == k:
                    msg[0] = np.uint64((int(keys.lwe_key[i]) * g) % 2**64)
                else:
                    msg = T.negacyclic_mul(np.array([(int(keys.lwe_key[i]) * g) % 2**64] + [0] * (N - 1),
                                                    dtype=np.uint64), S[j])
                    msg = (np.zeros(N, dtype=np.uint64) - msg)
                e = (ph - msg).astype(np.uint64)
                es = e.astype(np.int64)
                assert np.all(np.abs(es) <= (1 << p.glwe_noise_log2))


def test_ksk_rows_decrypt_under_small_key(keys):
    p = keys.params
    ksk = keys.ksk.reshape(p.k * p.N, p.ks_level, p.n + 1)
    for u in (0, 5, p.k * p.N - 1):
        for lev in range(1, p.ks_level + 1):
            row = ksk[u, lev - 1]
            ph = (int(row[-1]) - sum(int(a) * int(s) for a, s in zip(row[:-1], keys.lwe_key))) % 2**64
            e = (ph - int(keys.glwe_key[u]) * (1 << (64 - lev * p.ks_base_log))) % 2**64
            e = e - 2**64 if e >= 2**63 else e
            assert abs(e) <= 1 << p.lwe_noise_log2


def test_encrypt_decrypt_all_plaintexts(keys):
    for mu in range(32):
        ct = T.encrypt(keys, mu, 3, 1, mu)
        assert T.decrypt(keys, ct) == mu
        err = (T.phase(keys, ct) - mu * T.DELTA) % 2**64
        err = err - 2**64 if err >= 2**63 else err
        assert abs(err) <= 1 << keys.params.glwe_noise_log2


def test_keyswitch_preserves_message(keys):
    for mu in range(32):
        ct = T.encrypt(keys, mu, 4, 2, mu)
        assert T.decrypt_small(keys, T.keyswitch(keys, ct)) == mu


def test_modswitch_closed_form(keys):
    p = keys.params
    twoN = 2 * p.N
    rng = random.Random(2)
    vals = [rng.randrange(twoN) for _ in range(p.n + 1)]
    exact = np.array([(v * (2**64 // twoN)) % 2**64 for v in vals], dtype=np.uint64)
    assert list(T.modswitch(keys, exact)) == vals
    # just below the rounding midpoint stays, at the midpoint rounds up (wraps at 2N)
    half = 2**64 // twoN // 2
    x = np.array([(v * (2**64 // twoN) + half - 1) % 2**64 for v in vals], dtype=np.uint64)
    assert list(T.modswitch(keys, x)) == vals
    x = np.array([(v * (2**64 // twoN) + half) % 2**64 for v in vals], dtype=np.uint64)
    assert list(T.modswitch(keys, x)) == [(v + 1) % twoN for v in vals]


def test_lut_poly_closed_form(keys):
    p = keys.params
    N, box = p.N, p.N // 16
    f = list(range(3, 19))
    v = T.lut_poly(keys, f)
    for t in range(N):
        if t < N - box // 2:
            want = (f[(t + box // 2) // box] % 32) * T.DELTA
        else:
            want = (-(f[0] % 32) * T.DELTA) % 2**64
        assert int(v[t]) == want % 2**64


def test_blind_rotate_zero_mask_closed_form(keys):
    """With every a_i = 0 each CMux adds the external product of 0, which is
    exactly 0: the accumulator stays X^{-b} v (masks zero)."""
    p = keys.params
    v = T.lut_poly(keys, P.LUT_MIN)
    for b in (0, 1, 77, p.N, 2 * p.N - 1):
        ms = np.zeros(p.n + 1, dtype=np.uint32)
        ms[-1] = b
        acc = T.blind_rotate(keys, ms, v)
        assert np.all(acc[: p.k * p.N] == 0)
        assert np.array_equal(acc[p.k * p.N:], T.poly_rotate(v, (2 * p.N - b) % (2 * p.N)))


def test_sample_extract_phase_is_coefficient_zero(keys):
    p = keys.params
    N, k = p.N, p.k
    rng = np.random.default_rng(3)
    acc = rng.integers(0, 2**63, size=(k + 1) * N, dtype=np.uint64) * np.uint64(2)
    lwe = T.sample_extract(keys, acc)
    S = keys.glwe_key.reshape(k, N)
    ph = acc[k * N:].copy()
    for j in range(k):
        ph = ph - T.negacyclic_mul(acc[j * N:(j + 1) * N], S[j])
    assert T.phase(keys, lwe) == int(ph[0])


@pytest.mark.parametrize("lutname", ["relu", "min", "eq9"])
def test_pbs_all_32_inputs(keys, lutname):
    if lutname == "relu":
        f = [(x - 4) % 32 for x in range(16)]
        _, rows = golden_lines("lut_relu.txt")
        want = {int(x): int(o) for x, o in rows}
        mod = 16
    elif lutname == "min":
        f = P.LUT_MIN_PRINTED
        _, rows = golden_lines("lut_min_printed.txt")
        want = {int(x): int(o) for x, o in rows}
        mod = 16
    else:
        f = P.LUT_EQ9
        want = {x: P.lookup(f, x) for x in range(32)}
        mod = 32
    cts = np.stack([T.encrypt(keys, x, 11, 3, x) for x in range(32)])
    outs = T.pbs_many(keys, cts, np.tile(np.array(f, dtype=np.uint32), (32, 1)))
    for x in range(32):
        assert T.decrypt(keys, outs[x]) % mod == want[x], x
    # the threaded and the single-call PBS are the same function
    assert np.array_equal(outs[5], T.pbs(keys, cts[5], f))


def test_pbs_pieces_compose(keys):
    ct = T.encrypt(keys, 9, 12, 0, 0)
    small = T.keyswitch(keys, ct)
    ms = T.modswitch(keys, small)
    acc = T.blind_rotate(keys, ms, T.lut_poly(keys, P.LUT_EQ9))
    assert np.array_equal(T.sample_extract(keys, acc), T.pbs(keys, ct, P.LUT_EQ9))


@pytest.mark.parametrize("alphabet,a,b", [
    (P.ALPHA_ASCII7, "k!d", "S|t"),
    (P.ALPHA_ASCII7, "abcx", "xabc"),
    (P.ALPHA_27, "AB C", "ABC"),
    (P.ALPHA_DNA4, "ACGTA", "AGTTC"),
])
def test_lvs_encrypted_matches_wf(keys, alphabet, a, b):
    xa = T.encrypt_string(keys, a, alphabet, 21, 0)
    yb = T.encrypt_string(keys, b, alphabet, 21, 1)
    res = T.lvs_encrypted(keys, xa, yb, alphabet, parallel=True)
    assert T.decrypt_distance(keys, res["h_row"], len(a)) == P.wf_distance(a, b)
    assert res["pbs"] == (P.eq_pbs_per_cell(alphabet) + 1) * len(a) * len(b)
    # every intermediate lookup decrypts to the plaintext oracle's value
    _, h, v, _ = P.lvs_plain(a, b, alphabet)
    for (i, j), M in res["M"].items():
        assert T.decrypt(keys, M) == (h[i][j] + v[i][j - 1]) % 32


def test_lvs_encrypted_paper_order_equals_diagonal_order(keys):
    a, b = "ab!", "b!a"
    xa = T.encrypt_string(keys, a, P.ALPHA_ASCII7, 5, 0)
    yb = T.encrypt_string(keys, b, P.ALPHA_ASCII7, 5, 1)
    r1 = T.lvs_encrypted(keys, xa, yb, P.ALPHA_ASCII7, parallel=False)
    r2 = T.lvs_encrypted(keys, xa, yb, P.ALPHA_ASCII7, parallel=True)
    for name in ("eq1", "eq9", "M"):
        for c in r1[name]:
            assert np.array_equal(r1[name][c], r2[name][c])
    assert T.decrypt_distance(keys, r1["h_row"], 3) == P.wf_distance(a, b)


def test_lvs_encrypted_band_exact_skip_and_approx(keys):
    """Algorithm alg_levenshtein's band on ciphertexts: the diagonal readout
    equals Wagner-Fischer with the exact-skip band floor(m/2) (Section 3.2),
    and the plaintext banded oracle with a narrow band; fewer PBS."""
    for a, b, band in [("abcd", "bcda", 2), ("kitten", "sittin", 3), ("aaaaa", "bbbaa", 1)]:
        xa = T.encrypt_string(keys, a, P.ALPHA_ASCII7, 31, 0)
        yb = T.encrypt_string(keys, b, P.ALPHA_ASCII7, 31, 1)
        res = T.lvs_encrypted(keys, xa, yb, P.ALPHA_ASCII7, parallel=True, band=band)
        m = len(a)
        E9 = [[0] * (m + 1) for _ in range(m + 1)]
        for i in range(1, m + 1):
            for j in range(1, m + 1):
                E9[i][j] = 9 if a[i - 1] == b[j - 1] else 0
        h, v = P.lvs_on_eq9(E9, m, m, band=band)
        want = P.readout_diagonal(h, v, m)
        assert T.decrypt_path(keys, res["diag"]) == want
        if band >= m // 2:
            assert want == P.wf_distance(a, b)
        assert res["pbs"] == 3 * P.band_cells(m, band)


def test_readout_sum_decrypts_to_distance(keys):
    """The return of Algorithm algo_complete taken on ciphertexts (one LWE
    sum, no bootstrap) decrypts to Wagner-Fischer, for the last-row readout
    (base m) and the band path (base 0)."""
    for a, b, band in [("kitten", "sitting", None), ("abcd", "ab", None), ("flaw", "lawn", 1), ("GATT", "ACA", 0)]:
        alpha = P.ALPHA_DNA4 if a.isupper() else P.ALPHA_ASCII7
        xa = T.encrypt_string(keys, a, alpha, 41, 0)
        yb = T.encrypt_string(keys, b, alpha, 41, 1)
        res = T.lvs_encrypted(keys, xa, yb, alpha, parallel=True, band=band)
        if band is None:
            got = T.decrypt(keys, T.readout_sum(keys, res["h_row"], len(a)))
            assert got == P.wf_distance(a, b) == T.decrypt_distance(keys, res["h_row"], len(a))
        else:
            got = T.decrypt(keys, T.readout_sum(keys, res["path"], 0))
            assert got == T.decrypt_path(keys, res["path"])
    # a planted off-by-one base is seen
    xa = T.encrypt_string(keys, "ab", P.ALPHA_ASCII7, 42, 0)
    yb = T.encrypt_string(keys, "ba", P.ALPHA_ASCII7, 42, 1)
    res = T.lvs_encrypted(keys, xa, yb, P.ALPHA_ASCII7, parallel=True)
    assert T.decrypt(keys, T.readout_sum(keys, res["h_row"], 3)) != P.wf_distance("ab", "ba")
