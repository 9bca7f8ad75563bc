"""Pins for the plaintext oracle (oracle/plain.py) -- no GPU.

Each check ties the oracle to something other than itself: the worked examples
printed in the paper (tests/golden/), brute force over the definition of the
edit distance, closed forms and exhaustive enumeration.
"""
import itertools
import random

import pytest

from oracle import plain as P
from tests.conftest import golden_lines


def _matrix(rows):
    return [[int(x) for x in r] for r in rows]


# ---------------------------------------------------------------- Wagner-Fischer

@pytest.mark.parametrize("name", ["dmatrix_monday_friday.txt", "dmatrix_abcx_xabc.txt"])
def test_wf_matrix_matches_fig_dmatrix(name):
    meta, rows = golden_lines(name)
    assert P.wf_matrix(meta["a"], meta["b"]) == _matrix(rows)


def test_fig_myers_matrix_and_arrows():
    meta, rows = golden_lines("myers_kid_sit.txt")
    D = [[int(x) for x in r[1:]] for r in rows if r[0] == "D"]
    assert P.wf_matrix(meta["a"], meta["b"]) == D
    dv, dh = P.deltas_from_matrix(D)
    for r in rows:
        if r[0] == "dh":
            i = int(r[1])
            assert [dh[i][j] for j in range(1, 4)] == [int(x) for x in r[2:]]
        if r[0] == "dv":
            j = int(r[1])
            assert [dv[i][j] for i in range(1, 4)] == [int(x) for x in r[2:]]


def test_lvs_plain_reproduces_fig_myers_arrows():
    meta, rows = golden_lines("myers_kid_sit.txt")
    dist, h, v, _ = P.lvs_plain(meta["a"], meta["b"])
    assert dist == 2
    for r in rows:
        if r[0] == "dh" and int(r[1]) >= 1:
            i = int(r[1])
            assert [P.signed(h[i][j]) for j in range(1, 4)] == [int(x) for x in r[2:]]
        if r[0] == "dv" and int(r[1]) >= 1:
            j = int(r[1])
            assert [P.signed(v[i][j]) for i in range(1, 4)] == [int(x) for x in r[2:]]


def test_counts_fixture():
    _, rows = golden_lines("counts.txt")
    for r in rows:
        if r[0] == "hamming":
            assert P.hamming(r[1], r[2]) == int(r[3])
        elif r[0] == "edit":
            assert P.wf_distance(r[1], r[2]) == int(r[3])
            assert P.edit_distance_bfs(r[1], r[2]) == int(r[3])
        elif r[0] == "band":
            m, l, cells = int(r[1]), int(r[2]), int(r[3])
            assert P.band_cells(m, l) == cells == m * (2 * l + 1) - l * l - l
        elif r[0] == "pbs_exact":
            m, n, total = int(r[1]), int(r[2]), int(r[3])
            assert P.pbs_count_exact(m, n) == total


def test_wf_equals_bfs_definition_exhaustive_small():
    alpha = "abc"
    strs = [""] + ["".join(t) for L in range(1, 4) for t in itertools.product(alpha, repeat=L)]
    for a in strs:
        for b in strs:
            assert P.wf_distance(a, b) == P.edit_distance_bfs(a, b), (a, b)


def test_wf_closed_forms_and_metric_axioms():
    rng = random.Random(5)
    alpha = "abcd"
    for _ in range(300):
        a = "".join(rng.choice(alpha) for _ in range(rng.randint(0, 9)))
        b = "".join(rng.choice(alpha) for _ in range(rng.randint(0, 9)))
        c = "".join(rng.choice(alpha) for _ in range(rng.randint(0, 9)))
        dab = P.wf_distance(a, b)
        assert P.wf_distance(a, a) == 0
        assert P.wf_distance(a, "") == len(a) and P.wf_distance("", b) == len(b)
        assert dab == P.wf_distance(b, a)
        assert dab <= P.wf_distance(a, c) + P.wf_distance(c, b)
        assert abs(len(a) - len(b)) <= dab <= max(len(a), len(b))
        if len(a) == len(b):
            assert dab <= P.hamming(a, b)


# ---------------------------------------------------------------- the cell

def test_myers_cell_from_wf_recurrence():
    """All 18 inputs: the Myers min-equations equal the differences produced by
    Eq. eq_wf on a 2x2 block with those incoming differences."""
    for dv in (-1, 0, 1):
        for dh in (-1, 0, 1):
            for eq in (0, 1):
                c = 10
                up, left = c + dh, c + dv          # D[i-1][j], D[i][j-1]
                d = c if eq else 1 + min(up, left, c)
                assert P.myers_cell(dv, dh, eq) == (d - up, d - left)
                assert P.lvs_cell(dv, dh, eq) == (d - up, d - left)


def test_lut_min_printed_table():
    _, rows = golden_lines("lut_min_printed.txt")
    for x, out in rows:
        assert P.lookup(P.LUT_MIN_PRINTED, int(x)) % 16 == int(out)


def test_lut_min_key2_against_cell_truth_table():
    for dv in (-1, 0, 1):
        for dh in (-1, 0, 1):
            for eq in (0, 1):
                x = P.key_eq2(dv, dh, eq)
                assert P.lookup(P.LUT_MIN, x) == P.lvs_M(dv, dh, eq)
                x1 = P.key_eq(dv, dh, eq)
                assert P.lookup(P.LUT_MIN_PRINTED, x1) == P.lvs_M(dv, dh, eq)
    assert P.LUT_MIN == [0, 0, 0, 1, 1, 0, 1, 1, 0] + [0] * 7


def test_lut_relu_table_semantics():
    _, rows = golden_lines("lut_relu.txt")
    f = [(x - 4) % 32 for x in range(16)]
    for x, out in rows:
        assert P.lookup(f, int(x)) % 16 == int(out)


# ---------------------------------------------------------------- equality

def test_equality_ascii_exhaustive():
    for x in range(128):
        for y in range(128):
            e = P.eq_two_lookup(P.split_symbol(x, P.ALPHA_ASCII7), P.split_symbol(y, P.ALPHA_ASCII7))
            assert e == (9 if x == y else 0)


def test_equality_alpha27_and_dna_exhaustive():
    for x in range(27):
        for y in range(27):
            e = P.eq_two_lookup(P.split_symbol(x, P.ALPHA_27), P.split_symbol(y, P.ALPHA_27))
            assert e == (9 if x == y else 0)
    for x in range(4):
        for y in range(4):
            assert P.eq_one_lookup((x,), (y,)) == (9 if x == y else 0)


def test_preprocess_abbey_table():
    meta, rows = golden_lines("preprocess_abbey.txt")
    word = meta["word"]
    # the table stores EQ (not EQ9) in the printed example; lowercase letters
    xs = [(ord(c) & 15, ord(c) >> 4) for c in word]
    for r in rows:
        sig = r[0]
        ys = (ord(sig) & 15, ord(sig) >> 4)
        got = [P.eq_two_lookup(x, ys, times9=False) for x in xs]
        assert got == [int(v) for v in r[1:]]
    t = P.preprocess_table(word.upper(), "ABCDEY", P.ALPHA_27, times9=False)
    for r in rows:
        assert t[r[0].upper()] == [int(v) for v in r[1:]]


# ---------------------------------------------------------------- Leuvenshtein

def test_lvs_plain_equals_wf_exhaustive_small():
    alpha = "ab c"
    strs = ["".join(t) for L in range(1, 4) for t in itertools.product(alpha, repeat=L)]
    for a in strs:
        for b in strs:
            d, _, _, lookups = P.lvs_plain(a, b)
            assert d == P.wf_distance(a, b), (a, b)
            assert lookups == 3 * len(a) * len(b)


def test_lvs_plain_random_alphabets():
    rng = random.Random(11)
    for alphabet, pool in [(P.ALPHA_ASCII7, [chr(c) for c in range(0x20, 0x7F)]),
                           (P.ALPHA_27, list("ABCDEFGHIJKLMNOPQRSTUVWXYZ ")),
                           (P.ALPHA_DNA4, list("ACGT"))]:
        for _ in range(150):
            a = "".join(rng.choice(pool[:6] if rng.random() < 0.5 else pool) for _ in range(rng.randint(1, 14)))
            b = "".join(rng.choice(pool[:6] if rng.random() < 0.5 else pool) for _ in range(rng.randint(1, 14)))
            d, _, _, lookups = P.lvs_plain(a, b, alphabet)
            assert d == P.wf_distance(a, b)
            assert lookups == (P.eq_pbs_per_cell(alphabet) + 1) * len(a) * len(b)


def test_lvs_printed_key_would_be_wrong_with_key2_table():
    """Sensitivity: the Eq. eq_keyeq2 key with the printed (Eq. eq_keyeq) table
    must break the distance somewhere -- the pins above can tell them apart."""
    bad = 0
    for a, b in [("KID", "SIT"), ("abcx", "xabc"), ("monday", "friday")]:
        saved = P.LUT_MIN
        try:
            P.LUT_MIN = P.LUT_MIN_PRINTED
            d = P.lvs_plain(a, b)[0]
        finally:
            P.LUT_MIN = saved
        bad += d != P.wf_distance(a, b)
    assert bad > 0


def test_readout_paper_printed_is_off_by_one():
    """The printed readout of Algorithm algo_complete sums h[m][0..n]; h[m][0]
    is the OneMatrix boundary 1, so that sum is D + 1 (the oracle uses j >= 1)."""
    for a, b in [("KID", "SIT"), ("abcx", "xabc"), ("monday", "friday")]:
        d, h, _, _ = P.lvs_plain(a, b)
        m, n = len(a), len(b)
        printed = m + sum(P.signed(h[m][j]) for j in range(0, n + 1))
        assert printed == d + 1 == P.wf_distance(a, b) + 1


def test_band_and_diagonal_readout_square():
    """Section 3.2: with m = n, cells with |i - j| <= floor(m/2) suffice and the
    diagonal readout gives the exact distance."""
    rng = random.Random(3)
    for _ in range(200):
        m = rng.randint(1, 9)
        a = "".join(rng.choice("abc") for _ in range(m))
        b = "".join(rng.choice("abc") for _ in range(m))
        E9 = [[0] * (m + 1) for _ in range(m + 1)]
        for i in range(1, m + 1):
            for j in range(1, m + 1):
                E9[i][j] = 9 if a[i - 1] == b[j - 1] else 0
        h, v = P.lvs_on_eq9(E9, m, m, band=m // 2)
        assert P.readout_diagonal(h, v, m) == P.wf_distance(a, b)
        hf, vf = P.lvs_on_eq9(E9, m, m)
        assert P.readout_row(hf, m, m) == P.wf_distance(a, b)


def test_preprocessed_plain_equals_wf():
    rng = random.Random(9)
    pool = "ABCDEFGHIJKLMNOPQRSTUVWXYZ "
    for _ in range(100):
        a = "".join(rng.choice(pool) for _ in range(rng.randint(1, 12)))
        b = "".join(rng.choice(pool) for _ in range(rng.randint(1, 12)))
        t = P.preprocess_table(a, pool, P.ALPHA_27)
        assert P.lvs_preprocessed_plain(t, b, len(a)) == P.wf_distance(a, b)
    # DNA: the one-lookup table of Section 6.3
    for _ in range(100):
        a = "".join(rng.choice("ACGT") for _ in range(rng.randint(1, 12)))
        b = "".join(rng.choice("ACGT") for _ in range(rng.randint(1, 12)))
        t = P.preprocess_table(a, "ACGT", P.ALPHA_DNA4)
        assert all(x in (0, 9) for col in t.values() for x in col)
        assert P.lvs_preprocessed_plain(t, b, len(a)) == P.wf_distance(a, b)


def _e9(a, b):
    m, n = len(a), len(b)
    return [[9 if i and j and a[i - 1] == b[j - 1] else 0 for j in range(n + 1)] for i in range(m + 1)]


def test_general_band_reduces_to_square_band():
    for m in range(1, 9):
        for band in range(0, m + 1):
            for i in range(1, m + 1):
                for j in range(1, m + 1):
                    assert P.in_band(i, j, m, m, band) == (abs(i - j) <= band)
    assert P.band_cells_general(7, 7, 2) == P.band_cells(7, 2)


def test_readout_path_is_monotone_inside_bands_from_1():
    for m in range(0, 7):
        for n in range(0, 7):
            path = P.readout_path_cells(m, n)
            assert len(path) == m + n
            pos = (0, 0)
            for i, j, s in path:
                # one step down (v) or right (h)
                assert (i, j) == ((pos[0] + 1, pos[1]) if s == "v" else (pos[0], pos[1] + 1))
                pos = (i, j)
                assert j == 0 or P.in_band(i, j, m, n, 1)
            assert pos == (m, n)


def test_non_square_band_exact_and_upper_bound():
    """Ukkonen's argument: an edit path through diagonal k = j - i costs at
    least |k| + |(n - m) - k|, so with band >= ceil(min(m, n) / 2) every
    optimal path lies in the band and the readout is exact; narrower bands
    are exact whenever D <= |n - m| + 2 band and never below D."""
    rng = random.Random(11)
    for _ in range(1500):
        m, n = rng.randint(1, 9), rng.randint(1, 9)
        a = "".join(rng.choice("abc") for _ in range(m))
        b = "".join(rng.choice("abc") for _ in range(n))
        wf = P.wf_distance(a, b)
        E9 = _e9(a, b)
        h, v = P.lvs_on_eq9(E9, m, n, (min(m, n) + 1) // 2)
        assert P.readout_path(h, v, m, n) == wf
        band = rng.randint(0, max(m, n))
        h, v = P.lvs_on_eq9(E9, m, n, band)
        d = P.readout_path(h, v, m, n)
        assert d >= wf
        if wf <= abs(n - m) + 2 * band:
            assert d == wf


def test_table_tab_pbs_band_rows():
    """Table tab_pbs: Exact Skipping ~ 2.25 m n and Approx. l = 10 ~ 60 n
    follow from the band count of Section 3.2 with 3 PBS per cell (the printed
    approximations drop the corner terms; l = m/4 is ~ 6 l n minus 3 l^2)."""
    m = 256
    skip = 3 * P.band_cells(m, m // 2)
    assert abs(skip / (m * m) - 2.25) < 0.01
    approx10 = 3 * P.band_cells(m, 10)
    assert abs(approx10 / (60 * m) - 1) < 0.05
    l = m // 4
    approx_q = 3 * P.band_cells(m, l)
    assert approx_q == 6 * l * m + 3 * m - 3 * l * l - 3 * l
    assert abs(approx_q / (6 * l * m) - 1) < 0.15


def test_general_band_cell_count_by_path_cost():
    """band_cells_general counts the cells through which an edit path costs at
    most |n - m| + 2 band (|k| to reach diagonal k = j - i, |n - m - k| to get
    back), the characterisation of the widened band; every cell once the band
    covers the longer string."""
    for m in range(1, 9):
        for n in range(1, 9):
            for band in range(0, 5):
                want = sum(1 for i in range(1, m + 1) for j in range(1, n + 1)
                           if abs(j - i) + abs((n - m) - (j - i)) <= abs(n - m) + 2 * band)
                assert P.band_cells_general(m, n, band) == want, (m, n, band)
            assert P.band_cells_general(m, n, max(m, n)) == m * n
