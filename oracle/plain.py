"""Plaintext oracle for the Leuvenshtein method -- TEST INFRASTRUCTURE ONLY.

Everything here is plain Python on small integers.  Each function names the
passage of the paper it restates.  Values that live in the TFHE plaintext space
are kept in Z_32 (one padding bit + 4 message bits, Section 2.2), and every
lookup applies the negacyclic rule f(x + 16) = -f(x) (Section 2.2, Table
table_lutrelu; Section 3.1.2).
"""
from collections import deque

PLAIN_MOD = 32          # 5-bit plaintext space (padding bit + 4 bits), Section 2.2
HALF = 16               # a lookup table holds 16 free values


# ---------------------------------------------------------------------------
# Wagner-Fischer and the definition of the edit distance
# ---------------------------------------------------------------------------

def wf_matrix(a, b):
    """The d-matrix of Eq. eq_wf: D[i][j] = ed(a[:i], b[:j]).

    D[i][0] = i, D[0][j] = j; D[i][j] = D[i-1][j-1] if a_i = b_j, otherwise
    1 + min(D[i-1][j], D[i][j-1], D[i-1][j-1]).
    """
    m, n = len(a), len(b)
    D = [[0] * (n + 1) for _ in range(m + 1)]
    for i in range(m + 1):
        D[i][0] = i
    for j in range(n + 1):
        D[0][j] = j
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            if a[i - 1] == b[j - 1]:
                D[i][j] = D[i - 1][j - 1]
            else:
                D[i][j] = 1 + min(D[i - 1][j], D[i][j - 1], D[i - 1][j - 1])
    return D


def wf_distance(a, b):
    """Levenshtein distance by Wagner-Fischer (Eq. eq_wf)."""
    return wf_matrix(a, b)[len(a)][len(b)]


def edit_distance_bfs(a, b, alphabet=None):
    """Edit distance straight from its definition (Section 2.3): the least
    number of single-character insertions, deletions and substitutions that
    turn ``a`` into ``b``, found by breadth-first search over strings.

    Only for tiny inputs.  Strings are tuples of symbols.  The search alphabet
    defaults to the symbols of both strings (inserting any other symbol can
    never shorten a path to ``b``).
    """
    a, b = tuple(a), tuple(b)
    if alphabet is None:
        alphabet = sorted(set(a) | set(b))
    if a == b:
        return 0
    seen = {a}
    frontier = deque([(a, 0)])
    while frontier:
        s, d = frontier.popleft()
        nxt = set()
        for p in range(len(s) + 1):
            for c in alphabet:
                nxt.add(s[:p] + (c,) + s[p:])              # insertion
        for p in range(len(s)):
            nxt.add(s[:p] + s[p + 1:])                      # deletion
            for c in alphabet:
                if c != s[p]:
                    nxt.add(s[:p] + (c,) + s[p + 1:])       # substitution
        for t in nxt:
            if t == b:
                return d + 1
            if t not in seen and len(t) <= max(len(a), len(b)) + 1:
                seen.add(t)
                frontier.append((t, d + 1))
    raise AssertionError("unreachable")


def hamming(a, b):
    """Hamming distance of two equal-length strings (Section 2.3)."""
    assert len(a) == len(b)
    return sum(x != y for x, y in zip(a, b))


# ---------------------------------------------------------------------------
# Myers differences and the Leuvenshtein cell
# ---------------------------------------------------------------------------

def deltas_from_matrix(D):
    """Eq. eq:delta: dv[i][j] = D[i][j] - D[i-1][j], dh[i][j] = D[i][j] - D[i][j-1]."""
    m, n = len(D) - 1, len(D[0]) - 1
    dv = [[None] * (n + 1) for _ in range(m + 1)]
    dh = [[None] * (n + 1) for _ in range(m + 1)]
    for i in range(m + 1):
        for j in range(n + 1):
            if i >= 1:
                dv[i][j] = D[i][j] - D[i - 1][j]
            if j >= 1:
                dh[i][j] = D[i][j] - D[i][j - 1]
    return dv, dh


def myers_cell(dv_in, dh_in, eq):
    """The cell equations of Section 2.3.3 (Myers):
    dv_out = min(1, dv_in + 1 - dh_in, 1 - eq - dh_in),
    dh_out = min(1, 1 + dh_in - dv_in, 1 - eq - dv_in)."""
    dv_out = min(1, dv_in + 1 - dh_in, 1 - eq - dh_in)
    dh_out = min(1, 1 + dh_in - dv_in, 1 - eq - dv_in)
    return dv_out, dh_out


def lvs_M(dv_in, dh_in, eq):
    """The shared non-linear part of Eq. mye_eq_2: M = 1 + min(-eq, dv_in, dh_in)."""
    return 1 + min(-eq, dv_in, dh_in)


def lvs_cell(dv_in, dh_in, eq):
    """Section 3.1.1: dv_out = M - dh_in, dh_out = M - dv_in."""
    M = lvs_M(dv_in, dh_in, eq)
    return M - dh_in, M - dv_in


def key_eq(dv_in, dh_in, eq):
    """Eq. eq_keyeq: (dv_in + 1) + 3 (1 + dh_in) + 9 eq  -- the printed Table LUTmin key."""
    return (dv_in + 1) + 3 * (1 + dh_in) + 9 * eq


def key_eq2(dv_in, dh_in, eq):
    """Eq. eq_keyeq2 (the noise-reduced key used by both algorithms):
    (1 - dv_in) + 3 (1 + dh_in) + 9 eq."""
    return (1 - dv_in) + 3 * (1 + dh_in) + 9 * eq


def lut_from_key(keyfn):
    """The 16-entry LUT of 'M as a function of the key' (Section 3.1.2).

    Enumerates the 18 (dv_in, dh_in, eq) inputs.  Keys 16 and 17 fall in the
    negacyclic half, so the table only works if M is 0 there and at keys 0, 1
    (f(x + 16) = -f(x)); that is asserted, not assumed.  Unused keys are 0.
    """
    f = [None] * 18
    for eq in (0, 1):
        for dh in (-1, 0, 1):
            for dv in (-1, 0, 1):
                x = keyfn(dv, dh, eq)
                M = lvs_M(dv, dh, eq)
                assert 0 <= x < 18
                assert f[x] in (None, M), "key is not injective on M"
                f[x] = M
    f = [0 if v is None else v for v in f]
    assert f[16] == 0 and f[17] == 0 and f[0] == 0 and f[1] == 0
    return f[:16]


def key_eq2_swapped(dv_in, dh_in, eq):
    """Eq. eq_keyeq2 with the roles of dv_in and dh_in exchanged:
    (1 - dh_in) + 3 (1 + dv_in) + 9 eq."""
    return key_eq2(dh_in, dv_in, eq)


def lut_out_from_key(keyfn, outfn):
    """The 16-entry LUT of an output outfn(dv_in, dh_in, eq) (in Z_32) as a
    function of the key keyfn.  Keys 16 and 17 fall in the negacyclic half:
    the table is only valid if out(16 + x) = -out(x) mod 32 there, which is
    asserted.  Unused keys are 0."""
    f = [None] * 18
    for eq in (0, 1):
        for dh in (-1, 0, 1):
            for dv in (-1, 0, 1):
                x = keyfn(dv, dh, eq)
                o = outfn(dv, dh, eq) % PLAIN_MOD
                assert 0 <= x < 18
                assert f[x] in (None, o), "key is not injective on the output"
                f[x] = o
    for x in (16, 17):
        if f[x] is not None:
            assert f[x - 16] is not None and (f[x] + f[x - 16]) % PLAIN_MOD == 0, "not negacyclic"
    f = [0 if v is None else v for v in f]
    return f[:16]


def lvs_refresh_v(dv_in, dh_in, eq):
    """dv_out of Section 3.1.1 as one function of the cell inputs: M - dh_in."""
    return lvs_M(dv_in, dh_in, eq) - dh_in


LUT_MIN_PRINTED = None   # filled below: Table LUTmin (key of Eq. eq_keyeq)
LUT_MIN = None           # key of Eq. eq_keyeq2, used by Algorithms alg_levenshtein / algo_complete
LUT_EQ = [1] + [0] * 15  # Eq. eq_eqlut
LUT_EQ9 = [9] + [0] * 15  # Eq. eq_eqlut9
LUT_MIN_PRINTED = lut_from_key(key_eq)
LUT_MIN = lut_from_key(key_eq2)
# Refreshed cell (Section 3.1.3, refresh of dv and dh by a bootstrap): dv_out
# straight from the key, and dh_out = M - dv_in from the swapped key through the
# same table (M is symmetric in dv_in and dh_in).
LUT_V = lut_out_from_key(key_eq2, lvs_refresh_v)


def lookup(lut16, x):
    """Negacyclic 16-entry lookup on x in Z_32 (Section 2.2):
    f(x) for x < 16, -f(x - 16) mod 32 otherwise."""
    x %= PLAIN_MOD
    if x < HALF:
        return lut16[x] % PLAIN_MOD
    return (-lut16[x - HALF]) % PLAIN_MOD


def signed(x):
    """Z_32 residue -> signed integer in [-16, 16)."""
    x %= PLAIN_MOD
    return x - PLAIN_MOD if x >= HALF else x


# ---------------------------------------------------------------------------
# Symbol encodings and equality
# ---------------------------------------------------------------------------

ALPHA_ASCII7 = "ascii7"
ALPHA_27 = "alpha27"
ALPHA_DNA4 = "dna4"

DNA_SYMBOLS = "ACGT"


def symbol_index(c, alphabet):
    """Character -> symbol index.  ASCII: the byte (7 bits).  27-symbol:
    'A'..'Z' -> 0..25, ' ' -> 26.  DNA: A, C, G, T -> 0..3."""
    if isinstance(c, str):
        c = ord(c)
    if alphabet == ALPHA_ASCII7:
        assert 0 <= c < 128
        return c
    if alphabet == ALPHA_27:
        if c == ord(' '):
            return 26
        assert ord('A') <= c <= ord('Z')
        return c - ord('A')
    if alphabet == ALPHA_DNA4:
        return DNA_SYMBOLS.index(chr(c))
    raise ValueError(alphabet)


def split_symbol(idx, alphabet):
    """Section 4.3: a 7-bit character is kept as a 4-bit symbol x1 and a 3-bit
    symbol x2; we take x1 = low 4 bits, x2 = the rest (the 27-symbol alphabet
    uses the same split, x2 in {0, 1}).  DNA symbols stay whole (one symbol)."""
    if alphabet == ALPHA_DNA4:
        return (idx,)
    return (idx & 15, idx >> 4)


def eq_two_lookup(x, y, times9=True):
    """Algorithm alg_ascii in Z_32: z0 = x1 - y1; eq1 = LUT_EQ(z0);
    z1 = 2 (x2 - y2) + (1 - eq1); result = LUT_EQ9(z1) (or LUT_EQ(z1))."""
    z0 = (x[0] - y[0]) % PLAIN_MOD
    eq1 = lookup(LUT_EQ, z0)
    z1 = (2 * (x[1] - y[1]) + (1 - eq1)) % PLAIN_MOD
    return lookup(LUT_EQ9 if times9 else LUT_EQ, z1)


def eq_one_lookup(x, y, times9=True):
    """Section 4.1 (4-bit subtraction equality, used for DNA with one lookup):
    LUT_EQ9(x - y) (or LUT_EQ)."""
    return lookup(LUT_EQ9 if times9 else LUT_EQ, (x[0] - y[0]) % PLAIN_MOD)


def eq9(x, y, alphabet):
    if alphabet == ALPHA_DNA4:
        return eq_one_lookup(x, y)
    return eq_two_lookup(x, y)


def eq_pbs_per_cell(alphabet):
    """Equality lookups per cell: 2 (Algorithm alg_ascii), 1 for DNA (Section 6.3)."""
    return 1 if alphabet == ALPHA_DNA4 else 2


# ---------------------------------------------------------------------------
# Leuvenshtein in plaintext (Algorithm algo_complete, Algorithm alg_levenshtein)
# ---------------------------------------------------------------------------

def lvs_plain(a, b, alphabet=ALPHA_ASCII7):
    """Algorithm algo_complete evaluated on plaintext Z_32 values.

    h, v start as all-ones (OneMatrix); v[i][0] = 1, h[0][j] = 1.  For
    j = 1..n, i = 1..m: eq9 from the equality lookups, key by Eq. eq_keyeq2,
    M = LUT_min(key), v[i][j] = M - h[i-1][j], h[i][j] = M - v[i][j-1].
    Returns (distance, h, v, lookups).  The distance is read out as
    m + sum_{j=1..n} h[m][j] (the printed readout starts the sum at j = 0,
    which counts the boundary h[m][0] = 1 once too often).
    """
    xs = [split_symbol(symbol_index(c, alphabet), alphabet) for c in a]
    ys = [split_symbol(symbol_index(c, alphabet), alphabet) for c in b]
    m, n = len(xs), len(ys)
    h = [[1] * (n + 1) for _ in range(m + 1)]
    v = [[1] * (n + 1) for _ in range(m + 1)]
    lookups = 0
    for j in range(1, n + 1):
        for i in range(1, m + 1):
            e9 = eq9(xs[i - 1], ys[j - 1], alphabet)
            lookups += eq_pbs_per_cell(alphabet)
            key = ((1 - v[i][j - 1]) + 3 * (1 + h[i - 1][j]) + e9) % PLAIN_MOD
            M = lookup(LUT_MIN, key)
            lookups += 1
            v[i][j] = (M - h[i - 1][j]) % PLAIN_MOD
            h[i][j] = (M - v[i][j - 1]) % PLAIN_MOD
    dist = m + sum(signed(h[m][j]) for j in range(1, n + 1))
    return dist, h, v, lookups


def in_band(i, j, m, n, band):
    """The band of Section 3.2 (Algorithm alg_levenshtein: |i - j| <= band for
    m = n), widened for m != n to the diagonals k = j - i with
    min(0, n - m) - band <= k <= max(0, n - m) + band: the cells with
    |k| + |(n - m) - k| <= |n - m| + 2 band, where every edit path of cost at
    most |n - m| + 2 band lies (a path through diagonal k costs at least |k| to
    get there and |n - m - k| to get back).  band None: every cell."""
    if band is None:
        return True
    k, delta = j - i, n - m
    return min(0, delta) - band <= k <= max(0, delta) + band


def lvs_on_eq9(E9, m, n, band=None):
    """Algorithm alg_levenshtein on a given EQ9 matrix (E9[i][j] in {0, 9},
    1-based), with optional band (in_band).  Out-of-band cells keep the
    OneMatrix value 1.  Returns (h, v) in Z_32."""
    h = [[1] * (n + 1) for _ in range(m + 1)]
    v = [[1] * (n + 1) for _ in range(m + 1)]
    for j in range(1, n + 1):
        for i in range(1, m + 1):
            if not in_band(i, j, m, n, band):
                continue
            key = ((1 - v[i][j - 1]) + 3 * (1 + h[i - 1][j]) + E9[i][j]) % PLAIN_MOD
            M = lookup(LUT_MIN, key)
            v[i][j] = (M - h[i - 1][j]) % PLAIN_MOD
            h[i][j] = (M - v[i][j - 1]) % PLAIN_MOD
    return h, v


def readout_row(h, m, n):
    """D[m][n] = D[m][0] + sum_j dh[m][j] = m + sum_{j=1..n} h[m][j]."""
    return m + sum(signed(h[m][j]) for j in range(1, n + 1))


def readout_diagonal(h, v, m):
    """Square band readout (Section 3.2): D[m][m] = sum_{i=1..m} (v[i][i-1] + h[i][i])."""
    return sum(signed(v[i][i - 1]) + signed(h[i][i]) for i in range(1, m + 1))


def readout_path_cells(m, n):
    """The monotone path of the band readout from (0, 0) to (m, n): down the
    main diagonal (v[i][i-1], then h[i][i]) for i <= min(m, n), then along row
    m (h[m][j], j > m) or down column n (v[i][n], i > n).  For band >= 1
    every step is a boundary value or a cell inside the band (band 0 leaves
    the v[i][i-1] at their OneMatrix value).  Returns [(i, j, 'v' | 'h')]:
    D[m][n] is the sum."""
    r = min(m, n)
    path = []
    for i in range(1, r + 1):
        path += [(i, i - 1, "v"), (i, i, "h")]
    if n > m:
        path += [(m, j, "h") for j in range(m + 1, n + 1)]
    else:
        path += [(i, n, "v") for i in range(n + 1, m + 1)]
    return path


def readout_path(h, v, m, n):
    """D[m][n] as the sum of the differences along readout_path_cells."""
    return sum(signed((v if s == "v" else h)[i][j]) for i, j, s in readout_path_cells(m, n))


# ---------------------------------------------------------------------------
# Preprocessing (Section 5, Table tab_pre) and PBS counts (Table tab_pbs)
# ---------------------------------------------------------------------------

def preprocess_table(enc_string, subset, alphabet, times9=True):
    """Section 5: T[sigma][i] = EQ(a_i, sigma) for every sigma of the subset,
    computed by the same lookups as the online equality (plaintext here)."""
    xs = [split_symbol(symbol_index(c, alphabet), alphabet) for c in enc_string]
    table = {}
    for s in subset:
        ys = split_symbol(symbol_index(s, alphabet), alphabet)
        if alphabet == ALPHA_DNA4:
            table[s] = [eq_one_lookup(x, ys, times9) for x in xs]
        else:
            table[s] = [eq_two_lookup(x, ys, times9) for x in xs]
    return table


def lvs_preprocessed_plain(table, plain_b, m):
    """Online phase of Section 5: EQ9[i][j] = T[b_j][i], then Algorithm
    alg_levenshtein with no band.  Returns the distance (row readout)."""
    n = len(plain_b)
    E9 = [[0] * (n + 1) for _ in range(m + 1)]
    for j in range(1, n + 1):
        col = table[plain_b[j - 1]]
        for i in range(1, m + 1):
            E9[i][j] = col[i - 1]
    h, v = lvs_on_eq9(E9, m, n)
    return readout_row(h, m, n)


def pbs_count_exact(m, n, eq_per_cell=2):
    """Table tab_pbs, Leuvenshtein Exact: (eq lookups + 1) per cell."""
    return (eq_per_cell + 1) * m * n


def band_cells_general(m, n, band):
    """Cells of an m x n matrix inside in_band."""
    return sum(1 for i in range(1, m + 1) for j in range(1, n + 1) if in_band(i, j, m, n, band))


def band_cells(m, band):
    """Cells with |i - j| <= band in an m x m matrix (Section 3.2 count:
    m (2 l + 1) - l^2 - l)."""
    return sum(1 for i in range(1, m + 1) for j in range(1, m + 1) if abs(i - j) <= band)

