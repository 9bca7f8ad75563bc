"""The wavefront plan the library launches (lvs_plan_pair, host only) run on
plaintext Z_32 values: every launch step is race-free (no row written twice,
no job reading a row that another job of the step writes in its epilogue, no
row read before it is written), the PBS count and the number of steps are those
of the method, and the planned lookups compute the distance: Wagner-Fischer for
the full matrix, refreshed anti-diagonals and exact bands, the plaintext banded
oracle otherwise (Algorithm algo_complete and Algorithm alg_levenshtein taken
as the GPU takes them, Section 6.2's anti-diagonal parallelism)."""
import random

import pytest

from oracle import plain as P
from paper_2508_14568_gb300 import lvs as L

LUTS = {0: P.LUT_EQ, 1: P.LUT_EQ9, 2: P.LUT_MIN, 3: P.LUT_V}
ALPHA = {P.ALPHA_ASCII7: 2, P.ALPHA_27: 2, P.ALPHA_DNA4: 1}


def simulate(a, b, alphabet, band=-1, refresh=None, preprocessed=False):
    """Runs the plan on plaintext values; returns (distance, layout, jobs)."""
    m, n = len(a), len(b)
    if preprocessed:
        subset = "".join(sorted(set(b)))
        lay, jobs = L.lvs_plan_pair(m, n, 0, band, refresh, b, subset or None)
    else:
        lay, jobs = L.lvs_plan_pair(m, n, ALPHA[alphabet], band, refresh)
    rows = [None] * lay["rows"]
    if preprocessed:
        for k, s in enumerate(subset):
            for i in range(m):
                rows[lay["table"] + k * m + i] = 9 if a[i] == s else 0
    else:
        C = ALPHA[alphabet]
        for base, st in ((lay["a"], a), (lay["b"], b)):
            for ci, c in enumerate(st):
                for si, v in enumerate(P.split_symbol(P.symbol_index(c, alphabet), alphabet)):
                    rows[base + ci * C + si] = v
    for r in range(lay["v"], lay["h"] + n):
        rows[r] = 1                                   # OneMatrix boundary
    if lay["path"] >= 0:
        for r in range(lay["path"], lay["path"] + m + n):
            rows[r] = 1
    _execute(rows, jobs, lay["steps"])
    if lay["path"] >= 0:
        dist = sum(P.signed(rows[lay["path"] + t]) for t in range(m + n))
    else:
        dist = m + sum(P.signed(rows[lay["h"] + t]) for t in range(n))
    return dist, lay, jobs


def _execute(rows, jobs, nsteps):
    """Runs planned launch steps on the plaintext rows (in place)."""
    steps = sorted({j["step"] for j in jobs})
    assert steps == list(range(len(steps)))
    assert len(steps) == nsteps
    for s in steps:
        step_jobs = [j for j in jobs if j["step"] == s]
        # key switch of the launch: every input is gathered before any output
        ins = []
        for j in step_jobs:
            x = j["cst"]
            for src, c in zip(j["src"], j["coef"]):
                if src >= 0:
                    assert rows[src] is not None, ("read before write", s, j)
                    x += c * rows[src]
            ins.append(x % 32)
        written = set()
        for j in step_jobs:
            for r in list(j["dst"]) + [j["tap"]]:
                if r >= 0:
                    assert r not in written, ("row written twice in a step", s, r)
                    written.add(r)
        # blind rotation + epilogue
        updates = []
        for j, x in zip(step_jobs, ins):
            out = P.lookup(LUTS[j["lut"]], x)
            if j["kind"] == 1:
                vi, hj = j["dst"]
                v_new, h_new = (out - rows[hj]) % 32, (out - rows[vi]) % 32
                updates += [(vi, v_new), (hj, h_new)]
                if j["tapsel"]:
                    updates.append((j["tap"], v_new if j["tapsel"] == 1 else h_new))
            else:
                assert j["dst"][1] < 0
                updates.append((j["dst"][0], out))
                if j["tapsel"]:
                    updates.append((j["tap"], out))
        for r, v in updates:
            rows[r] = v


def _e9(a, b):
    return [[9 if i and j and a[i - 1] == b[j - 1] else 0 for j in range(len(b) + 1)] for i in range(len(a) + 1)]


@pytest.mark.parametrize("alphabet,pool", [(P.ALPHA_ASCII7, "ab!~"), (P.ALPHA_27, "AB Z"), (P.ALPHA_DNA4, "ACGT")])
def test_full_matrix_plan_computes_wf(alphabet, pool):
    rng = random.Random(61)
    C = ALPHA[alphabet]
    for _ in range(60):
        a = "".join(rng.choice(pool) for _ in range(rng.randint(0, 9)))
        b = "".join(rng.choice(pool) for _ in range(rng.randint(0, 9)))
        d, lay, jobs = simulate(a, b, alphabet)
        assert d == P.wf_distance(a, b), (a, b)
        m, n = len(a), len(b)
        assert len(jobs) == (C + 1) * m * n                       # Table tab_pbs: (C + 1) PBS per cell
        assert lay["steps"] == (m + n - 1 + C if m and n else 0)  # anti-diagonals + the equality pipeline
        for j in jobs:
            if j["kind"] == 1:
                assert j["lut"] == 2


@pytest.mark.parametrize("alphabet", [P.ALPHA_ASCII7, P.ALPHA_DNA4])
def test_band_plan_computes_banded_oracle(alphabet):
    rng = random.Random(62)
    pool = "abcd" if alphabet == P.ALPHA_ASCII7 else "ACGT"
    C = ALPHA[alphabet]
    for _ in range(60):
        a = "".join(rng.choice(pool) for _ in range(rng.randint(1, 9)))
        b = "".join(rng.choice(pool) for _ in range(rng.randint(1, 9)))
        m, n = len(a), len(b)
        for band in (0, 1, 2, (min(m, n) + 1) // 2):
            d, lay, jobs = simulate(a, b, alphabet, band=band)
            h, v = P.lvs_on_eq9(_e9(a, b), m, n, band=band)
            assert d == P.readout_path(h, v, m, n), (a, b, band)
            assert len(jobs) == (C + 1) * P.band_cells_general(m, n, band)
            if band >= (min(m, n) + 1) // 2:
                assert d == P.wf_distance(a, b)


def test_refreshed_plan_computes_wf():
    """Refreshed anti-diagonals (Section 3.1.3) from the library's own plan at a
    small budget: two LUT_V lookups per refreshed cell, the distance unchanged."""
    rng = random.Random(63)
    for _ in range(30):
        a = "".join(rng.choice("abc") for _ in range(rng.randint(4, 11)))
        b = "".join(rng.choice("abc") for _ in range(rng.randint(4, 11)))
        m, n = len(a), len(b)
        diags, _ = L.lvs_noise_plan(m, n, -1, 60.0)
        refresh = [1 if d in diags else 0 for d in range(m + n + 1)]
        d, lay, jobs = simulate(a, b, P.ALPHA_ASCII7, refresh=refresh)
        assert d == P.wf_distance(a, b), (a, b, diags)
        extra = sum(1 for i in range(1, m + 1) for j in range(1, n + 1) if refresh[i + j])
        assert len(jobs) == 3 * m * n + extra
        assert sum(1 for j in jobs if j["lut"] == 3) == 2 * extra
        # with a band: the refreshed cells on the readout path feed it too
        band = 2
        diags, _ = L.lvs_noise_plan(m, n, band, 40.0)
        refresh = [1 if d in diags else 0 for d in range(m + n + 1)]
        d, lay, jobs = simulate(a, b, P.ALPHA_ASCII7, band=band, refresh=refresh)
        h, v = P.lvs_on_eq9(_e9(a, b), m, n, band=band)
        assert d == P.readout_path(h, v, m, n), (a, b, diags)


def test_preprocessed_plan_computes_wf():
    """Section 5's online phase: one cell lookup per cell reading the table row
    of the plaintext symbol, with and without a band."""
    rng = random.Random(64)
    for _ in range(60):
        a = "".join(rng.choice("ABCD ") for _ in range(rng.randint(1, 10)))
        b = "".join(rng.choice("ABC ") for _ in range(rng.randint(1, 10)))
        m, n = len(a), len(b)
        d, lay, jobs = simulate(a, b, P.ALPHA_27, preprocessed=True)
        assert d == P.wf_distance(a, b)
        assert len(jobs) == m * n and lay["steps"] == m + n - 1
        d, _, jobs = simulate(a, b, P.ALPHA_27, band=1, preprocessed=True)
        h, v = P.lvs_on_eq9(_e9(a, b), m, n, band=1)
        assert d == P.readout_path(h, v, m, n)


def test_plan_argument_errors():
    with pytest.raises(L.LvsError):
        L.lvs_plan_pair(3, 3, 3)
    with pytest.raises(L.LvsError):
        L.lvs_plan_pair(2, 2, 0, -1, None, "AB", "A")          # symbol outside the subset
    with pytest.raises(L.LvsError):
        L.lvs_plan_pair(2, 2, 0, -1, None, "AB", "ABA")        # repeated subset symbol


@pytest.mark.parametrize("alphabet,lib_alpha,symbols", [
    (P.ALPHA_ASCII7, L.LVS_ALPHA_ASCII7, "".join(chr(c) for c in range(128))),
    (P.ALPHA_27, L.LVS_ALPHA_27, "ABCDEFGHIJKLMNOPQRSTUVWXYZ "),
    (P.ALPHA_DNA4, L.LVS_ALPHA_DNA4, "ACGT")])
def test_table_plan_computes_eq9_table(alphabet, lib_alpha, symbols):
    """Section 5's table build as lvs_preprocess and the server plan it, run on
    plaintext values: T[sigma][i] = 9 EQ(a_i, sigma) for every symbol of the
    alphabet (Table tab_pre's table), 2 lookups per entry (1 for DNA)."""
    rng = random.Random(65)
    a = "".join(rng.choice(symbols) for _ in range(12)) + symbols[:3]
    m, C = len(a), ALPHA[alphabet]
    lay, jobs = L.lvs_plan_table(m, lib_alpha, symbols)
    assert len(jobs) == C * m * len(symbols) and lay["steps"] == C
    rows = [None] * lay["rows"]
    for ci, c in enumerate(a):
        for si, v in enumerate(P.split_symbol(P.symbol_index(c, alphabet), alphabet)):
            rows[lay["a"] + ci * C + si] = v
    _execute(rows, jobs, lay["steps"])
    want = P.preprocess_table(a, symbols, alphabet)
    for k, sym in enumerate(symbols):
        assert [rows[lay["table"] + k * m + i] for i in range(m)] == want[sym], sym
        assert want[sym] == [9 if x == sym else 0 for x in a]


def test_table_then_preprocessed_plan_computes_wf():
    """A plaintext-reference query as the server runs it: the table of the
    reference's symbols, then one cell lookup per cell reading it."""
    rng = random.Random(66)
    for _ in range(40):
        a = "".join(rng.choice("ABCD Z") for _ in range(rng.randint(1, 10)))
        b = "".join(rng.choice("ABZ ") for _ in range(rng.randint(1, 10)))
        subset = "".join(sorted(set(b)))
        m, n = len(a), len(b)
        tl, tjobs = L.lvs_plan_table(m, L.LVS_ALPHA_27, subset)
        trows = [None] * tl["rows"]
        for ci, c in enumerate(a):
            for si, v in enumerate(P.split_symbol(P.symbol_index(c, P.ALPHA_27), P.ALPHA_27)):
                trows[tl["a"] + ci * 2 + si] = v
        _execute(trows, tjobs, tl["steps"])
        lay, jobs = L.lvs_plan_pair(m, n, 0, -1, None, b, subset)
        rows = [None] * lay["rows"]
        rows[lay["table"]:lay["table"] + len(subset) * m] = trows[tl["table"]:tl["table"] + len(subset) * m]
        for r in range(lay["v"], lay["h"] + n):
            rows[r] = 1
        _execute(rows, jobs, lay["steps"])
        assert m + sum(P.signed(rows[lay["h"] + t]) for t in range(n)) == P.wf_distance(a, b)


def test_table_plan_argument_errors():
    with pytest.raises(L.LvsError):
        L.lvs_plan_table(3, L.LVS_ALPHA_27, "Ab")        # lowercase outside the alphabet
    with pytest.raises(L.LvsError):
        L.lvs_plan_table(3, L.LVS_ALPHA_DNA4, "ACA")     # repeated


# --------------------------------------------------------------- batch schedule

@pytest.mark.parametrize("eq_lookups,band", [(2, -1), (1, -1), (2, 3)])
def test_batch_schedule_keeps_each_pair_in_order_and_fills_waves(eq_lookups, band):
    """The batch call's launch schedule (lvs_plan_batch): every pair's steps
    run in increasing launches (one step of a pair per launch, so each step
    sees all of its own earlier steps done), the launch count is the longest
    pair's step count, every job is scheduled once, and holding pairs back
    never needs more waves of the grid than stepping all pairs together."""
    rng = random.Random(41 + eq_lookups + band)
    wave = 152
    for trial in range(4):
        sizes = [(rng.randint(1, 20), rng.randint(1, 20)) for _ in range(rng.randint(30, 120))]
        if band >= 0:
            sizes = [(a, a) for a, b in sizes]          # square pairs for the band
        counts = []
        for a, b in sizes:
            lay, jobs = L.lvs_plan_pair(a, b, eq_lookups, band)
            c = [0] * lay["steps"]
            for j in jobs:
                c[j["step"]] += 1
            counts.append(c)
        longest = max(len(c) for c in counts)
        waves = {}
        for w in (0, wave):
            launch_of, nl = L.lvs_plan_batch(sizes, eq_lookups, band, w)
            assert nl == longest
            per_launch = [0] * nl
            for c, lo in zip(counts, launch_of):
                assert len(lo) == len(c)
                assert all(0 <= t < nl for t in lo)
                assert all(x < y for x, y in zip(lo, lo[1:]))
                for s, t in enumerate(lo):
                    per_launch[t] += c[s]
            assert sum(per_launch) == sum(map(sum, counts))
            if w == 0:
                assert all(lo == list(range(len(lo))) for lo in launch_of)
            waves[w] = sum(-(-j // wave) for j in per_launch)
        assert waves[wave] <= waves[0]


def test_batch_schedule_argument_errors():
    with pytest.raises(L.LvsError):
        L.lvs_plan_batch([(3, 4)], 3)
