"""Parity of the CUDA path with the oracle, through the C ABI (needs a GPU).

Bit-exact everywhere: every quantity on this path is an integer (torus values
mod 2^64, plaintexts in Z_32, distances).  Inputs come from the seeded
generators (paper_2508_14568_gb300.workloads, numpy seeds) and from the
oracle's own encryption; expected values come only from oracle/.
"""
import numpy as np
import pytest

from oracle import plain as P
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L
from paper_2508_14568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALPHA = {P.ALPHA_ASCII7: L.LVS_ALPHA_ASCII7, P.ALPHA_27: L.LVS_ALPHA_27, P.ALPHA_DNA4: L.LVS_ALPHA_DNA4}


def to_dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def from_dev(t, dtype=np.uint64):
    a = t.cpu().numpy()
    return a.view(dtype) if a.dtype.itemsize == np.dtype(dtype).itemsize else a.astype(dtype)


class Setup:
    def __init__(self, params_lib, params_orc, seed):
        self.ck, self.sk = L.lvs_keygen(params_lib, seed)
        self.K = T.Keys(params_orc, seed)
        self.ctx = L.lvs_ctx_create(self.sk, 0)
        self.p = params_orc
        self.big = params_orc.k * params_orc.N


@pytest.fixture(scope="module")
def small():
    return Setup(L.lvs_params_test(), T.params_test(), 0)


@pytest.fixture(scope="module")
def full():
    return Setup(L.lvs_params_default(), T.params_lvs(), 0)


# ----------------------------------------------------------------- products

def _poly_case(N, count, seed, extreme=False):
    rng = np.random.default_rng(seed)
    dig = rng.integers(-4096, 4096, size=(count, 4, N), dtype=np.int32)
    poly = rng.integers(0, 2**63, size=(count, 4, 2, N), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=(count, 4, 2, N), dtype=np.uint64)
    if extreme:
        dig[0] = -4096
        dig[1 % count] = 4095
        poly[0] = np.uint64(2**63)                 # most negative signed value
        poly[1 % count] = np.uint64(2**63 - 1)
    return dig, poly


def _poly_expected(dig, poly):
    count, _, N = dig.shape
    out = np.zeros((count, 2, N), np.uint64)
    for it in range(count):
        for c in range(2):
            acc = np.zeros(N, np.uint64)
            for r in range(4):
                acc = acc + T.negacyclic_mul(dig[it, r].astype(np.int64).view(np.uint64), poly[it, r, c])
            out[it, c] = acc
    return out


@pytest.mark.parametrize("which", ["small", "full"])
def test_negacyclic_products_bit_exact(which, request):
    S = request.getfixturevalue(which)
    N = S.p.N
    for seed, count, extreme in [(1, 3, True), (2, 5, False)]:
        dig, poly = _poly_case(N, count, seed, extreme)
        d_dig, d_poly = to_dev(dig), to_dev(poly)
        d_out = torch.zeros((count, 2, N), dtype=torch.int64, device="cuda")
        L.lvs_poly_mul_device(S.ctx, d_dig, d_poly, d_out, count)
        L.lvs_ctx_synchronize(S.ctx)
        got = from_dev(d_out)
        assert np.array_equal(got, _poly_expected(dig, poly))


# ----------------------------------------------------------------- key switch

@pytest.mark.parametrize("which,count", [("small", 37), ("full", 5)])
def test_keyswitch_bit_exact(which, count, request):
    S = request.getfixturevalue(which)
    cts = np.stack([T.encrypt(S.K, (3 * i) % 32, 5, 7, i) for i in range(count)])
    stride = S.big + 3          # a ragged row stride on purpose
    buf = np.zeros((count, stride), np.uint64)
    buf[:, : S.big + 1] = cts
    d_in = to_dev(buf)
    d_out = torch.zeros((count, S.p.n + 1), dtype=torch.int32, device="cuda")
    L.lvs_keyswitch_batch_device(S.ctx, d_in, stride, d_out, count)
    L.lvs_ctx_synchronize(S.ctx)
    got = from_dev(d_out, np.uint32)
    for i in range(count):
        want = T.modswitch(S.K, T.keyswitch(S.K, cts[i]))
        assert np.array_equal(got[i], want), i


# ----------------------------------------------------------------- PBS

def _pbs_gpu(S, cts, luts):
    count = cts.shape[0]
    d_in = to_dev(cts)
    d_lut = torch.from_numpy(np.ascontiguousarray(np.asarray(luts, np.uint8) % 32)).cuda()
    d_out = torch.zeros((count, S.big + 1), dtype=torch.int64, device="cuda")
    L.lvs_pbs_batch_device(S.ctx, d_in, S.big + 1, d_lut, d_out, S.big + 1, count)
    L.lvs_ctx_synchronize(S.ctx)
    return from_dev(d_out)


def test_pbs_bit_exact_small_many(small):
    """More jobs than resident CTAs (persistent loop) and every LUT of the method."""
    S = small
    count = 400
    rng = np.random.default_rng(4)
    msgs = rng.integers(0, 32, size=count)
    lut_pool = [P.LUT_EQ, P.LUT_EQ9, P.LUT_MIN, [(x - 4) % 32 for x in range(16)], list(rng.integers(0, 32, 16))]
    luts = [lut_pool[i % len(lut_pool)] for i in range(count)]
    cts = np.stack([T.encrypt(S.K, int(m), 6, 0, i) for i, m in enumerate(msgs)])
    got = _pbs_gpu(S, cts, luts)
    want = T.pbs_many(S.K, cts, np.asarray(luts, np.uint32))
    assert np.array_equal(got, want)
    for i in range(count):
        assert T.decrypt(S.K, got[i]) == P.lookup([int(v) for v in luts[i]], int(msgs[i]))


def test_pbs_bit_exact_full_params(full):
    S = full
    msgs = [0, 9, 17, 31, 4, 12, 8, 25]
    luts = [P.LUT_MIN, P.LUT_EQ9, P.LUT_EQ, P.LUT_MIN, P.LUT_MIN, P.LUT_EQ, [(x - 4) % 32 for x in range(16)], P.LUT_EQ9]
    cts = np.stack([T.encrypt(S.K, m, 8, 0, i) for i, m in enumerate(msgs)])
    got = _pbs_gpu(S, cts, luts)
    want = T.pbs_many(S.K, cts, np.asarray(luts, np.uint32))
    assert np.array_equal(got, want)
    for i, m in enumerate(msgs):
        assert T.decrypt(S.K, got[i]) == P.lookup(luts[i], m)


def test_pbs_one_cta_form_two_waves_full_params(full):
    """The blind-rotation form the throughput launches use (one CTA per
    ciphertext; the three-CTA form switched off) at the full parameters, on a
    launch of 160 PBS: more than one wave of the persistent grid (one CTA per
    SM), so jobs 152..159 are the second job of their CTA.  A sample of both
    waves, with every kind of lookup table, is compared element by element
    with the oracle's PBS of the same inputs."""
    S = full
    count = 160
    rng = np.random.default_rng(77)
    msgs = rng.integers(0, 32, size=count)
    kinds = [P.LUT_MIN, P.LUT_EQ9, P.LUT_EQ, P.LUT_V, [(x - 4) % 32 for x in range(16)]]
    luts = np.asarray([kinds[i % len(kinds)] for i in range(count)], np.uint32)
    cts = np.stack([T.encrypt(S.K, int(m), 9, 0, i) for i, m in enumerate(msgs)])
    split0 = L.lvs_ctx_br_split(S.ctx)
    L.lvs_ctx_set_br_split(S.ctx, 0)
    try:
        got = _pbs_gpu(S, cts, luts)
    finally:
        L.lvs_ctx_set_br_split(S.ctx, split0)
    sample = [0, 1, 75, 76, 150, 151] + list(range(152, 160))
    want = T.pbs_many(S.K, cts[sample], luts[sample])
    assert np.array_equal(got[sample], want)
    for i in range(count):
        assert T.decrypt(S.K, got[i]) == P.lookup(luts[i], int(msgs[i]))


# ----------------------------------------------------------------- edit distance

def _gpu_batch(S, pairs, alpha, seed=50, use_graph=True):
    A = [L.lvs_encrypt_string(S.ck, a, ALPHA[alpha], seed, 2 * k) for k, (a, b) in enumerate(pairs)]
    B = [L.lvs_encrypt_string(S.ck, b, ALPHA[alpha], seed, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
    r = L.lvs_edit_distance_batch(S.ctx, A, B, L.lvs_opts_default(use_graph))
    return r, L.lvs_decrypt_all(S.ck, r)


@pytest.mark.parametrize("alpha,pool", [(P.ALPHA_ASCII7, W.PRINTABLE), (P.ALPHA_27, W.ALPHA27), (P.ALPHA_DNA4, W.DNA)])
def test_edit_distance_batch_matches_wf_ragged(small, alpha, pool):
    pairs = W.random_pairs(17, 40, pool[:5], 0, 11) + [("", ""), (pool[0], ""), ("", pool[1] * 3), (pool[0], pool[0])]
    r, d = _gpu_batch(small, pairs, alpha)
    assert d == [P.wf_distance(a, b) for a, b in pairs]


def test_edit_distance_ciphertexts_bit_exact_vs_oracle(small):
    """The encrypted last row h[m][1..n] equals the oracle's Algorithm
    algo_complete run on the same ciphertexts, bit for bit."""
    S = small
    pairs = [("k!d", "S|t"), ("abcx", "xabc"), ("AB", "ABBA")]
    r, d = _gpu_batch(S, pairs, P.ALPHA_ASCII7, seed=51)
    for k, (a, b) in enumerate(pairs):
        xa = T.encrypt_string(S.K, a, P.ALPHA_ASCII7, 51, 2 * k)
        yb = T.encrypt_string(S.K, b, P.ALPHA_ASCII7, 51, 2 * k + 1)
        res = T.lvs_encrypted(S.K, xa, yb, P.ALPHA_ASCII7, parallel=True)
        got = L.lvs_result_export(r, k, S.big)
        assert np.array_equal(got, np.stack(res["h_row"]))
        assert d[k] == P.wf_distance(a, b) == T.decrypt_distance(S.K, res["h_row"], len(a))


def test_edit_distance_dna_ciphertexts_bit_exact(small):
    S = small
    pairs = [("GATTACA", "GCATGCT"), ("ACGT", "T")]
    r, d = _gpu_batch(S, pairs, P.ALPHA_DNA4, seed=52, use_graph=False)
    for k, (a, b) in enumerate(pairs):
        xa = T.encrypt_string(S.K, a, P.ALPHA_DNA4, 52, 2 * k)
        yb = T.encrypt_string(S.K, b, P.ALPHA_DNA4, 52, 2 * k + 1)
        res = T.lvs_encrypted(S.K, xa, yb, P.ALPHA_DNA4, parallel=True)
        assert np.array_equal(L.lvs_result_export(r, k, S.big), np.stack(res["h_row"]))
    assert d == [P.wf_distance(a, b) for a, b in pairs]


def test_pinned_host_strings_identical(small):
    S = small
    pairs = W.random_pairs(29, 6, W.PRINTABLE, 1, 9)
    A = [L.lvs_encrypt_string(S.ck, a, L.LVS_ALPHA_ASCII7, 54, 2 * k) for k, (a, b) in enumerate(pairs)]
    B = [L.lvs_encrypt_string(S.ck, b, L.LVS_ALPHA_ASCII7, 54, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
    r1 = L.lvs_edit_distance_batch(S.ctx, A, B)
    for s in A + B:
        L.lvs_ct_string_pin(s)
        L.lvs_ct_string_pin(s)       # no-op
    r2 = L.lvs_edit_distance_batch(S.ctx, A, B)
    for k in range(len(pairs)):
        assert np.array_equal(L.lvs_result_export(r1, k, S.big), L.lvs_result_export(r2, k, S.big))
    assert L.lvs_decrypt_all(S.ck, r2) == [P.wf_distance(a, b) for a, b in pairs]


def test_graph_and_direct_launches_identical(small):
    pairs = W.random_pairs(23, 12, W.PRINTABLE, 1, 9)
    r1, d1 = _gpu_batch(small, pairs, P.ALPHA_ASCII7, use_graph=True)
    r2, d2 = _gpu_batch(small, pairs, P.ALPHA_ASCII7, use_graph=False)
    assert d1 == d2 == [P.wf_distance(a, b) for a, b in pairs]
    for k in range(len(pairs)):
        assert np.array_equal(L.lvs_result_export(r1, k, small.big), L.lvs_result_export(r2, k, small.big))


def test_wave_fill_schedule_changes_no_ciphertext(small):
    """Holding pairs back to fill the waves of the blind-rotation grid moves
    steps between launches but never a result: every result row is bit-equal
    to the all-pairs-together schedule's, on a batch wide enough that pairs
    are held back, and the distances equal WF."""
    S = small
    pairs = W.random_pairs(29, 90, W.PRINTABLE, 4, 18)
    L.lvs_ctx_set_wave_fill(S.ctx, True)
    r1, d1 = _gpu_batch(S, pairs, P.ALPHA_ASCII7, seed=57)
    L.lvs_ctx_set_wave_fill(S.ctx, False)
    try:
        r2, d2 = _gpu_batch(S, pairs, P.ALPHA_ASCII7, seed=57)
    finally:
        L.lvs_ctx_set_wave_fill(S.ctx, True)
    assert d1 == d2 == [P.wf_distance(a, b) for a, b in pairs]
    for k in range(len(pairs)):
        assert np.array_equal(L.lvs_result_export(r1, k, S.big), L.lvs_result_export(r2, k, S.big))


def test_full_params_one_cell_chain_bit_exact(full):
    """Full parameter set, one ASCII pair of single characters: EQ1 -> EQ9 ->
    cell, every ciphertext of the chain bit-exact (the readout row)."""
    S = full
    pairs = [("q", "q")]
    r, d = _gpu_batch(S, pairs, P.ALPHA_ASCII7, seed=53)
    xa = T.encrypt_string(S.K, "q", P.ALPHA_ASCII7, 53, 0)
    yb = T.encrypt_string(S.K, "q", P.ALPHA_ASCII7, 53, 1)
    res = T.lvs_encrypted(S.K, xa, yb, P.ALPHA_ASCII7, parallel=True)
    assert np.array_equal(L.lvs_result_export(r, 0, S.big), np.stack(res["h_row"]))
    assert d == [0]


def test_config1_full_params_bit_exact(full):
    """Config 1 end to end at the full parameter set: the 48 PBS (16 EQ1, 16
    EQ9, 16 cells) feed one another, so the encrypted last row equal to the
    oracle's bit for bit means every PBS of the chain was; distance = WF."""
    S = full
    pairs = W.config1()
    r, d = _gpu_batch(S, pairs, P.ALPHA_ASCII7, seed=0)
    assert d == [P.wf_distance(a, b) for a, b in pairs]
    a, b = pairs[0]
    xa = T.encrypt_string(S.K, a, P.ALPHA_ASCII7, 0, 0)
    yb = T.encrypt_string(S.K, b, P.ALPHA_ASCII7, 0, 1)
    res = T.lvs_encrypted(S.K, xa, yb, P.ALPHA_ASCII7, parallel=True)
    assert res["pbs"] == 48
    assert np.array_equal(L.lvs_result_export(r, 0, S.big), np.stack(res["h_row"]))


# ----------------------------------------------------------------- equality and preprocessing

def test_lvs_eq_all_modes(small):
    S = small
    a = L.lvs_encrypt_string(S.ck, "Az~", L.LVS_ALPHA_ASCII7, 60, 0)
    b = L.lvs_encrypt_string(S.ck, "zA~", L.LVS_ALPHA_ASCII7, 60, 1)
    for i in range(3):
        for j in range(3):
            for t9 in (True, False):
                r = L.lvs_eq(S.ctx, a, i, b, j, t9)
                want = ("Az~"[i] == "zA~"[j]) * (9 if t9 else 1)
                assert L.lvs_decrypt(S.ck, r, 0) == want
    # bit-exact against Algorithm alg_ascii in the oracle
    xa = T.encrypt_string(S.K, "Az~", P.ALPHA_ASCII7, 60, 0)
    yb = T.encrypt_string(S.K, "zA~", P.ALPHA_ASCII7, 60, 1)
    one = T.trivial(S.K, 1)
    e1 = T.pbs(S.K, xa[2][0] - yb[2][0], P.LUT_EQ)
    e9 = T.pbs(S.K, T.scalar(2, xa[2][1] - yb[2][1]) + (one - e1), P.LUT_EQ9)
    r = L.lvs_eq(S.ctx, a, 2, b, 2, True)
    assert np.array_equal(L.lvs_result_export(r, 0, S.big)[0], e9)


def test_preprocessed_path(small):
    S = small
    qs = W.config3(queries=12)
    qs = [(a[:9], b[:9]) for a, b in qs] + [("A", "A"), ("AB", "")]
    tables, plains = [], []
    for k, (a, b) in enumerate(qs):
        enc = L.lvs_encrypt_string(S.ck, a, L.LVS_ALPHA_27, 70, k)
        tables.append(L.lvs_preprocess(S.ctx, enc))
        plains.append(b)
    r = L.lvs_edit_distance_preprocessed_batch(S.ctx, tables, plains)
    assert L.lvs_decrypt_all(S.ck, r) == [P.wf_distance(a, b) for a, b in qs]
    # table entries decrypt to 9 * [a_i == sigma] (Table tab_pre with EQ9)
    a = qs[0][0]
    enc = L.lvs_encrypt_string(S.ck, a, L.LVS_ALPHA_27, 71, 0)
    t = L.lvs_preprocess(S.ctx, enc, "AEZ ")
    r = L.lvs_edit_distance_preprocessed_batch(S.ctx, [t], ["ZEA "])
    assert L.lvs_decrypt_all(S.ck, r) == [P.wf_distance(a, "ZEA ")]
    with pytest.raises(L.LvsError):
        L.lvs_edit_distance_preprocessed_batch(S.ctx, [t], ["B"])   # not in the subset


def test_preprocess_table_bit_exact(small):
    S = small
    a = "GATC"
    enc = L.lvs_encrypt_string(S.ck, a, L.LVS_ALPHA_DNA4, 72, 0)
    xa = T.encrypt_string(S.K, a, P.ALPHA_DNA4, 72, 0)
    t = L.lvs_preprocess(S.ctx, enc, "CG")
    r = L.lvs_edit_distance_preprocessed_batch(S.ctx, [t], ["CG"])
    # oracle: EQ9[i][j] = PBS(x_i - sigma; LUT_EQ9), then Algorithm alg_levenshtein
    one = T.trivial(S.K, 1)
    m, n = len(a), 2
    v = {(i, 0): one for i in range(m + 1)}
    h = {(0, j): one for j in range(n + 1)}
    for j in range(1, n + 1):
        sig = P.symbol_index("CG"[j - 1], P.ALPHA_DNA4)
        for i in range(1, m + 1):
            e9 = T.pbs(S.K, T.add_const(xa[i - 1][0], -sig), P.LUT_EQ9)
            key = (one - v[(i, j - 1)]) + T.scalar(3, one + h[(i - 1, j)]) + e9
            M = T.pbs(S.K, key, P.LUT_MIN)
            v[(i, j)] = M - h[(i - 1, j)]
            h[(i, j)] = M - v[(i, j - 1)]
    assert np.array_equal(L.lvs_result_export(r, 0, S.big), np.stack([h[(m, j)] for j in range(1, n + 1)]))


def test_preprocess_batch_equals_single_tables(small):
    """Section 5 offline phase for many strings at once (one set of launches):
    the online results from batched tables equal those from per-string tables
    bit for bit, for ASCII / 27-symbol (two lookups) and DNA (one lookup)."""
    S = small
    for alpha, abc, pool in [(L.LVS_ALPHA_27, "AB EZ", W.ALPHA27[:6]), (L.LVS_ALPHA_DNA4, None, W.DNA)]:
        rng = np.random.default_rng(5)
        strs = ["".join(pool[x] for x in rng.integers(0, len(pool), size=int(rng.integers(1, 8)))) for _ in range(5)]
        plains = ["".join(pool[x] for x in rng.integers(0, len(pool), size=int(rng.integers(1, 8)))) for _ in range(5)]
        if abc is not None:
            plains = ["".join(c for c in p if c in abc) or abc[0] for p in plains]
        encs = [L.lvs_encrypt_string(S.ck, a, alpha, 73, k) for k, a in enumerate(strs)]
        single = [L.lvs_preprocess(S.ctx, e, abc) for e in encs]
        batch = L.lvs_preprocess_batch(S.ctx, encs, abc)
        r1 = L.lvs_edit_distance_preprocessed_batch(S.ctx, single, plains)
        r2 = L.lvs_edit_distance_preprocessed_batch(S.ctx, batch, plains)
        for k in range(len(strs)):
            assert np.array_equal(L.lvs_result_export(r1, k, S.big), L.lvs_result_export(r2, k, S.big))
        assert L.lvs_decrypt_all(S.ck, r2) == [P.wf_distance(a, b) for a, b in zip(strs, plains)]


def test_config2_full_size_distances(full):
    """Config 2 at full size in the launch configuration of the benchmark
    (256 pairs, union launches, CUDA graph): every distance equals Wagner-Fischer."""
    pairs = W.config2()
    r, d = _gpu_batch(full, pairs, P.ALPHA_ASCII7, seed=0)
    assert d == [P.wf_distance(a, b) for a, b in pairs]


def test_long_pairs_deep_wavefront(small):
    """Long strings: thousands of anti-diagonal steps, wide launches and large
    arenas (test parameters keep it fast); every distance equals WF."""
    S = small
    import random
    rng = random.Random(77)
    a = "".join(rng.choice(W.DNA) for _ in range(700))
    pairs = [(a, W.mutate_rate(rng, a, W.DNA, 0.2)), (a[:300], a[:650]), ("A" * 500, "C" * 20)]
    r, d = _gpu_batch(S, pairs, P.ALPHA_DNA4, seed=78)
    assert d == [P.wf_distance(x, y) for x, y in pairs]
