"""Server-side readout (lvs_result_sum): the return of Algorithm algo_complete
taken on ciphertexts, one LWE per pair encrypting the distance.  Bit-exact
with the oracle's sum of its own encrypted run, decrypts to Wagner-Fischer,
and refuses what does not fit the 5-bit plaintext."""
import numpy as np
import pytest

from oracle import plain as P
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALPHA = {P.ALPHA_ASCII7: L.LVS_ALPHA_ASCII7, P.ALPHA_DNA4: L.LVS_ALPHA_DNA4}


@pytest.fixture(scope="module")
def small():
    ck, sk = L.lvs_keygen(L.lvs_params_test(), 0)
    return ck, L.lvs_ctx_create(sk, 0), T.Keys(T.params_test(), 0)


@pytest.mark.parametrize("band", [None, 1])
def test_sum_bit_exact_with_oracle(small, band):
    ck, ctx, K = small
    pairs = [("kitten", "sitting", P.ALPHA_ASCII7), ("GATTACA", "GCATGCT", P.ALPHA_DNA4),
             ("a", "bcd", P.ALPHA_ASCII7)]
    seed = 51
    opts = L.lvs_opts_default(band=-1 if band is None else band)
    for k, (a, b, alpha) in enumerate(pairs):
        A = L.lvs_encrypt_string(ck, a, ALPHA[alpha], seed, 2 * k)
        B = L.lvs_encrypt_string(ck, b, ALPHA[alpha], seed, 2 * k + 1)
        r = L.lvs_edit_distance_batch(ctx, [A], [B], opts)
        launches0 = L.lvs_ctx_launch_count(ctx)
        pbs0 = L.lvs_ctx_pbs_count(ctx)
        s = L.lvs_result_sum(ctx, r)
        assert L.lvs_ctx_pbs_count(ctx) == pbs0          # no bootstrap
        assert L.lvs_ctx_launch_count(ctx) == launches0 + 1
        r.close()                                         # the sum does not need r any more
        got = L.lvs_result_export(s, 0, K.big_dim)
        assert got.shape == (1, K.big_dim + 1)
        xa = T.encrypt_string(K, a, alpha, seed, 2 * k)
        yb = T.encrypt_string(K, b, alpha, seed, 2 * k + 1)
        res = T.lvs_encrypted(K, xa, yb, alpha, parallel=True, band=band)
        want = T.readout_sum(K, res["h_row"], len(a)) if band is None else T.readout_sum(K, res["path"], 0)
        assert np.array_equal(got[0], want)
        d = L.lvs_decrypt(ck, s, 0)
        assert d == T.decrypt(K, want)
        if band is None:
            assert d == P.wf_distance(a, b)


def test_sum_of_a_batch_and_of_the_preprocessed_path(small):
    ck, ctx, _ = small
    import random
    rng = random.Random(52)
    pairs = [("".join(rng.choice("abc") for _ in range(rng.randint(1, 15))),
              "".join(rng.choice("abc") for _ in range(rng.randint(1, 15)))) for _ in range(40)]
    A = [L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_ASCII7, 53, 2 * k) for k, (a, b) in enumerate(pairs)]
    B = [L.lvs_encrypt_string(ck, b, L.LVS_ALPHA_ASCII7, 53, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
    want = [P.wf_distance(a, b) for a, b in pairs]
    s = L.lvs_result_sum(ctx, L.lvs_edit_distance_batch(ctx, A, B))
    assert L.lvs_result_info(s)["items"] == len(pairs)
    assert L.lvs_decrypt_all(ck, s) == want
    # band 8 >= ceil(min(m, n) / 2): exact, readout along the path
    s = L.lvs_result_sum(ctx, L.lvs_edit_distance_batch(ctx, A, B, L.lvs_opts_default(band=8)))
    assert L.lvs_decrypt_all(ck, s) == want
    tables = L.lvs_preprocess_batch(ctx, A, "abc")
    s = L.lvs_result_sum(ctx, L.lvs_edit_distance_preprocessed_batch(ctx, tables, [b for _, b in pairs]))
    assert L.lvs_decrypt_all(ck, s) == want


def test_sum_refuses_what_does_not_fit(small):
    ck, ctx, _ = small
    a = L.lvs_encrypt_string(ck, "a" * 16, L.LVS_ALPHA_ASCII7, 54, 0)
    b = L.lvs_encrypt_string(ck, "b", L.LVS_ALPHA_ASCII7, 54, 1)
    r = L.lvs_edit_distance_batch(ctx, [a], [b])
    with pytest.raises(L.LvsError):
        L.lvs_result_sum(ctx, r)
    e = L.lvs_eq(ctx, a, 0, b, 0)
    with pytest.raises(L.LvsError):
        L.lvs_result_sum(ctx, e)
    s = L.lvs_result_sum(ctx, L.lvs_edit_distance_batch(ctx, [], []))
    assert L.lvs_result_info(s)["items"] == 0
