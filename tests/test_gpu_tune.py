"""Key-switch launch plans (jobs per CTA, split of the input coefficients
over CTAs) and their autotuner: every plan is bit-exact with the oracle's key
switch + modulus switch (Section 2.2), and autotuning changes no result."""
import numpy as np
import pytest

from oracle import plain as P
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def full():
    ck, sk = L.lvs_keygen(L.lvs_params_default(), 0)
    return ck, L.lvs_ctx_create(sk, 0), T.Keys(T.params_lvs(), 0)


PLANS = [(4, 1), (4, 8), (16, 1), (16, 2), (16, 32), (16, 3)]


@pytest.mark.parametrize("count", [1, 3, 17, 70])
def test_every_plan_bit_exact(full, count):
    ck, ctx, K = full
    p = K.params
    big = K.big_dim
    cts = np.stack([T.encrypt(K, (5 * i) % 32, 12, 3, i) for i in range(count)])
    want = np.stack([T.modswitch(K, T.keyswitch(K, c)) for c in cts])
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    for tj, split in PLANS:
        L.lvs_ctx_set_ks_plan(ctx, count, tj, split)
        assert L.lvs_ctx_ks_plan(ctx, count) == (tj, split)
        d_out = torch.zeros((count, p.n + 1), dtype=torch.int32, device="cuda")
        L.lvs_keyswitch_batch_device(ctx, d_in, big + 1, d_out, count)
        L.lvs_ctx_synchronize(ctx)
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), (tj, split)
    L.lvs_ctx_set_ks_plan(ctx, count, 0, 1)   # back to the default


def test_set_plan_rejects_bad_shapes(full):
    _, ctx, _ = full
    for tj, split in [(8, 1), (16, 0), (16, 33), (-4, 1)]:
        with pytest.raises(L.LvsError):
            L.lvs_ctx_set_ks_plan(ctx, 10, tj, split)


def test_autotune_keeps_results(full):
    ck, ctx, K = full
    big = K.big_dim
    msgs = [0, 9, 17, 31, 4, 12]
    luts = np.asarray([P.LUT_MIN, P.LUT_EQ9, P.LUT_EQ, P.LUT_MIN, P.LUT_V, P.LUT_EQ], np.uint8)
    cts = np.stack([T.encrypt(K, m, 8, 1, i) for i, m in enumerate(msgs)])
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(luts).cuda()

    def run():
        d_out = torch.zeros_like(d_in)
        L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, d_out, big + 1, len(msgs))
        L.lvs_ctx_synchronize(ctx)
        return d_out.cpu().numpy().view(np.uint64).copy()

    before = run()
    L.lvs_ctx_autotune(ctx)
    plans = [L.lvs_ctx_ks_plan(ctx, n) for n in (1, 10, 50, 200, 800, 5000)]
    assert all(tj in (4, 16) and 1 <= s <= 32 for tj, s in plans)
    after = run()
    assert np.array_equal(before, after)
    assert np.array_equal(after, T.pbs_many(K, cts, luts.astype(np.uint32)))


def test_int_mul_probe_plausible():
    """The measured multiply issue rates that set the blind rotation's
    roofline: positive, at most 128 per SM per clock (4 sub-partitions x 32
    lanes), and the high half no faster than the low half."""
    lo, hi = L.lvs_probe_int_mul(0)
    assert 8 <= lo <= 128 and 4 <= hi <= 128
    assert hi <= lo * 1.05


def test_modmul_probe_below_the_multiply_issue_rates():
    """The achievable rates of the NTT's arithmetic: a Shoup product needs two
    low-half and one high-half multiply, so its stream cannot beat the issue
    rates of lvs_probe_int_mul (5% slack for timing), and a complete lazy
    butterfly (a product plus three additions) is no faster than a product."""
    lo, hi = L.lvs_probe_int_mul(0)
    shoup, bfly = L.lvs_probe_modmul(0)
    bound = 1.0 / (2.0 / lo + 1.0 / hi)
    assert 1.0 <= bfly <= shoup * 1.05
    assert shoup <= bound * 1.05


def test_key_product_probe_plausible():
    """The key product's ceilings: 64-bit multiply-accumulates no faster than
    the high-half multiply issue rate (both are double-width products on the
    multiply pipe, 10% slack for timing), and L2 -> SM bytes per SM per clock
    positive and below what 384 threads with 32 bytes each could move per clock
    if every load returned at once (12 KB)."""
    lo, hi = L.lvs_probe_int_mul(0)
    wide, l2 = L.lvs_probe_key_product(0)
    assert 1.0 <= wide <= hi * 1.1
    assert 1.0 <= l2 <= 384 * 32


@pytest.mark.parametrize("which", ["test", "default"])
def test_three_cta_blind_rotation_bit_exact(which):
    """The blind rotation split over a cluster of three CTAs (one per NTT
    prime) gives the same ciphertexts as one CTA per ciphertext and as the
    oracle, for PBS launches and for the edit-distance pipeline (cell
    epilogue, band taps)."""
    params, oparams = (L.lvs_params_test(), T.params_test()) if which == "test" else \
        (L.lvs_params_default(), T.params_lvs())
    ck, sk = L.lvs_keygen(params, 4)
    ctx = L.lvs_ctx_create(sk, 0)
    K = T.Keys(oparams, 4)
    big = K.big_dim
    count = 40 if which == "test" else 9
    rng = np.random.default_rng(11)
    msgs = rng.integers(0, 32, size=count)
    luts = rng.integers(0, 32, size=(count, 16), dtype=np.uint8)
    cts = np.stack([T.encrypt(K, int(m), 13, 2, i) for i, m in enumerate(msgs)])
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(luts).cuda()
    outs = []
    for split in (0, 10 ** 6):
        L.lvs_ctx_set_br_split(ctx, split)
        assert L.lvs_ctx_br_split(ctx) == split
        d_out = torch.zeros_like(d_in)
        L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, d_out, big + 1, count)
        L.lvs_ctx_synchronize(ctx)
        outs.append(d_out.cpu().numpy().view(np.uint64).copy())
    assert np.array_equal(outs[0], outs[1])
    if which == "test":
        assert np.array_equal(outs[1], T.pbs_many(K, cts, luts.astype(np.uint32)))
        # the pipeline: cell epilogue and band taps through the three-CTA form
        pairs = [("kitten", "sittin"), ("abc", "abd")]
        A = [L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_ASCII7, 14, 2 * k) for k, (a, b) in enumerate(pairs)]
        B = [L.lvs_encrypt_string(ck, b, L.LVS_ALPHA_ASCII7, 14, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
        for band in (-1, 2):
            res = []
            for split in (0, 10 ** 6):
                L.lvs_ctx_set_br_split(ctx, split)
                r = L.lvs_edit_distance_batch(ctx, A, B, L.lvs_opts_default(band=band))
                res.append([L.lvs_result_export(r, k, big) for k in range(len(pairs))])
                assert L.lvs_decrypt_all(ck, r) == [P.wf_distance(a, b) for a, b in pairs]
            for x, y in zip(*res):
                assert np.array_equal(x, y)
    L.lvs_ctx_free(ctx)


def test_autotune_sets_blind_rotation_split(full):
    ck, ctx, K = full
    L.lvs_ctx_autotune(ctx)
    assert 0 <= L.lvs_ctx_br_split(ctx) <= 152


@pytest.mark.parametrize("which", ["test", "default"])
def test_tensor_core_keyswitch_bit_exact(which):
    """The key switch as bf16 GEMMs over the key's bytes (exact integer partial
    sums) equals the oracle's key switch + modulus switch bit for bit, alone and
    inside the edit-distance pipeline."""
    params, oparams = (L.lvs_params_test(), T.params_test()) if which == "test" else \
        (L.lvs_params_default(), T.params_lvs())
    ck, sk = L.lvs_keygen(params, 6)
    ctx = L.lvs_ctx_create(sk, 0)
    K = T.Keys(oparams, 6)
    p = K.params
    big = K.big_dim
    L.lvs_ctx_set_ks_gemm_min(ctx, 1)
    assert L.lvs_ctx_ks_gemm_min(ctx) == 1

    def ks(d_in, count, gemm_min):
        L.lvs_ctx_set_ks_gemm_min(ctx, gemm_min)
        d_out = torch.zeros((count, p.n + 1), dtype=torch.int32, device="cuda")
        L.lvs_keyswitch_batch_device(ctx, d_in, big + 1, d_out, count)
        L.lvs_ctx_synchronize(ctx)
        return d_out.cpu().numpy().view(np.uint32)

    # 1, 17, 300 (ragged tiles): every output against the oracle;
    # 4096 and 8300 (the second crosses the 8192-job pass of the digit
    # scratch): every output against the kernel path (bit-exact with the oracle
    # for every plan), and a sample against the oracle
    for count in (1, 17, 300, 4096, 8300):
        cts = np.stack([T.encrypt(K, (7 * i) % 32, 15, 4, i) for i in range(count)])
        d_in = torch.from_numpy(cts.view(np.int64)).cuda()
        got = ks(d_in, count, 1)
        sample = range(count) if count <= 300 else sorted(set(range(0, count, count // 61)) | {count - 1})
        want = np.stack([T.modswitch(K, T.keyswitch(K, cts[i])) for i in sample])
        assert np.array_equal(got[list(sample)], want), count
        if count > 300:
            assert np.array_equal(got, ks(d_in, count, 0)), count
    if which == "test":
        pairs = [("kitten", "sitting"), ("abc", "abd"), ("flaw", "lawn")]
        A = [L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_ASCII7, 16, 2 * k) for k, (a, b) in enumerate(pairs)]
        B = [L.lvs_encrypt_string(ck, b, L.LVS_ALPHA_ASCII7, 16, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
        res = []
        for m in (0, 1):
            L.lvs_ctx_set_ks_gemm_min(ctx, m)
            r = L.lvs_edit_distance_batch(ctx, A, B)
            res.append([L.lvs_result_export(r, k, big) for k in range(len(pairs))])
            assert L.lvs_decrypt_all(ck, r) == [P.wf_distance(a, b) for a, b in pairs]
        for x, y in zip(*res):
            assert np.array_equal(x, y)
    L.lvs_ctx_free(ctx)


def test_autotune_sets_keyswitch_gemm_threshold(full):
    ck, ctx, K = full
    L.lvs_ctx_autotune(ctx)
    assert L.lvs_ctx_ks_gemm_min(ctx) in (0, 256, 1024, 4096)


@pytest.mark.parametrize("which", ["test", "default"])
def test_key_staged_blind_rotation_bit_exact(which):
    """The key-staged blind rotation (the head of each bootstrapping-key row
    copied into shared memory by bulk copies during the previous CMux) gives
    the same ciphertexts as the default form, over several jobs per CTA (the
    staging runs across job boundaries), and the oracle's: every output at the
    test parameters, a sample of both waves at the full parameters."""
    params, oparams = (L.lvs_params_test(), T.params_test()) if which == "test" else \
        (L.lvs_params_default(), T.params_lvs())
    ck, sk = L.lvs_keygen(params, 8)
    ctx = L.lvs_ctx_create(sk, 0)
    K = T.Keys(oparams, 8)
    big = K.big_dim
    count = 700 if which == "test" else 170
    rng = np.random.default_rng(19)
    msgs = rng.integers(0, 32, size=count)
    luts = rng.integers(0, 32, size=(count, 16), dtype=np.uint8)
    cts = np.stack([T.encrypt(K, int(m), 17, 2, i) for i, m in enumerate(msgs)])
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(luts).cuda()
    L.lvs_ctx_set_br_split(ctx, 0)
    outs = []
    for staged in (False, True, False):
        L.lvs_ctx_set_key_staging(ctx, staged)
        assert L.lvs_ctx_key_staging(ctx) == staged
        d_out = torch.zeros_like(d_in)
        L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, d_out, big + 1, count)
        L.lvs_ctx_synchronize(ctx)
        outs.append(d_out.cpu().numpy().view(np.uint64).copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    sample = list(range(count)) if which == "test" else [0, 1, 151, 152, 169]
    want = T.pbs_many(K, cts[sample], luts[sample].astype(np.uint32))
    assert np.array_equal(outs[1][sample], want)
    L.lvs_ctx_free(ctx)


def test_key_staging_wait_runs_out_reports_timeout_and_recovers():
    """A staging copy that is never issued (test hook): the bounded wait for it
    gives up after about a second, the launch ends normally with its results
    void, the next synchronize returns LVS_ERR_TIMEOUT, and the same context
    then computes bit-exact results again."""
    params = L.lvs_params_test()
    ck, sk = L.lvs_keygen(params, 9)
    ctx = L.lvs_ctx_create(sk, 0)
    K = T.Keys(T.params_test(), 9)
    big = K.big_dim
    count = 200
    msgs = np.arange(count) % 32
    luts = np.tile(np.arange(16, dtype=np.uint8), (count, 1))
    cts = np.stack([T.encrypt(K, int(m), 23, 0, i) for i, m in enumerate(msgs)])
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(luts).cuda()
    L.lvs_ctx_set_br_split(ctx, 0)
    ref = torch.zeros_like(d_in)
    L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, ref, big + 1, count)
    L.lvs_ctx_synchronize(ctx)
    L.lvs_ctx_set_key_staging(ctx, True)
    L.lvs_debug_drop_key_copy(ctx, True)
    d_out = torch.zeros_like(d_in)
    L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, d_out, big + 1, count)
    with pytest.raises(L.LvsError) as e:
        L.lvs_ctx_synchronize(ctx)
    assert e.value.status == L.LVS_ERR_TIMEOUT
    L.lvs_debug_drop_key_copy(ctx, False)
    L.lvs_ctx_synchronize(ctx)   # the give-up was reported once
    d_out.zero_()
    L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, d_out, big + 1, count)
    L.lvs_ctx_synchronize(ctx)
    assert np.array_equal(d_out.cpu().numpy(), ref.cpu().numpy())
    L.lvs_ctx_free(ctx)
