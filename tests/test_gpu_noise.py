"""Noise of the bootstrap on the GPU against the noise model of the chosen
parameter set (the basis of the failure-probability claim; the paper's own
accounting is Section 3.1.3 "Limiting the noise growth").

For a PBS output (sample extract of the blind-rotation accumulator) the phase
error is dominated by the gadget rounding of the external products: each CMux
with s_i = 1 adds the rounding error of X^a ACC - ACC, uniform on
[-2^(63-beta), 2^(63-beta)) per coefficient (beta = level * base_log),
weighted by (1 + |S|) for the body and the mask under the binary GLWE key S.
The bootstrapping-key noise adds n (k+1) l N E[d^2] var(TUniform(b_glwe)).
"""
import numpy as np
import pytest

from oracle import noise as Nz
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def predicted_pbs_variance(p, lwe_key, glwe_key):
    """The oracle's bootstrap-output variance model (oracle.noise.var_pbs,
    pinned against the oracle's own bootstraps) for the keys' actual
    weights; p is the library's parameter set, which must be the oracle's."""
    orc = T.params_lvs() if p.n == T.params_lvs().n else T.params_test()
    pd = orc.as_dict()
    for f in ("n", "k", "N", "pbs_level", "pbs_base_log", "glwe_noise_log2"):
        assert pd[f] == getattr(p, f), f
    return Nz.var_pbs(pd, float(np.sum(lwe_key)), float(np.sum(glwe_key)))


def test_pbs_output_noise_matches_model():
    p = L.lvs_params_default()
    ck, sk = L.lvs_keygen(p, 5)
    ctx = L.lvs_ctx_create(sk, 0)
    lwe_key, glwe_key = L.lvs_client_key_export(ck)
    big = p.k * p.N
    count = 2048
    rng = np.random.default_rng(1)
    msgs = rng.integers(0, 16, size=count)
    cts = np.stack([L.lvs_encrypt_lwe(ck, int(m), 8, 0, i, big) for i, m in enumerate(msgs)])
    ident = np.tile(np.arange(16, dtype=np.uint8), (count, 1))          # f(x) = x
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_out = torch.zeros_like(d_in)
    L.lvs_pbs_batch_device(ctx, d_in, big + 1, torch.from_numpy(ident).cuda(), d_out, big + 1, count)
    L.lvs_ctx_synchronize(ctx)
    out = d_out.cpu().numpy().view(np.uint64)
    mask = glwe_key.astype(bool)
    phase = out[:, big] - out[:, :big][:, mask].sum(axis=1, dtype=np.uint64)
    err = (phase - (msgs.astype(np.uint64) << np.uint64(59))).view(np.int64).astype(np.float64)
    measured = float(np.mean(err ** 2))
    predicted = predicted_pbs_variance(p, lwe_key, glwe_key)
    ratio = measured / predicted
    print("PBS noise: measured 2^%.3f predicted 2^%.3f ratio %.3f" % (np.log2(measured), np.log2(predicted), ratio))
    assert abs(float(np.mean(err))) < 4 * np.sqrt(measured / count)
    assert 0.85 < ratio < 1.15
    # every output decrypts (margin 2^58 = many standard deviations)
    assert np.max(np.abs(err)) < 2.0 ** 58


def test_failure_rate_of_increasingly_noisy_ciphertexts():
    """Section 3.1.3's experiment: bootstrap ciphertexts carrying more and
    more accumulated noise and count decoding errors.  An input
    m + c * Z (Z a fresh PBS output of 0, so the added variance is c^2 times
    that of a PBS output) is bootstrapped with the identity table; the error
    count must follow the failure probability of the noise model (normal
    tail of the key, key-switch and modulus-switch variances)."""
    from oracle import noise as Nz
    from oracle import tfhe as T

    p = L.lvs_params_default()
    pd = T.params_lvs().as_dict()
    ck, sk = L.lvs_keygen(p, 9)
    ctx = L.lvs_ctx_create(sk, 0)
    big = p.k * p.N
    count = 4096
    rng = np.random.default_rng(4)
    ident = torch.from_numpy(np.tile(np.arange(16, dtype=np.uint8), (count, 1))).cuda()

    def pbs(cts):
        d_in = torch.from_numpy(np.ascontiguousarray(cts).view(np.int64)).cuda()
        d_out = torch.zeros_like(d_in)
        L.lvs_pbs_batch_device(ctx, d_in, big + 1, ident, d_out, big + 1, cts.shape[0])
        L.lvs_ctx_synchronize(ctx)
        return d_out.cpu().numpy().view(np.uint64).copy()

    zeros = pbs(np.stack([L.lvs_encrypt_lwe(ck, 0, 10, 0, i, big) for i in range(count)]))
    msgs = rng.integers(0, 16, size=count)
    fresh = pbs(np.stack([L.lvs_encrypt_lwe(ck, int(m), 11, 0, i, big) for i, m in enumerate(msgs)]))
    rows = []
    for c in (1200, 1800, 2400, 3000):
        noisy = fresh + np.uint64(c) * zeros
        out = pbs(noisy)
        got = np.array([L.lvs_decrypt_lwe(ck, r) for r in out])
        errors = int(np.sum(got != msgs))
        pred = Nz.pfail_of(pd, 1 + c * c)
        expect = pred * count
        rows.append((c, errors, expect))
        print("c = %d: key variance %d PBS units, %d errors, predicted %.1f" % (c, 1 + c * c, errors, expect))
        # binomial agreement: 5 sigma plus 20 % model slack
        assert abs(errors - expect) <= 5 * np.sqrt(expect + 1) + 0.2 * expect
    # errors grow with the noise
    assert rows[-1][1] > rows[0][1]
    L.lvs_ctx_free(ctx)


def test_dp_noise_growth_matches_model():
    """Section 3.1.3 on real ciphertexts: the phase error of the last-row
    differences h[m][j] of long DNA pairs (full parameters) grows as the
    oracle's noise tracker predicts (h[m][j] carries 2j - 1 PBS-output
    variances for m >= j).  The errors, scaled by their predicted standard
    deviation, must have unit variance."""
    from oracle import noise as Nz
    from oracle import plain as P
    from paper_2508_14568_gb300 import workloads as W
    import random

    p = L.lvs_params_default()
    ck, sk = L.lvs_keygen(p, 13)
    ctx = L.lvs_ctx_create(sk, 0)
    lwe_key, glwe_key = L.lvs_client_key_export(ck)
    big = p.k * p.N
    rng = random.Random(17)
    m = 128
    pairs = []
    for _ in range(4):
        a = "".join(rng.choice(W.DNA) for _ in range(m))
        pairs.append((a, W.mutate_rate(rng, a, W.DNA, 0.10)[:m].ljust(m, "A")))
    A = [L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_DNA4, 21, 2 * k) for k, (a, b) in enumerate(pairs)]
    B = [L.lvs_encrypt_string(ck, b, L.LVS_ALPHA_DNA4, 21, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
    r = L.lvs_edit_distance_batch(ctx, A, B)
    var_pbs = predicted_pbs_variance(p, lwe_key, glwe_key)
    pred = Nz.output_variances(m, m)
    mask = glwe_key.astype(bool)
    z = []
    for k, (a, b) in enumerate(pairs):
        rows = L.lvs_result_export(r, k, big)
        _, h, _, _ = P.lvs_plain(a, b, P.ALPHA_DNA4)
        phase = rows[:, big] - rows[:, :big][:, mask].sum(axis=1, dtype=np.uint64)
        want = np.array([h[m][j] for j in range(1, m + 1)], dtype=np.uint64) << np.uint64(59)
        err = (phase - want).view(np.int64).astype(np.float64)
        sd = np.sqrt(np.array([pred[(m, j)][1] for j in range(1, m + 1)]) * var_pbs)
        z.append(err / sd)
    z = np.concatenate(z)
    ratio = float(np.mean(z ** 2))
    print("DP noise growth: %d samples, measured / predicted variance %.3f" % (z.size, ratio))
    assert 0.8 < ratio < 1.2
    L.lvs_ctx_free(ctx)
