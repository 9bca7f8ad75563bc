"""FP64-FFT blind rotation (the double-precision polynomial products of the
TFHE-rs bootstrap the paper measures on) against the exact NTT path and the
noise model of the PBS (Section 2.2; noise accounting Section 3.1.3).

The FFT path is not bit-exact: it must decrypt to the same messages, keep
the phase close to the exact NTT output's, and add no measurable noise to the
bootstrap (output variance within 1.2x of the predicted one).
"""
import numpy as np
import pytest

from paper_2508_14568_gb300 import lvs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from tests.test_gpu_noise import predicted_pbs_variance  # noqa: E402


def _run(ctx, fn, cts, luts, big):
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_out = torch.zeros_like(d_in)
    fn(ctx, d_in, big + 1, torch.from_numpy(luts).cuda(), d_out, big + 1, cts.shape[0])
    L.lvs_ctx_synchronize(ctx)
    return d_out.cpu().numpy().view(np.uint64)


def _phase_err(out, glwe_key, expect, big):
    mask = glwe_key.astype(bool)
    phase = out[:, big] - out[:, :big][:, mask].sum(axis=1, dtype=np.uint64)
    return (phase - (expect.astype(np.uint64) << np.uint64(59))).view(np.int64).astype(np.float64)


@pytest.mark.parametrize("params", ["test", "default"])
def test_fft_pbs_decrypts_and_tracks_ntt(params):
    p = L.lvs_params_test() if params == "test" else L.lvs_params_default()
    ck, sk = L.lvs_keygen(p, 21)
    ctx = L.lvs_ctx_create(sk, 0)
    L.lvs_ctx_prepare_fft64(ctx, sk)
    L.lvs_ctx_prepare_fft64(ctx, sk)            # second call is a no-op
    lwe_key, glwe_key = L.lvs_client_key_export(ck)
    big = p.k * p.N
    count = 600 if params == "test" else 300
    rng = np.random.default_rng(7)
    msgs = rng.integers(0, 32, size=count)
    luts = rng.integers(0, 32, size=(count, 16), dtype=np.uint8)
    cts = np.stack([L.lvs_encrypt_lwe(ck, int(m), 31, 1, i, big) for i, m in enumerate(msgs)])
    ntt = _run(ctx, L.lvs_pbs_batch_device, cts, luts, big)
    fft = _run(ctx, L.lvs_pbs_batch_device_fft64, cts, luts, big)
    # the LUT is negacyclic: inputs 16..31 give -f(x - 16) mod 32
    expect = np.where(msgs < 16, luts[np.arange(count), msgs % 16], (32 - luts[np.arange(count), msgs % 16]) % 32)
    got = [L.lvs_decrypt_lwe(ck, row) for row in fft]
    assert got == [int(v) for v in expect]
    assert got == [L.lvs_decrypt_lwe(ck, row) for row in ntt]
    # The two outputs are not close coefficient by coefficient: the FFT's
    # rounding moves some accumulator values across a gadget rounding
    # boundary, which changes a digit and adds a whole bootstrapping-key row
    # (a fresh-looking mask) while the phase barely moves.  Compare phases.
    mask = glwe_key.astype(bool)

    def phase(o):
        return o[:, big] - o[:, :big][:, mask].sum(axis=1, dtype=np.uint64)

    dphase = (phase(fft) - phase(ntt)).view(np.int64).astype(np.float64)
    print("FFT - NTT phase: max |diff| 2^%.2f, rms 2^%.2f" % (
        np.log2(max(float(np.max(np.abs(dphase))), 1.0)), 0.5 * np.log2(max(float(np.mean(dphase ** 2)), 1.0))))
    # both decode with margin: the phases differ by far less than half a plaintext step (2^58)
    assert float(np.max(np.abs(dphase))) < 2.0 ** 57
    L.lvs_ctx_free(ctx)


def test_fft_pbs_noise_matches_model():
    p = L.lvs_params_default()
    ck, sk = L.lvs_keygen(p, 5)
    ctx = L.lvs_ctx_create(sk, 0)
    L.lvs_ctx_prepare_fft64(ctx, sk)
    lwe_key, glwe_key = L.lvs_client_key_export(ck)
    big = p.k * p.N
    count = 2048
    rng = np.random.default_rng(1)
    msgs = rng.integers(0, 16, size=count)
    cts = np.stack([L.lvs_encrypt_lwe(ck, int(m), 8, 0, i, big) for i, m in enumerate(msgs)])
    ident = np.tile(np.arange(16, dtype=np.uint8), (count, 1))
    out = _run(ctx, L.lvs_pbs_batch_device_fft64, cts, ident, big)
    err = _phase_err(out, glwe_key, msgs, big)
    measured = float(np.mean(err ** 2))
    predicted = predicted_pbs_variance(p, lwe_key, glwe_key)
    ratio = measured / predicted
    print("FFT PBS noise: measured 2^%.3f predicted 2^%.3f ratio %.3f" % (np.log2(measured), np.log2(predicted), ratio))
    assert abs(float(np.mean(err))) < 4 * np.sqrt(measured / count)
    assert 0.85 < ratio < 1.2
    assert np.max(np.abs(err)) < 2.0 ** 58
    L.lvs_ctx_free(ctx)


def test_fft_requires_prepare_and_matching_key():
    p = L.lvs_params_test()
    ck, sk = L.lvs_keygen(p, 3)
    ctx = L.lvs_ctx_create(sk, 0)
    big = p.k * p.N
    d = torch.zeros((1, big + 1), dtype=torch.int64, device="cuda")
    lut = torch.zeros((1, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvsError) as ei:
        L.lvs_pbs_batch_device_fft64(ctx, d, big + 1, lut, d, big + 1, 1)
    assert ei.value.status == L.LVS_ERR_STATE
    _, sk2 = L.lvs_keygen(L.lvs_params_default(), 3)
    with pytest.raises(L.LvsError) as ei:
        L.lvs_ctx_prepare_fft64(ctx, sk2)
    assert ei.value.status == L.LVS_ERR_ARG
    L.lvs_ctx_free(ctx)
