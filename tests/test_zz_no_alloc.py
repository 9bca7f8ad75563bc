"""lvs_pbs_batch_device_noalloc: the allocation-free PBS entry point, for
callers that cannot allocate device memory at call time (a server whose
memory budget is reserved at start-up, a latency-critical path, a host whose
allocator belongs to another framework).  Its output must equal that of
lvs_pbs_batch_device, which allocates its scratch through the context, bit
for bit (all values are integers mod 2^64), on two calls in a row that share
the static scratch array.  Collected last on purpose (file name)."""
import numpy as np
import pytest

from paper_2508_14568_gb300 import lvs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs(ck, big, count, seed):
    rng = np.random.default_rng(seed)
    msgs = rng.integers(0, 32, size=count)
    cts = np.stack([L.lvs_encrypt_lwe(ck, int(m), seed, 0, i, big) for i, m in enumerate(msgs)])
    luts = rng.integers(0, 32, size=(count, 16)).astype(np.uint8)
    luts[::3] = [9] + [0] * 15                               # LUT_EQ9
    luts[1::3] = [0, 0, 0, 1, 1, 0, 1, 1] + [0] * 8          # LUT_min (key of Eq. eq_keyeq2)
    return msgs, cts, luts


def _lookup(lut, x):
    return int(lut[x]) % 32 if x < 16 else (-int(lut[x - 16])) % 32


@pytest.mark.parametrize("which", ["test", "default"])
def test_noalloc_matches_allocating_entry_point_twice(which):
    params = L.lvs_params_test() if which == "test" else L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 21)
    ctx = L.lvs_ctx_create(sk, 0)
    big = params.k * params.N
    for call, (count, seed) in enumerate([(37, 5), (23, 6)]):     # two calls in a row
        msgs, cts, luts = _inputs(ck, big, count, seed)
        d_in = torch.from_numpy(cts.view(np.int64)).cuda()
        d_lut = torch.from_numpy(np.ascontiguousarray(luts)).cuda()
        ref = torch.zeros_like(d_in)
        out = torch.full_like(d_in, -1)
        L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, ref, big + 1, count)
        L.lvs_pbs_batch_device_noalloc(ctx, d_in, big + 1, d_lut, out, big + 1, count)
        L.lvs_ctx_synchronize(ctx)
        a, b = ref.cpu().numpy(), out.cpu().numpy()
        assert np.array_equal(a, b), "call %d differs" % call
        for i in range(count):
            assert L.lvs_decrypt_lwe(ck, b[i].view(np.uint64)) == _lookup(luts[i], int(msgs[i]))


def test_noalloc_rejects_counts_beyond_the_static_scratch():
    params = L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 22)
    ctx = L.lvs_ctx_create(sk, 0)
    big = params.k * params.N
    d = torch.zeros((2, big + 1), dtype=torch.int64, device="cuda")
    lut = torch.zeros((2, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvsError) as e:
        L.lvs_pbs_batch_device_noalloc(ctx, d, big + 1, lut, d, big + 1, 100000)
    assert e.value.status == L.LVS_ERR_ARG and "static scratch" in str(e.value)
