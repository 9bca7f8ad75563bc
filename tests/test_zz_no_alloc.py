"""lvs_pbs_batch_device_noalloc: the allocation-free PBS entry point, for
callers that cannot allocate device memory at call time (a server whose
memory budget is reserved at start-up, a latency-critical path, a host whose
allocator belongs to another framework).  Its output must equal that of
lvs_pbs_batch_device, which allocates its scratch through the context, bit
for bit (all values are integers mod 2^64), on two calls in a row that share
the static scratch array, in both blind-rotation forms, at the array's exact
size limit, and while another host thread changes the context's launch
settings.  Collected last on purpose (file name)."""
import threading

import numpy as np
import pytest

from paper_2508_14568_gb300 import lvs as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# largest call the 4 MiB static array takes at n = 834: 1232 * 64 bytes of jobs
# (already a multiple of 256) + 1232 * 835 * 4 bytes of masks = 4,193,728 bytes
LIMIT_DEFAULT = 1232


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


def _both(ctx, ck, big, count, seed, check_decrypt=True):
    msgs, cts, luts = _inputs(ck, big, count, seed)
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(np.ascontiguousarray(luts)).cuda()
    ref = torch.zeros_like(d_in)
    out = torch.full_like(d_in, -1)
    L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, ref, big + 1, count)
    L.lvs_pbs_batch_device_noalloc(ctx, d_in, big + 1, d_lut, out, big + 1, count)
    L.lvs_ctx_synchronize(ctx)
    a, b = ref.cpu().numpy(), out.cpu().numpy()
    if check_decrypt:
        for i in range(count):
            assert L.lvs_decrypt_lwe(ck, b[i].view(np.uint64)) == _lookup(luts[i], int(msgs[i]))
    return a, b


@pytest.fixture(scope="module")
def default_ctx():
    params = L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 21)
    ctx = L.lvs_ctx_create(sk, 0)
    return params, ck, ctx


@pytest.mark.parametrize("which", ["test", "default"])
def test_noalloc_matches_allocating_entry_point_twice(which):
    params = L.lvs_params_test() if which == "test" else L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 21)
    ctx = L.lvs_ctx_create(sk, 0)
    big = params.k * params.N
    for call, (count, seed) in enumerate([(37, 5), (23, 6)]):     # two calls in a row
        a, b = _both(ctx, ck, big, count, seed)
        assert np.array_equal(a, b), "call %d differs" % call


def test_noalloc_one_cta_form_and_the_size_limit(default_ctx):
    """Default parameters above the three-CTA crossover (the one-CTA blind
    rotation runs through the static scratch), then exactly the largest call
    the array takes, then one PBS more, which is refused."""
    params, ck, ctx = default_ctx
    big = params.k * params.N
    assert L.lvs_ctx_br_split(ctx) < 200
    a, b = _both(ctx, ck, big, 200, 8)
    assert np.array_equal(a, b)
    a, b = _both(ctx, ck, big, LIMIT_DEFAULT, 9, check_decrypt=False)
    assert np.array_equal(a, b)
    d = torch.zeros((LIMIT_DEFAULT + 1, big + 1), dtype=torch.int64, device="cuda")
    lut = torch.zeros((LIMIT_DEFAULT + 1, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvsError) as e:
        L.lvs_pbs_batch_device_noalloc(ctx, d, big + 1, lut, d, big + 1, LIMIT_DEFAULT + 1)
    assert e.value.status == L.LVS_ERR_ARG and "static scratch" in str(e.value)


def test_noalloc_rejects_counts_beyond_the_static_scratch(default_ctx):
    params, ck, ctx = default_ctx
    big = params.k * params.N
    d = torch.zeros((2, big + 1), dtype=torch.int64, device="cuda")
    lut = torch.zeros((2, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvsError) as e:
        L.lvs_pbs_batch_device_noalloc(ctx, d, big + 1, lut, d, big + 1, 100000)
    assert e.value.status == L.LVS_ERR_ARG and "static scratch" in str(e.value)


def test_noalloc_bit_exact_while_another_thread_changes_the_settings(default_ctx):
    """A second host thread flips the blind rotation's form crossover and the
    key-switch plans while this thread repeats allocation-free calls: both
    take the context's lock, every form computes the same integers, so every
    output stays equal to the reference."""
    params, ck, ctx = default_ctx
    big = params.k * params.N
    count = 120
    msgs, cts, luts = _inputs(ck, big, count, 10)
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(np.ascontiguousarray(luts)).cuda()
    ref = torch.zeros_like(d_in)
    L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, ref, big + 1, count)
    L.lvs_ctx_synchronize(ctx)
    want = ref.cpu().numpy()
    split0 = L.lvs_ctx_br_split(ctx)
    stop = threading.Event()
    errors = []

    def setter():
        k = 0
        try:
            while not stop.is_set():
                L.lvs_ctx_set_br_split(ctx, (0, 200, split0)[k % 3])
                L.lvs_ctx_set_ks_plan(ctx, count, (4, 16, 0)[k % 3], (1, 8, 1)[k % 3])
                k += 1
        except Exception as ex:   # reported by the main thread
            errors.append(ex)

    t = threading.Thread(target=setter)
    t.start()
    try:
        for it in range(8):
            out = torch.full_like(d_in, -1)
            L.lvs_pbs_batch_device_noalloc(ctx, d_in, big + 1, d_lut, out, big + 1, count)
            L.lvs_ctx_synchronize(ctx)
            assert np.array_equal(out.cpu().numpy(), want), "iteration %d differs" % it
    finally:
        stop.set()
        t.join()
        L.lvs_ctx_set_br_split(ctx, split0)
        L.lvs_ctx_set_ks_plan(ctx, count, 0, 1)
    assert not errors, errors


def test_noalloc_launches_are_timed_and_counted(default_ctx):
    params, ck, ctx = default_ctx
    big = params.k * params.N
    count = 40
    msgs, cts, luts = _inputs(ck, big, count, 11)
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_lut = torch.from_numpy(np.ascontiguousarray(luts)).cuda()
    out = torch.zeros_like(d_in)
    L.lvs_ctx_set_timing(ctx, True)
    n0 = L.lvs_ctx_launch_count(ctx)
    L.lvs_pbs_batch_device_noalloc(ctx, d_in, big + 1, d_lut, out, big + 1, count)
    L.lvs_ctx_synchronize(ctx)
    assert L.lvs_ctx_launch_count(ctx) - n0 == 3
    br = L.lvs_ctx_kernel_stats(ctx, 0)
    ks = L.lvs_ctx_kernel_stats(ctx, 1)
    L.lvs_ctx_set_timing(ctx, False)
    assert br["launches"] == 1 and br["items"] == count and br["total_ms"] > 0
    assert ks["launches"] == 1 and ks["items"] == count
