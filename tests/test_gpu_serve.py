"""Continuous-batching server (lvs_server_*) on the GPU: every result equals
the result of the same query run alone (bit for bit: the NTT path is exact),
decrypts to the Wagner-Fischer distance, and queries are admitted under the
device-memory budget and merged while others run."""
import time

import numpy as np
import pytest

from oracle import plain as P
from paper_2508_14568_gb300 import lvs as L
from paper_2508_14568_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    ck, sk = L.lvs_keygen(L.lvs_params_test(), 0)
    ctx = L.lvs_ctx_create(sk, 0)
    return ck, ctx, 512


def _queries(seed, count):
    import random
    rng = random.Random(seed)
    out = []
    for k in range(count):
        a = "".join(rng.choice(W.ALPHA27[:7]) for _ in range(rng.randint(1, 9)))
        b = "".join(rng.choice(W.ALPHA27[:7]) for _ in range(rng.randint(0 if k == 3 else 1, 9)))
        out.append((a, b, k % 2 == 0))       # plaintext reference on even k
    return out


def _submit(ck, server, qs, seed):
    tickets, keep = [], []
    for k, (a, b, plain) in enumerate(qs):
        qa = L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_27, seed, 2 * k)
        if plain:
            t = L.lvs_server_submit(server, qa, ref_plain=b)
        else:
            rb = L.lvs_encrypt_string(ck, b, L.LVS_ALPHA_27, seed, 2 * k + 1)
            t = L.lvs_server_submit(server, qa, ref_enc=rb)
            keep.append(rb)
        keep.append(qa)
        tickets.append(t)
    return tickets


def _collect(server, tickets, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = L.lvs_server_poll(server, t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.002)
    return [res[t] for t in tickets]


def test_server_results_same_alone_and_in_the_mix(setup):
    ck, ctx, big = setup
    qs = _queries(1, 12)
    server = L.lvs_server_create(ctx, 1 << 34)
    mix = _collect(server, _submit(ck, server, qs, 40))
    d_mix = [L.lvs_decrypt(ck, r, 0) for r in mix]
    assert d_mix == [P.wf_distance(a, b) for a, b, _ in qs]
    ct_mix = [L.lvs_result_export(r, 0, big) for r in mix]
    del server
    # each query alone, same ciphertexts (same encryption seeds and ids)
    for k, q in enumerate(qs):
        server = L.lvs_server_create(ctx, 1 << 34)
        qa = L.lvs_encrypt_string(ck, q[0], L.LVS_ALPHA_27, 40, 2 * k)
        if q[2]:
            t = L.lvs_server_submit(server, qa, ref_plain=q[1])
        else:
            rb = L.lvs_encrypt_string(ck, q[1], L.LVS_ALPHA_27, 40, 2 * k + 1)
            t = L.lvs_server_submit(server, qa, ref_enc=rb)
        (r,) = _collect(server, [t])
        assert np.array_equal(L.lvs_result_export(r, 0, big), ct_mix[k]), k
        del server
    # encrypted-reference queries also equal the batch call
    enc = [(k, q) for k, q in enumerate(qs) if not q[2]]
    A = [L.lvs_encrypt_string(ck, q[0], L.LVS_ALPHA_27, 40, 2 * k) for k, q in enc]
    B = [L.lvs_encrypt_string(ck, q[1], L.LVS_ALPHA_27, 40, 2 * k + 1) for k, q in enc]
    rb = L.lvs_edit_distance_batch(ctx, A, B)
    for idx, (k, q) in enumerate(enc):
        assert np.array_equal(L.lvs_result_export(rb, idx, big), ct_mix[k])


def test_server_admission_under_small_budget(setup):
    ck, ctx, big = setup
    qs = _queries(2, 8)
    stride_bytes = (big + 2) * 8
    budget = 140 * stride_bytes          # roughly one query at a time
    server = L.lvs_server_create(ctx, budget)
    res = _collect(server, _submit(ck, server, qs, 41))
    assert [L.lvs_decrypt(ck, r, 0) for r in res] == [P.wf_distance(a, b) for a, b, _ in qs]
    st = L.lvs_server_stats_get(server)
    assert st["completed"] == st["submitted"] == len(qs)
    assert st["mem_in_use"] == 0 and st["pending"] == 0
    with pytest.raises(L.LvsError) as e:                       # one query larger than the budget
        L.lvs_server_submit(server, L.lvs_encrypt_string(ck, "A" * 60, L.LVS_ALPHA_27, 1, 1), ref_plain="B" * 60)
    assert e.value.status == L.LVS_ERR_ARG
    with pytest.raises(L.LvsError):
        L.lvs_server_poll(server, 10**9)


def test_server_merges_arrivals_while_running(setup):
    ck, ctx, big = setup
    qs = _queries(3, 10)
    server = L.lvs_server_create(ctx, 1 << 34, max_active=3)
    tickets = []
    keep = []
    for k, (a, b, plain) in enumerate(qs):
        qa = L.lvs_encrypt_string(ck, a, L.LVS_ALPHA_27, 42, 2 * k)
        keep.append(qa)
        tickets.append(L.lvs_server_submit(server, qa, ref_plain=b) if plain else
                       L.lvs_server_submit(server, qa, ref_enc=L.lvs_encrypt_string(ck, b, L.LVS_ALPHA_27, 42, 2 * k + 1)))
        time.sleep(0.003)
    res = _collect(server, tickets)
    assert [L.lvs_decrypt(ck, r, 0) for r in res] == [P.wf_distance(a, b) for a, b, _ in qs]
    st = L.lvs_server_stats_get(server)
    assert st["steps"] >= 1 and st["pbs"] > 0


def test_batch_call_reports_injected_allocation_failure(setup):
    """Host-side fault injection: a failed device allocation is an error
    status (LVS_ERR_OOM), not a crash, and the next call works."""
    ck, ctx, _ = setup
    A = [L.lvs_encrypt_string(ck, "ABC", L.LVS_ALPHA_27, 91, 0)]
    B = [L.lvs_encrypt_string(ck, "ABD", L.LVS_ALPHA_27, 91, 1)]
    L.lvs_debug_fail_allocations(1)
    with pytest.raises(L.LvsError) as ei:
        L.lvs_edit_distance_batch(ctx, A, B)
    assert ei.value.status == L.LVS_ERR_OOM
    r = L.lvs_edit_distance_batch(ctx, A, B)
    assert L.lvs_decrypt_all(ck, r) == [1]


def test_server_requeues_a_query_whose_allocation_failed(setup):
    ck, ctx, _ = setup
    server = L.lvs_server_create(ctx, 1 << 34)
    import random
    rng = random.Random(92)
    long_a = "".join(rng.choice(W.ALPHA27[:5]) for _ in range(120))
    long_b = "".join(rng.choice(W.ALPHA27[:5]) for _ in range(120))
    qs = [(long_a, long_b, False), ("HELLO", "HALLO", True)]
    t1 = _submit(ck, server, qs[:1], 93)
    t0 = time.time()
    while L.lvs_server_stats_get(server)["active"] < 1:
        assert time.time() - t0 < 30
        time.sleep(0.0005)
    L.lvs_debug_fail_allocations(1)      # the next admission's allocation fails
    t2 = _submit(ck, server, qs[1:], 94)
    res = _collect(server, t1 + t2)
    st = L.lvs_server_stats_get(server)
    L.lvs_debug_fail_allocations(0)
    assert st["requeued"] >= 1
    for r, (a, b, _) in zip(res, qs):
        assert L.lvs_decrypt(ck, r, 0) == P.wf_distance(a, b)
    L.lvs_server_free(server)


def test_server_lone_query_allocation_failure_is_reported(setup):
    ck, ctx, _ = setup
    server = L.lvs_server_create(ctx, 1 << 34)
    L.lvs_debug_fail_allocations(1)
    t = _submit(ck, server, [("AB", "BA", True)], 95)
    t0 = time.time()
    with pytest.raises(L.LvsError) as ei:
        while L.lvs_server_poll(server, t[0]) is None:
            assert time.time() - t0 < 30
            time.sleep(0.002)
    assert ei.value.status == L.LVS_ERR_OOM
    L.lvs_debug_fail_allocations(0)
    L.lvs_server_free(server)
