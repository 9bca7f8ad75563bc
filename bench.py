#!/usr/bin/env python3
"""Benchmark of the encrypted Leuvenshtein hot path on GB300.

Default workload (one "step"): the batching configuration -- 256 encrypted
ASCII pairs, lengths uniform in [8, 16], 30% near-duplicates -- under the full
TFHE parameter set (n=834, N=2048), all pairs advanced together in
anti-diagonal-union launches (3 PBS per cell).  Metric: encrypted DP cells/s
(whole job, all GPUs); PBS/s and the roofline fraction of the blind-rotation
kernel ride along.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lvs|reference]
                  [--config 1|2|3|4] [--pairs P] [--no-e2e] [--no-cpu-baseline]

N > 1 is launched with torch.distributed.run (one rank per GPU): every rank
runs its own batch of independent pairs (weak scaling, no data-path
collective); timing is max over ranks.  --impl reference times the CPU oracle
(oracle/, schoolbook TFHE) on the host cores on a bounded sample of the same
workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))

# The paper's own figures, quoted beside ours as context only: CPU (dual AMD
# EPYC 9174F, 32 cores / 64 threads, TFHE-rs v0.7.2 with its "4-bit message,
# 0-bit carry" parameters, Section 6.2), another machine and another parameter
# set, so no ratio to them is taken.
PAPER_CONTEXT = {
    "hardware": "2x AMD EPYC 9174F (32 cores, 64 threads), TFHE-rs v0.7.2, 4-bit message / 0-bit carry set",
    # Table tab_lat: Leuvenshtein Exact, one thread, m = n = 100 in 7 min 19 s (3 PBS per cell)
    "exact_1_thread_m100_cells_per_s": round(100 * 100 / 439.0, 1),
    "exact_1_thread_m100_pbs_per_s": round(3 * 100 * 100 / 439.0, 1),
    # Table table:results_parallel: 64 distances in a batch, 14.7 s per distance amortised
    "exact_64_threads_m100_cells_per_s": round(100 * 100 / 14.7, 1),
    # Table tab_unenc: preprocessed online phase, m = n = 256 in 950 s (1 PBS per cell)
    "preprocessed_1_thread_m256_cells_per_s": round(256 * 256 / 950.0, 1),
    "speedups_claimed": {
        "vs_concrete_m256_exact_skip": "278x (Table tab_lat)",
        "vs_wagner_fischer_on_tfhe_rs": "39-40x (Table tab_lat, Section 1.1)",
        "preprocessing_online": "3x (Table tab_unenc)",
        "batching_64_threads": "~32x (Table table:results_parallel)",
    },
}
sys.path.insert(0, ROOT)

SM_COUNT_NOMINAL = 152
MUL32_PER_SM_CLK = 64        # 32-bit integer multiply throughput per SM per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lvs", choices=["lvs", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--rate", type=float, default=200.0, help="config 5: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="config 5: arrival window in seconds")
    ap.add_argument("--slots", type=int, default=16, help="config 5: server slots (admitted queries)")
    ap.add_argument("--serve-rate", type=float, default=2.0,
                    help="serving segment of the default run: Poisson arrivals per second (0: no segment)")
    ap.add_argument("--serve-duration", type=float, default=30.0, help="serving segment: arrival window in seconds")
    ap.add_argument("--serve-alone", type=int, default=16,
                    help="serving segment: queries of the segment also run one at a time (alone on the server)")
    ap.add_argument("--serial-pairs", type=int, default=8,
                    help="pairs run one at a time for the one-pair-at-a-time comparison (0: skip)")
    ap.add_argument("--pairs", type=int, default=None, help="override the number of pairs (small profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=None, help="PBS in the oracle sample (default: host cores)")
    ap.add_argument("--pbs-variants", type=int, default=0, metavar="COUNT",
                    help="instead of a config: time COUNT independent PBS through the exact NTT blind rotation "
                         "and through the FP64-FFT one (side measurement, its own JSON line)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- workloads

def workload(cfg, rank, pairs_override):
    from paper_2508_14568_gb300 import workloads as W
    if cfg == 1:
        pairs = W.config1(W.SEED_BASE + 1 + 100 * rank)
        alpha, desc = "ascii7", "config 1: one encrypted ASCII pair, lengths 4 and 4"
    elif cfg == 2:
        pairs = W.config2(W.SEED_BASE + 2 + 100 * rank, pairs=pairs_override or 256)
        alpha = "ascii7"
        desc = "config 2: %d encrypted ASCII pairs, lengths U[8,16], 30%% near-duplicates" % len(pairs)
    elif cfg == 3:
        pairs = W.config3(W.SEED_BASE + 3 + 100 * rank, queries=pairs_override or 1024)
        alpha = "alpha27"
        desc = "config 3: %d preprocessed queries, 27 symbols, lengths U[8,32]" % len(pairs)
    else:
        pairs = W.config4(W.SEED_BASE + 4 + 100 * rank, pairs=pairs_override or 64)
        alpha = "dna4"
        desc = "config 4: %d encrypted DNA pairs, lengths U[64,256], 10%% mutation" % len(pairs)
    return pairs, alpha, desc


def pbs_per_cell(cfg):
    return {1: 3, 2: 3, 3: 1, 4: 2}[cfg]


def key_row_bytes(params):
    """Bytes of one NTT-domain BSK row (one CMux): 3 primes x (k+1)^2 l_b polynomials x N residues x 4 B."""
    return 3 * (params.k + 1) ** 2 * params.pbs_level * params.N * 4


def modmul_per_pbs(p):
    """Algorithmic modular multiplications of one blind rotation on the exact
    NTT path: n * P * [((k+1) l + (k+1)) (N/2) log2 N + (k+1)^2 l N]
    (forward transforms of the digit polynomials, inverse transforms of the
    outputs, pointwise key products), P = 3 primes."""
    logN = p.N.bit_length() - 1
    k, l = p.k, p.pbs_level
    return p.n * 3 * (((k + 1) * l + (k + 1)) * (p.N // 2) * logN + (k + 1) ** 2 * l * p.N)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- checks

def levenshtein(a, b):
    """Plain edit distance (two-row Wagner-Fischer), to check every decrypted
    distance the bench produces."""
    prev = list(range(len(b) + 1))
    for i, ca in enumerate(a, 1):
        cur = [i] + [0] * len(b)
        for j, cb in enumerate(b, 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (ca != cb))
        prev = cur
    return prev[-1]


# ----------------------------------------------------------------------------- oracle timing

def oracle_sample(pairs, alpha, count, seed=0):
    """`count` PBS inputs of the workload (first-equality inputs x1_i - y1_j of
    successive cells, LUT_EQ; all PBS of the method cost the same), built by the
    oracle itself from its own keys and encryption."""
    import numpy as np
    from oracle import plain as P
    from oracle import tfhe as T
    K = T.Keys(T.params_lvs(), seed)
    cts, luts = [], []
    k = 0
    for pi, (a, b) in enumerate(pairs):
        xa = T.encrypt_string(K, a[:4], alpha, 99, 2 * pi)
        yb = T.encrypt_string(K, b[:4], alpha, 99, 2 * pi + 1)
        for i in range(len(xa)):
            for j in range(len(yb)):
                if k < count:
                    cts.append(xa[i][0] - yb[j][0])
                    luts.append(P.LUT_EQ)
                    k += 1
        if k >= count:
            break
    return K, np.stack(cts), np.asarray(luts, np.uint32)


def time_oracle(K, cts, luts, cores):
    from oracle import tfhe as T
    t0 = time.perf_counter()
    out = T.pbs_many(K, cts, luts, nthreads=cores)
    return time.perf_counter() - t0, out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import tfhe as T
    cfg = args.config
    pairs, alpha, desc = workload(cfg, 0, args.pairs)
    cores = os.cpu_count() or 1
    count = args.cpu_sample or cores
    T.build()
    K, cts, luts = oracle_sample(pairs, alpha, count)
    for _ in range(args.warmup):
        time_oracle(K, cts[:min(len(cts), cores)], luts[:min(len(cts), cores)], cores)
    total = 0.0
    for _ in range(args.steps):
        dt, _ = time_oracle(K, cts, luts, cores)
        total += dt
    pbs_s = count * args.steps / total
    cells_s = pbs_s / pbs_per_cell(cfg)
    sample = "%d independent full-parameter PBS per step (schoolbook TFHE, %d threads); cells/s = PBS/s / %d" % (
        count, cores, pbs_per_cell(cfg))
    line = {
        "impl": "reference", "metric": "encrypted DP cells/s", "value": cells_s, "unit": "cells/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": desc, "params": "n=834 k=1 N=2048 pbs 2x2^13 ks 5x2^3"},
        "pbs_per_s": pbs_s,
        "cpu_baseline": {"value": cells_s, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": cells_s, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "ntt.cuh"):
        with open(os.path.join(ROOT, "paper_2508_14568_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record():
    """DRAM bytes per blind-rotation launch from the committed ncu summary, if
    it was taken on the current kernel source (else null)."""
    path = os.path.join(ROOT, "profiles", "br_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("kernel_source_hash") != kernel_source_hash():
        return None
    return rec


class Ranks:
    """The launch's ranks: barrier and max / sum of a scalar over ranks (the
    bench reports the whole-job value = units of all ranks / max time).  One
    rank: no process group.  device: 'cuda' under NCCL, 'cpu' under gloo."""

    def __init__(self, world, device="cuda"):
        self.world, self.device = world, device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def _reduce(self, x, op):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.MAX)

    def sum(self, x):
        import torch.distributed as dist
        return self._reduce(x, dist.ReduceOp.SUM)


def run_lvs(args):
    import torch
    import torch.distributed as dist
    from paper_2508_14568_gb300 import lvs as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ranks = Ranks(world, "cuda")
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    cfg = args.config
    pairs, alpha, desc = workload(cfg, rank, args.pairs)
    A_L = {"ascii7": L.LVS_ALPHA_ASCII7, "alpha27": L.LVS_ALPHA_27, "dna4": L.LVS_ALPHA_DNA4}[alpha]
    params = L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 0)
    # a stream of our own: the library runs on it and the timing events are
    # recorded on it (the default stream has handle 0, which the library reads
    # as "no stream given" and replaces with a non-blocking stream of its own)
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    ctx = L.lvs_ctx_create(sk, local, stream)
    # key-switch launch shapes by measurement (before any timing)
    L.lvs_ctx_autotune(ctx)
    ks_plans = {str(nj): list(L.lvs_ctx_ks_plan(ctx, nj)) for nj in (4, 16, 64, 256, 1024, 4096)}
    br_split = L.lvs_ctx_br_split(ctx)
    ks_gemm_min = L.lvs_ctx_ks_gemm_min(ctx)
    big = params.k * params.N
    cells = sum(len(a) * len(b) for a, b in pairs)
    want = [levenshtein(a, b) for a, b in pairs]

    def encrypt_all(seed):
        if cfg == 3:
            return [L.lvs_encrypt_string(ck, a, A_L, seed, k) for k, (a, b) in enumerate(pairs)], None
        A = [L.lvs_encrypt_string(ck, a, A_L, seed, 2 * k) for k, (a, b) in enumerate(pairs)]
        B = [L.lvs_encrypt_string(ck, b, A_L, seed, 2 * k + 1) for k, (a, b) in enumerate(pairs)]
        return A, B

    # device-resident inputs for the kernel-side number
    A_dev, B_dev = encrypt_all(7)
    tables = None
    table_build = None
    if cfg == 3:
        # offline phase (Section 5), timed on its own: every table in one set of launches
        torch.cuda.synchronize()
        tb0 = time.perf_counter()
        tables = L.lvs_preprocess_batch(ctx, A_dev)
        L.lvs_ctx_synchronize(ctx)
        tb = time.perf_counter() - tb0
        tb_pbs = sum(2 * 27 * len(a) for a, b in pairs)
        table_build = {"pbs": tb_pbs, "ms": 1e3 * tb, "pbs_per_s": tb_pbs / tb,
                       "note": "lvs_preprocess_batch: 27 symbols x len x 2 PBS per string, all strings at once, "
                               "host-timed around the call (not in value)"}
        plains = [b for a, b in pairs]
        step = lambda: L.lvs_edit_distance_preprocessed_batch(ctx, tables, plains)
    else:
        for s in A_dev + B_dev:
            L.lvs_ct_string_upload(ctx, s)
        step = lambda: L.lvs_edit_distance_batch(ctx, A_dev, B_dev)

    # noise budget of the workload (Section 3.1.3): the largest key variance of
    # any pair (PBS-output units) against the budget for a 2^-64 failure rate
    nb = L.lvs_noise_budget(params, -64.0)
    worst_key = max((L.lvs_noise_plan(len(a), len(b), -1, 0)[1] for a, b in pairs), default=0.0)
    noise = {"budget_key_var": nb, "max_key_var": worst_key,
             "log2_pfail_worst_key": L.lvs_noise_pfail(params, worst_key),
             "refreshed": worst_key > nb,
             "note": "key variance in PBS-output variances; refresh of dv/dh only above the budget"}

    # warm-up (+ correctness of every distance)
    r = None
    for w in range(max(1, args.warmup)):
        r = step()
        if w == 0:
            got = L.lvs_decrypt_all(ck, r)
            assert got == want, "decrypted distances differ from Wagner-Fischer"
    torch.cuda.synchronize()
    r = None

    L.lvs_ctx_set_timing(ctx, True)
    launches0 = L.lvs_ctx_launch_count(ctx)
    pbs0 = L.lvs_ctx_pbs_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        r = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    r = None
    dev_ms = ev0.elapsed_time(ev1)
    launches = L.lvs_ctx_launch_count(ctx) - launches0
    pbs_done = L.lvs_ctx_pbs_count(ctx) - pbs0
    br = L.lvs_ctx_kernel_stats(ctx, 0)
    ks = L.lvs_ctx_kernel_stats(ctx, 1)
    L.lvs_ctx_set_timing(ctx, False)

    t_max = max_over_ranks(dev_ms / 1e3)
    cells_all = sum_over_ranks(cells * args.steps)
    pbs_all = sum_over_ranks(pbs_done)
    value = cells_all / t_max

    # roofline of the blind-rotation kernel (ALU bound: modular multiplications)
    w_mod = modmul_per_pbs(params)
    avg_launch_s = br["total_ms"] / max(1, br["launches"]) / 1e3
    units_per_launch = br["items"] / max(1, br["launches"])
    achieved = w_mod * units_per_launch / avg_launch_s / 1e12 if br["launches"] else None
    sm_mhz_max = clk.get("sm_max_mhz") or 2070.0
    mul_lo, mul_hi = L.lvs_probe_int_mul(local)
    modmul_per_sm_clk = 1.0 / (2.0 / mul_lo + 1.0 / mul_hi)
    shoup_stream, bfly_stream = L.lvs_probe_modmul(local)
    wide_mac, l2_bytes_clk = L.lvs_probe_key_product(local)
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sms * modmul_per_sm_clk * sm_mhz_max * 1e6 / 1e12
    peak_mul32 = n_sms * MUL32_PER_SM_CLK * sm_mhz_max * 1e6 / 1e12
    trec = traffic_record()
    traffic = None
    if trec:
        traffic = trec["dram_bytes_per_pbs"] * units_per_launch

    # the plain one-pair-at-a-time GPU form on the same inputs (a sample of pairs)
    serial = None
    if rank == 0 and cfg in (2, 4) and args.serial_pairs > 0:
        lat = []
        cells_s = 0
        for k in range(min(args.serial_pairs, len(pairs))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r1 = L.lvs_edit_distance_batch(ctx, [A_dev[k]], [B_dev[k]])
            L.lvs_ctx_synchronize(ctx)
            lat.append(time.perf_counter() - t0)
            cells_s += len(pairs[k][0]) * len(pairs[k][1])
            r1 = None
        lat.sort()
        serial = {"cells_per_s": cells_s / sum(lat), "pairs": len(lat),
                  "latency_ms_p50": 1e3 * lat[len(lat) // 2], "latency_ms_max": 1e3 * lat[-1],
                  "note": "each pair alone through lvs_edit_distance_batch (same inputs, same kernels)"}
    batched_latency_ms = t_max * 1e3 / args.steps   # every pair of a batch completes at the end of its step

    # end to end: host strings in, decrypted distances out
    e2e = None
    if not args.no_e2e:
        A_h, B_h = encrypt_all(11)
        for s_ in A_h + (B_h or []):
            L.lvs_ct_string_pin(s_)       # inputs in page-locked host memory (set-up, not timed)
        if cfg == 3:
            e2e_step = lambda: L.lvs_edit_distance_preprocessed_batch(ctx, tables, plains)
            h2d = 0
        else:
            e2e_step = lambda: L.lvs_edit_distance_batch(ctx, A_h, B_h)
            h2d = sum((len(a) + len(b)) * (2 if cfg != 4 else 1) * (big + 1) * 8 for a, b in pairs)
        d2h = sum(len(b) * (big + 1) * 8 for a, b in pairs)
        got = L.lvs_decrypt_all(ck, e2e_step())
        assert got == want
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            got = L.lvs_decrypt_all(ck, e2e_step())
        torch.cuda.synchronize()
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": cells_all / t_e2e, "unit": "cells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * t_e2e / args.steps,
               "note": "pinned host encrypted strings -> lvs_edit_distance_batch (H2D inside) -> D2H + client "
                       "decryption"}

    # serving segment: continuous batching at a sustainable rate, with the same
    # queries one at a time (rank 0, N = 1; not part of value)
    serving = None
    if rank == 0 and world == 1 and cfg == 2 and args.serve_rate > 0:
        serving = serving_segment(L, ctx, ck, args.serve_rate, args.serve_duration, args.slots, args.serve_alone)

    # CPU oracle baseline (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np
        cores = os.cpu_count() or 1
        count = args.cpu_sample or cores
        K, cts, luts = oracle_sample(pairs, alpha, count)
        dt, out = time_oracle(K, cts, luts, cores)
        # the same inputs through the GPU PBS (parity of the sample)
        d_in = torch.from_numpy(np.ascontiguousarray(cts).view(np.int64)).cuda()
        d_lut = torch.from_numpy(np.ascontiguousarray(luts.astype(np.uint8))).cuda()
        d_out = torch.zeros_like(d_in)
        # the oracle keys equal the library keys from the same seed; the sample
        # runs through the blind-rotation form of the timed launches (one CTA
        # per ciphertext), not the three-CTA form its small size would pick
        split0 = L.lvs_ctx_br_split(ctx)
        L.lvs_ctx_set_br_split(ctx, 0)
        L.lvs_pbs_batch_device(ctx, d_in, big + 1, d_lut, d_out, big + 1, count)
        L.lvs_ctx_synchronize(ctx)
        L.lvs_ctx_set_br_split(ctx, split0)
        same = bool(np.array_equal(d_out.cpu().numpy().view(np.uint64), out))
        pbs_s = count / dt
        cpu = {"value": pbs_s / pbs_per_cell(cfg), "unit": "cells/s", "cores": cores, "kind": "oracle",
               "sample": "%d full-parameter PBS of the workload on %d threads (%.1f s); cells/s = PBS/s / %d"
                         % (count, cores, dt, pbs_per_cell(cfg)),
               "pbs_per_s": pbs_s, "sample_bit_exact_vs_gpu": same,
               "sample_gpu_form": "k_blind_rotate (one CTA per ciphertext), as in the timed launches"}

    if rank == 0:
        line = {
            "metric": "encrypted DP cells/s",
            "value": value,
            "unit": "cells/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_max * 1e3 / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": desc, "pairs_per_gpu": len(pairs), "cells_per_gpu_step": cells,
                       "pbs_per_gpu_step": pbs_done // max(1, args.steps),
                       "params": "n=834 k=1 N=2048 pbs 2x2^13 ks 5x2^3 (TUniform 2^45 / 2^17)",
                       "l2": "inputs larger than L2 (server key 232 MB on device)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "pbs_per_s": pbs_all / t_max,
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tmodmul/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "kernel": "k_blind_rotate<11>",
                         "units_per_launch": units_per_launch, "launch_ms": avg_launch_s * 1e3,
                         "modmul_per_pbs": w_mod,
                         "peak_note": "%d SMs x %.1f modmul/SM/clk x max SM clock %.0f MHz; a Shoup modmul = 2 "
                                      "low + 1 high 32-bit multiplies at the measured issue rates (lo %.1f, hi %.1f "
                                      "per SM per clk, lvs_probe_int_mul)" % (
                                          n_sms, modmul_per_sm_clk, sm_mhz_max, mul_lo, mul_hi),
                         "frac_all_mul_at_lo_rate": (3 * w_mod * units_per_launch / avg_launch_s / 1e12 / peak_mul32)
                         if achieved else None,
                         "achievable": {
                             "shoup_products_per_sm_clk": shoup_stream,
                             "lazy_butterflies_per_sm_clk": bfly_stream,
                             "frac_of_butterfly_stream": (achieved / (n_sms * bfly_stream * sm_mhz_max * 1e6 / 1e12))
                             if achieved else None,
                             "note": "lvs_probe_modmul: register-resident streams of Shoup products and of complete "
                                     "lazy NTT butterflies (the kernel's form), one CTA per SM; what a kernel made "
                                     "of these operations can reach, below the multiply issue rates of the peak",
                             "key_product": {
                                 "wide_mac_per_sm_clk": wide_mac,
                                 "l2_read_bytes_per_sm_clk": l2_bytes_clk,
                                 "key_row_bytes": key_row_bytes(params),
                                 "key_row_l2_cycles": key_row_bytes(params) / l2_bytes_clk if l2_bytes_clk else None,
                                 "note": "lvs_probe_key_product: 32x32->64 multiply-accumulates and L2->SM reads in "
                                         "the key product's shape; one BSK row per CMux per SM read within the "
                                         "product costs at least key_row_l2_cycles SM cycles"}}},
            "kernels": {"blind_rotate": br, "keyswitch": ks,
                        "ks_plans": {"note": "launch size bucket end -> [PBS per CTA, split] (lvs_ctx_autotune)",
                                     "plans": ks_plans},
                        "br_three_cta_max_pbs": br_split,
                        "ks_tensor_core_min_pbs": ks_gemm_min},
            "latency_ms": {"p50": batched_latency_ms, "p99": batched_latency_ms,
                           "note": "the batch step time: all pairs of a step complete together (query "
                                   "latencies under continuous batching: serving)"},
            "serving": serving,
            "one_pair_at_a_time": serial,
            "table_build": table_build,
            "noise": noise,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "paper_context": PAPER_CONTEXT,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def encrypt_arrivals(L, ck, arrivals, seed=5):
    """Client side: every query (and encrypted reference) encrypted before the clock starts."""
    enc = []
    for k, (t, q, ref, plain) in enumerate(arrivals):
        qa = L.lvs_encrypt_string(ck, q, L.LVS_ALPHA_27, seed, 2 * k)
        rb = None if plain else L.lvs_encrypt_string(ck, ref, L.LVS_ALPHA_27, seed, 2 * k + 1)
        enc.append((qa, rb))
    return enc


def serve(L, server, arrivals, enc, idx=None):
    """Submits the queries `idx` (default: all) at their arrival times (seconds
    after the call) and polls until every one is done; returns {i: latency s}
    (completion - arrival) and {i: result}."""
    idx = list(range(len(arrivals))) if idx is None else list(idx)
    t0 = time.perf_counter()
    tickets, done_t, results = {}, {}, {}
    k = 0
    while len(done_t) < len(idx):
        now = time.perf_counter() - t0
        while k < len(idx) and arrivals[idx[k]][0] <= now:
            i = idx[k]
            qa, rb = enc[i]
            tickets[i] = L.lvs_server_submit(server, qa, ref_enc=rb) if rb is not None else \
                L.lvs_server_submit(server, qa, ref_plain=arrivals[i][2])
            k += 1
        for i, tk in tickets.items():
            if i not in done_t:
                r = L.lvs_server_poll(server, tk)
                if r is not None:
                    done_t[i] = time.perf_counter() - t0
                    results[i] = r
        time.sleep(0.001)
    return {i: done_t[i] - arrivals[i][0] for i in done_t}, results, time.perf_counter() - t0


def pct(lat, q):
    v = sorted(lat)
    return 1e3 * v[min(len(v) - 1, int(q * len(v)))]


def serving_segment(L, ctx, ck, rate, duration, slots, alone):
    """Continuous batching at a sustainable rate (config 5's generator), and a
    sample of the same queries run one at a time (each alone on the server:
    the plain one-pair-at-a-time GPU form on the same inputs)."""
    from paper_2508_14568_gb300 import workloads as W
    arrivals = W.config5(rate=rate, duration=duration)
    enc = encrypt_arrivals(L, ck, arrivals)
    server = L.lvs_server_create(ctx, 64 << 30, slots)
    lat, res, wall = serve(L, server, arrivals, enc)
    st = L.lvs_server_stats_get(server)
    ok = all(L.lvs_decrypt(ck, res[i], 0) == levenshtein(arrivals[i][1], arrivals[i][2]) for i in res)
    cells = sum(len(q) * len(ref) for _, q, ref, _ in arrivals)
    out = {"workload": "config 5 generator: Poisson %.1f queries/s for %.0f s, 27 symbols, lengths U[4,64], "
                       "plaintext/encrypted reference 50/50, %d slots" % (rate, duration, slots),
           "queries": len(arrivals), "latency_ms": {"p50": pct(lat.values(), 0.5), "p99": pct(lat.values(), 0.99),
                                                    "max": 1e3 * max(lat.values())},
           "cells_per_s": cells / wall, "pbs_per_s": st["pbs"] / wall, "gpu_busy_frac": st["busy_ms"] / 1e3 / wall,
           "all_distances_correct": ok, "note": "latency = completion - arrival, wall clock"}
    if alone > 0:
        sample = list(range(0, len(arrivals), max(1, len(arrivals) // alone)))[:alone]
        lat1 = []
        ok1 = True
        for i in sample:
            one = [(0.0,) + tuple(arrivals[i][1:])]
            l1, r1, _ = serve(L, server, one, [enc[i]])
            lat1.append(l1[0])
            ok1 &= L.lvs_decrypt(ck, r1[0], 0) == L.lvs_decrypt(ck, res[i], 0)
        out["one_at_a_time"] = {"queries": len(sample), "latency_ms": {"p50": pct(lat1, 0.5), "p99": pct(lat1, 0.99)},
                                "same_distances_as_in_the_mix": bool(ok1),
                                "note": "the same queries submitted one at a time, each alone on the server"}
    L.lvs_server_free(server)
    return out


def run_serving(args):
    """Config 5: Poisson arrivals of encrypted 27-symbol queries (length
    U[4,64]) against plaintext or encrypted references (U[4,64], 50/50) into the
    continuous-batching server; latency = completion - arrival."""
    import torch
    from paper_2508_14568_gb300 import lvs as L
    from paper_2508_14568_gb300 import workloads as W
    arrivals = W.config5(rate=args.rate, duration=args.duration)
    params = L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 0)
    ctx = L.lvs_ctx_create(sk, 0)
    enc = encrypt_arrivals(L, ck, arrivals)
    server = L.lvs_server_create(ctx, 64 << 30, args.slots)
    clocks = ClockSampler(0)
    clocks.start()
    lat, results, wall = serve(L, server, arrivals, enc)
    clk = clocks.stop()
    st = L.lvs_server_stats_get(server)
    ok = all(L.lvs_decrypt(ck, results[i], 0) == levenshtein(arrivals[i][1], arrivals[i][2]) for i in results)
    cells = sum(len(q) * len(ref) for _, q, ref, _ in arrivals)
    line = {"metric": "serving p50/p99 query latency", "config": {
                "workload": "config 5: Poisson %.1f queries/s for %.0f s, 27 symbols, lengths U[4,64], "
                            "plaintext/encrypted reference 50/50, budget 64 GB, %d slots" % (args.rate, args.duration, args.slots),
                "queries": len(arrivals)},
            "latency_ms": {"p50": pct(lat.values(), 0.5), "p99": pct(lat.values(), 0.99), "max": 1e3 * max(lat.values())},
            "cells_per_s": cells / wall, "pbs_per_s": st["pbs"] / wall, "wall_s": wall,
            "server": st, "all_distances_correct": ok, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_pbs_variants(args):
    """PBS/s of the blind-rotation variants (exact NTT with the key read from
    global memory, the same with the head of each key row staged by bulk copy,
    FP64 FFT) on one batch of independent PBS at the default parameters (inputs
    resident on the device, identity table), with a decryption check of every
    output and the staged outputs compared bit for bit with the default form."""
    import numpy as np
    import torch
    from paper_2508_14568_gb300 import lvs as L
    params = L.lvs_params_default()
    ck, sk = L.lvs_keygen(params, 0)
    stream = torch.cuda.Stream(device=0)
    torch.cuda.set_stream(stream)
    ctx = L.lvs_ctx_create(sk, 0, stream)
    L.lvs_ctx_prepare_fft64(ctx, sk)
    big = params.k * params.N
    count = args.pbs_variants
    msgs = np.arange(count) % 16
    cts = np.stack([L.lvs_encrypt_lwe(ck, int(m), 3, 0, i, big) for i, m in enumerate(msgs)])
    d_in = torch.from_numpy(cts.view(np.int64)).cuda()
    d_out = torch.zeros_like(d_in)
    luts = torch.from_numpy(np.tile(np.arange(16, dtype=np.uint8), (count, 1))).cuda()
    line = {"metric": "PBS/s by blind-rotation variant", "unit": "PBS/s", "count": count,
            "steps": args.steps, "warmup": args.warmup,
            "params": "n=834 k=1 N=2048 pbs 2x2^13 ks 5x2^3", "variants": {}}
    clocks = ClockSampler(0)
    clocks.start()
    def staged(*a):
        L.lvs_ctx_set_key_staging(ctx, True)
        try:
            L.lvs_pbs_batch_device(*a)
        finally:
            L.lvs_ctx_set_key_staging(ctx, False)

    ref = None
    for name, fn in (("ntt_exact", L.lvs_pbs_batch_device), ("ntt_exact_key_staged", staged),
                     ("fft64", L.lvs_pbs_batch_device_fft64)):
        for _ in range(max(1, args.warmup)):
            fn(ctx, d_in, big + 1, luts, d_out, big + 1, count)
        torch.cuda.synchronize()
        got = [L.lvs_decrypt_lwe(ck, r) for r in d_out.cpu().numpy().view(np.uint64)]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            fn(ctx, d_in, big + 1, luts, d_out, big + 1, count)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        out = d_out.cpu().numpy()
        line["variants"][name] = {"value": count / (ms * 1e-3), "ms_per_batch": ms,
                                  "decrypt_ok": bool(np.array_equal(np.array(got), msgs))}
        if name == "ntt_exact":
            ref = out
        elif name == "ntt_exact_key_staged":
            line["variants"][name]["bit_equal_to_ntt_exact"] = bool(np.array_equal(out, ref))
    line["clocks"] = clocks.stop()
    L.lvs_ctx_free(ctx)
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.pbs_variants:
        return run_pbs_variants(args)
    if args.config == 5:
        return run_serving(args)
    return run_lvs(args)


if __name__ == "__main__":
    sys.exit(main())
