"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws strings.  The
paper's name lists and DNA data are not available, so these recipes stand in
for them (the lengths follow Section 6: ASCII strings of 4..32 characters
for names, DNA of length up to 256; the recipes are stated per function).
All randomness comes from ``random.Random(seed)`` with the seeds below.
"""
import random

PRINTABLE = [chr(c) for c in range(0x20, 0x7F)]
ALPHA27 = [chr(c) for c in range(ord("A"), ord("Z") + 1)] + [" "]
DNA = list("ACGT")

SEED_BASE = 1000


def _rand_string(rng, pool, lo, hi):
    return "".join(rng.choice(pool) for _ in range(rng.randint(lo, hi)))


def mutate_edits(rng, s, pool, k):
    """k random edits (insert / delete / substitute equally likely, random
    position and character)."""
    s = list(s)
    for _ in range(k):
        op = rng.randrange(3)
        if op == 0 or not s:
            s.insert(rng.randint(0, len(s)), rng.choice(pool))
        elif op == 1:
            del s[rng.randrange(len(s))]
        else:
            s[rng.randrange(len(s))] = rng.choice(pool)
    return "".join(s)


def mutate_rate(rng, s, pool, rate):
    """Per-position mutation with probability ``rate``; the mutation type is
    uniform over substitution, insertion (before the position) and deletion."""
    out = []
    for c in s:
        if rng.random() < rate:
            op = rng.randrange(3)
            if op == 0:
                out.append(rng.choice([x for x in pool if x != c] or pool))
            elif op == 1:
                out.append(rng.choice(pool))
                out.append(c)
            # op == 2: deletion
        else:
            out.append(c)
    return "".join(out)


def config1(seed=SEED_BASE + 1):
    """One pair of printable-ASCII strings (bytes 0x20..0x7E uniform), lengths 4 and 4."""
    rng = random.Random(seed)
    return [(_rand_string(rng, PRINTABLE, 4, 4), _rand_string(rng, PRINTABLE, 4, 4))]


def config2(seed=SEED_BASE + 2, pairs=256):
    """Batching: lengths uniform in [8, 16] independently per string, printable
    ASCII; 30% of pairs are (a, a with 1..3 random edits)."""
    rng = random.Random(seed)
    out = []
    for _ in range(pairs):
        a = _rand_string(rng, PRINTABLE, 8, 16)
        if rng.random() < 0.30:
            b = mutate_edits(rng, a, PRINTABLE, rng.randint(1, 3))
        else:
            b = _rand_string(rng, PRINTABLE, 8, 16)
        out.append((a, b))
    return out


def config3(seed=SEED_BASE + 3, queries=1024):
    """Preprocessed path: encrypted client strings of length [8, 32] over the
    27-symbol alphabet (A..Z and space) against plaintext server strings of
    length [8, 32] over the same alphabet."""
    rng = random.Random(seed)
    return [(_rand_string(rng, ALPHA27, 8, 32), _rand_string(rng, ALPHA27, 8, 32)) for _ in range(queries)]


def config4(seed=SEED_BASE + 4, pairs=64, lo=64, hi=256):
    """DNA-like batch: first sequence uniform over ACGT with length [64, 256];
    second derived at 10% per-position mutation (equal mix of substitution,
    insertion, deletion)."""
    rng = random.Random(seed)
    out = []
    for _ in range(pairs):
        a = _rand_string(rng, DNA, lo, hi)
        out.append((a, mutate_rate(rng, a, DNA, 0.10)))
    return out


def config5(seed=SEED_BASE + 5, rate=200.0, duration=60.0):
    """Serving: Poisson arrivals at ``rate`` per second for ``duration``
    seconds; each query an encrypted 27-symbol string of length [4, 64] against
    a reference of length [4, 64] that is plaintext or encrypted (50/50).
    Returns a list of (arrival_time_s, query, reference, reference_is_plain)."""
    rng = random.Random(seed)
    t, out = 0.0, []
    while True:
        t += rng.expovariate(rate)
        if t >= duration:
            break
        out.append((t, _rand_string(rng, ALPHA27, 4, 64), _rand_string(rng, ALPHA27, 4, 64), rng.random() < 0.5))
    return out


def random_pairs(seed, count, pool, lo, hi):
    """Generic pairs for tests: independent lengths in [lo, hi] (lo may be 0)."""
    rng = random.Random(seed)
    return [(_rand_string(rng, pool, lo, hi), _rand_string(rng, pool, lo, hi)) for _ in range(count)]
