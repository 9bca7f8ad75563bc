"""The bench's own distance check agrees with the oracle's Wagner-Fischer
(the bench uses the oracle only for its CPU baseline)."""
import random

from oracle import plain as P


def test_bench_levenshtein_equals_oracle():
    import bench
    rng = random.Random(3)
    for _ in range(500):
        a = "".join(rng.choice("abcd") for _ in range(rng.randint(0, 9)))
        b = "".join(rng.choice("abcd") for _ in range(rng.randint(0, 9)))
        assert bench.levenshtein(a, b) == P.wf_distance(a, b)
