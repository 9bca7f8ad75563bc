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


def _ntt_mults(N, p=97 * 2**20 + 1):
    """Modular multiplications of an explicit radix-2 negacyclic NTT of size N
    (Cooley-Tukey, one twiddle product per butterfly), checked against the
    transform's definition on a random input."""
    import random as _r
    rng = _r.Random(N)
    # psi: a primitive 2N-th root of unity mod p (p = 1 mod 2N)
    g = next(x for x in range(2, p) if pow(x, (p - 1) // 2, p) != 1)
    psi = pow(g, (p - 1) // (2 * N), p)
    a = [rng.randrange(p) for _ in range(N)]
    want = [sum(a[j] * pow(psi, (2 * i + 1) * j, p) for j in range(N)) % p for i in range(N)]
    x = [a[j] * pow(psi, j, p) % p for j in range(N)]      # pre-twist (folded into twiddles on the GPU)
    count = 0
    half = N // 2
    while half >= 1:                                        # decimation in frequency
        w = pow(psi, 2 * N // (2 * half), p)
        for start in range(0, N, 2 * half):
            for t in range(half):
                u, v = x[start + t], x[start + t + half]
                x[start + t] = (u + v) % p
                x[start + t + half] = (u - v) * pow(w, t, p) % p
                count += 1
        half //= 2
    bits = N.bit_length() - 1
    got = [x[int(format(i, "0%db" % bits)[::-1], 2)] for i in range(N)]
    assert got == want
    return count


def test_roofline_work_count():
    """The roofline's algorithmic work per PBS (n CMux; per CMux and prime:
    (k+1) l forward and (k+1) inverse transforms, (k+1)^2 l N key products)
    counted from an explicit transform, at both parameter sets."""
    import bench
    from oracle import tfhe as T
    per_ntt = {N: _ntt_mults(N) for N in (16, 32)}
    assert per_ntt == {16: 32, 32: 80}                      # (N/2) log2 N
    for p in (T.params_lvs(), T.params_test()):
        k, l, N, n = p.k, p.pbs_level, p.N, p.n
        per_transform = (N // 2) * (N.bit_length() - 1)
        per_cmux_prime = ((k + 1) * l + (k + 1)) * per_transform + (k + 1) ** 2 * l * N
        assert bench.modmul_per_pbs(p) == n * 3 * per_cmux_prime
    assert bench.modmul_per_pbs(T.params_lvs()) == 210_087_936                 # 834 x 3 x 83,968


def test_key_row_bytes():
    """Bytes of one NTT-domain bootstrapping-key row, the unit of the key
    product's L2 reads: 3 primes x (k+1)^2 l polynomials x N residues of 4
    bytes; n rows make the whole device key (164 MB at the default set)."""
    import bench
    from oracle import tfhe as T
    p = T.params_lvs()
    assert bench.key_row_bytes(p) == 3 * 2 * 2 * 2 * 2048 * 4 == 196_608
    assert p.n * bench.key_row_bytes(p) == 163_971_072
    q = T.params_test()
    assert bench.key_row_bytes(q) == 3 * (q.k + 1) ** 2 * q.pbs_level * q.N * 4
