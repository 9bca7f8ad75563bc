"""CPU TFHE oracle, Python side -- TEST INFRASTRUCTURE ONLY.

Loads ``tfhe_oracle.c`` (built with gcc into ``oracle/_build/``) and exposes
its primitives on numpy uint64 arrays, plus the encrypted Leuvenshtein driver
``lvs_encrypted`` that follows Algorithm algo_complete step by step (the loops
j = 1..n, i = 1..m; two equality lookups, the key of Eq. eq_keyeq2, one
LUT_min lookup and the two linear updates per cell).

Linear operations on ciphertexts (Section 2.2: addition, subtraction,
multiplication by a small integer, adding a plaintext constant) are written
out here on numpy uint64 vectors, which wrap mod 2^64 like the torus.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

from . import plain as P

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfhe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtfhe_oracle.so")
_lock = threading.Lock()
_lib = None

DELTA = 1 << 59          # 5-bit plaintext space: q / 32
U64 = np.uint64


class Params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in (
        "n", "k", "N", "pbs_level", "pbs_base_log", "ks_level", "ks_base_log",
        "lwe_noise_log2", "glwe_noise_log2")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def params_lvs():
    """The parameter set used for the paper's workloads (k=1, N=2048, n=834,
    two-level bootstrapping gadget with base 2^13, five-level key-switching
    gadget with base 2^3).  The paper does not print its numeric set."""
    return Params(n=834, k=1, N=2048, pbs_level=2, pbs_base_log=13, ks_level=5,
                  ks_base_log=3, lwe_noise_log2=45, glwe_noise_log2=17)


def params_test():
    """Small INSECURE set (n=64, N=512) with the same gadgets, for fast parity."""
    return Params(n=64, k=1, N=512, pbs_level=2, pbs_base_log=13, ks_level=5,
                  ks_base_log=3, lwe_noise_log2=45, glwe_noise_log2=17)


def build(force=False):
    """Compile tfhe_oracle.c with gcc (host code only, no nvcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-o", tmp,
                               _SRC, "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            pp = ctypes.POINTER(Params)
            L.orc_sm64.argtypes = [ctypes.c_uint64]
            L.orc_sm64.restype = ctypes.c_uint64
            L.orc_word.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_word.restype = ctypes.c_uint64
            L.orc_stream.argtypes = [ctypes.c_uint64] * 4
            L.orc_stream.restype = ctypes.c_uint64
            L.orc_tuniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            L.orc_tuniform.restype = ctypes.c_int64
            L.orc_negacyclic_mul.argtypes = [u64p, u64p, u64p, ctypes.c_uint32]
            L.orc_poly_rotate.argtypes = [u64p, ctypes.c_uint32, u64p, ctypes.c_uint32]
            L.orc_keygen.argtypes = [pp, ctypes.c_uint64, u64p, u64p, u64p, u64p]
            L.orc_lwe_encrypt.argtypes = [u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p]
            L.orc_lwe_phase.argtypes = [u64p, ctypes.c_uint32, u64p]
            L.orc_lwe_phase.restype = ctypes.c_uint64
            L.orc_lwe_decrypt.argtypes = [u64p, ctypes.c_uint32, u64p]
            L.orc_lwe_decrypt.restype = ctypes.c_uint32
            L.orc_decompose.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, i64p]
            L.orc_keyswitch.argtypes = [pp, u64p, u64p, u64p]
            L.orc_modswitch.argtypes = [pp, u64p, u32p]
            L.orc_lut_poly.argtypes = [pp, u32p, u64p]
            L.orc_blind_rotate.argtypes = [pp, u64p, u32p, u64p, u64p]
            L.orc_sample_extract.argtypes = [pp, u64p, u64p]
            L.orc_pbs.argtypes = [pp, u64p, u64p, u64p, u32p, u64p]
            L.orc_pbs_many.argtypes = [pp, u64p, u64p, ctypes.c_size_t, u64p, u32p, u64p, ctypes.c_int]
            L.orc_pbs_many.restype = ctypes.c_int
            _lib = L
    return _lib


def _p64(a):
    assert a.dtype == U64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _p32(a):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


# ---------------------------------------------------------------------------
# generator
# ---------------------------------------------------------------------------

def sm64(x):
    return int(lib().orc_sm64(x & (2**64 - 1)))


def word(key, c):
    return int(lib().orc_word(key, c))


def stream(seed, tag, i0, i1):
    return int(lib().orc_stream(seed, tag, i0, i1))


def tuniform(w, b):
    return int(lib().orc_tuniform(w, b))


# ---------------------------------------------------------------------------
# polynomials
# ---------------------------------------------------------------------------

def negacyclic_mul(a, b):
    a = np.ascontiguousarray(a, dtype=U64)
    b = np.ascontiguousarray(b, dtype=U64)
    out = np.zeros_like(a)
    lib().orc_negacyclic_mul(_p64(a), _p64(b), _p64(out), len(a))
    return out


def poly_rotate(a, r):
    a = np.ascontiguousarray(a, dtype=U64)
    out = np.zeros_like(a)
    lib().orc_poly_rotate(_p64(a), r, _p64(out), len(a))
    return out


def decompose(a, level, base_log):
    d = (ctypes.c_int64 * 64)()
    lib().orc_decompose(a, level, base_log, d)
    return [d[i] for i in range(level)]


# ---------------------------------------------------------------------------
# keys
# ---------------------------------------------------------------------------

class Keys:
    """Client key (lwe_key, glwe_key) and server key (bsk, ksk) from one seed."""

    def __init__(self, params, seed):
        p = params
        self.params = p
        self.seed = seed
        self.lwe_key = np.zeros(p.n, dtype=U64)
        self.glwe_key = np.zeros(p.k * p.N, dtype=U64)
        self.bsk = np.zeros(p.n * (p.k + 1) * p.pbs_level * (p.k + 1) * p.N, dtype=U64)
        self.ksk = np.zeros(p.k * p.N * p.ks_level * (p.n + 1), dtype=U64)
        lib().orc_keygen(ctypes.byref(p), seed, _p64(self.lwe_key), _p64(self.glwe_key),
                         _p64(self.bsk), _p64(self.ksk))

    @property
    def big_dim(self):
        return self.params.k * self.params.N


# ---------------------------------------------------------------------------
# LWE under the big key (dimension kN)
# ---------------------------------------------------------------------------

def encrypt(keys, mu_z32, noise_seed, i0, i1):
    """Fresh LWE encryption of a Z_32 value under the big key (stream (seed, ENC, i0, i1))."""
    d = keys.big_dim
    ct = np.zeros(d + 1, dtype=U64)
    mu = (int(mu_z32) % 32) * DELTA
    lib().orc_lwe_encrypt(_p64(keys.glwe_key), d, mu, keys.params.glwe_noise_log2,
                          noise_seed, i0, i1, _p64(ct))
    return ct


def phase(keys, ct):
    ct = np.ascontiguousarray(ct, dtype=U64)
    return int(lib().orc_lwe_phase(_p64(keys.glwe_key), keys.big_dim, _p64(ct)))


def decrypt(keys, ct):
    ct = np.ascontiguousarray(ct, dtype=U64)
    return int(lib().orc_lwe_decrypt(_p64(keys.glwe_key), keys.big_dim, _p64(ct)))


def decrypt_small(keys, ct):
    ct = np.ascontiguousarray(ct, dtype=U64)
    return int(lib().orc_lwe_decrypt(_p64(keys.lwe_key), keys.params.n, _p64(ct)))


def trivial(keys, mu_z32):
    """Noiseless ciphertext (0, mu * Delta) -- how OneMatrix and constants enter."""
    ct = np.zeros(keys.big_dim + 1, dtype=U64)
    ct[-1] = U64((int(mu_z32) % 32) * DELTA)
    return ct


def add_const(ct, mu_z32):
    out = ct.copy()
    out[-1] = U64((int(out[-1]) + (int(mu_z32) % 32) * DELTA) % 2**64)
    return out


def scalar(c, ct):
    """Multiply a ciphertext by a small integer (wrapping mod 2^64)."""
    return (U64(c % 2**64) * ct).astype(U64)


# ---------------------------------------------------------------------------
# PBS pieces
# ---------------------------------------------------------------------------

def keyswitch(keys, ct):
    p = keys.params
    ct = np.ascontiguousarray(ct, dtype=U64)
    out = np.zeros(p.n + 1, dtype=U64)
    lib().orc_keyswitch(ctypes.byref(p), _p64(keys.ksk), _p64(ct), _p64(out))
    return out


def modswitch(keys, small):
    p = keys.params
    small = np.ascontiguousarray(small, dtype=U64)
    out = np.zeros(p.n + 1, dtype=np.uint32)
    lib().orc_modswitch(ctypes.byref(p), _p64(small), _p32(out))
    return out


def lut_poly(keys, f16):
    p = keys.params
    f = np.ascontiguousarray([x % 32 for x in f16], dtype=np.uint32)
    v = np.zeros(p.N, dtype=U64)
    lib().orc_lut_poly(ctypes.byref(p), _p32(f), _p64(v))
    return v


def blind_rotate(keys, ms, v):
    p = keys.params
    ms = np.ascontiguousarray(ms, dtype=np.uint32)
    acc = np.zeros((p.k + 1) * p.N, dtype=U64)
    lib().orc_blind_rotate(ctypes.byref(p), _p64(keys.bsk), _p32(ms),
                           _p64(np.ascontiguousarray(v, dtype=U64)), _p64(acc))
    return acc


def sample_extract(keys, acc):
    p = keys.params
    out = np.zeros(keys.big_dim + 1, dtype=U64)
    lib().orc_sample_extract(ctypes.byref(p), _p64(np.ascontiguousarray(acc, dtype=U64)), _p64(out))
    return out


def pbs(keys, ct, f16):
    p = keys.params
    ct = np.ascontiguousarray(ct, dtype=U64)
    f = np.ascontiguousarray([x % 32 for x in f16], dtype=np.uint32)
    out = np.zeros(keys.big_dim + 1, dtype=U64)
    lib().orc_pbs(ctypes.byref(p), _p64(keys.ksk), _p64(keys.bsk), _p64(ct), _p32(f), _p64(out))
    return out


def pbs_many(keys, cts, luts, nthreads=None):
    """Independent PBS over host threads.  cts: (count, kN+1); luts: (count, 16)."""
    p = keys.params
    cts = np.ascontiguousarray(cts, dtype=U64)
    f = np.ascontiguousarray(np.asarray(luts) % 32, dtype=np.uint32)
    count = cts.shape[0]
    out = np.zeros_like(cts)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    nthreads = max(1, min(nthreads, count))
    lib().orc_pbs_many(ctypes.byref(p), _p64(keys.ksk), _p64(keys.bsk), count, _p64(cts),
                       _p32(f), _p64(out), nthreads)
    return out


# ---------------------------------------------------------------------------
# strings and the encrypted Leuvenshtein run (Algorithm algo_complete)
# ---------------------------------------------------------------------------

def encrypt_string(keys, s, alphabet, noise_seed, string_id):
    """Each character -> its symbols (Section 4.3 split, or one DNA symbol),
    each symbol one fresh LWE under the big key, noise stream
    (noise_seed, ENC, string_id, 2 * char_index + symbol)."""
    out = []
    for ci, c in enumerate(s):
        syms = P.split_symbol(P.symbol_index(c, alphabet), alphabet)
        out.append([encrypt(keys, v, noise_seed, string_id, 2 * ci + si) for si, v in enumerate(syms)])
    return out


def lvs_encrypted(keys, xa, yb, alphabet, parallel=False, band=None, refresh=()):
    """Algorithm algo_complete on ciphertexts (with ``band``: only the cells
    inside plain.in_band -- |i - j| <= band for m = n, the condition of
    Algorithm alg_levenshtein; the others keep the OneMatrix value 1).

    ``refresh``: anti-diagonals d = i + j whose dv, dh are refreshed by a
    bootstrap (Section 3.1.3): such a cell takes two lookups through LUT_V,
    v[i][j] = PBS(key; LUT_V) and h[i][j] = PBS(key'; LUT_V) with the swapped
    key' = (1 - h[i-1][j]) + 3 (1 + v[i][j-1]) + eq9, instead of M.

    xa, yb: lists (per character) of lists (per symbol) of ciphertexts.

    With ``parallel=False`` the steps run exactly in the paper's order: for
    j = 1..n, for i = 1..m: z1 = x1_i - y1_j, eq1 = PBS(z1; LUT_EQ),
    z2 = 2 (x2_i - y2_j) + (1 - eq1), eq9 = PBS(z2; LUT_EQ9) (DNA: one
    lookup on x_i - y_j), key = (1 - v[i][j-1]) + 3 (1 + h[i-1][j]) + eq9,
    M = PBS(key; LUT_min), v[i][j] = M - h[i-1][j], h[i][j] = M - v[i][j-1].

    With ``parallel=True`` the same lookups, on the same inputs, are handed to
    host threads in groups that do not depend on each other (all equality
    lookups, then one anti-diagonal i + j = const at a time, the independence
    the paper points out in Section 6.2 "Parallelism").  A test checks that
    both orders give identical ciphertexts.

    Returns a dict with the PBS outputs per cell ('eq1', 'eq9', 'M'), the
    final row h[m][1..n] ('h_row'), the final column v[1..m][n] ('v_col'),
    for square pairs the diagonal path [v[1][0], h[1][1], ..., v[m][m-1],
    h[m][m]] ('diag', the readout of Section 3.2), the band readout path of
    plain.readout_path_cells ('path') and the number of PBS.
    """
    m, n = len(xa), len(yb)
    one = trivial(keys, 1)
    h = {(0, j): one for j in range(n + 1)}
    v = {(i, 0): one for i in range(m + 1)}
    res = {"eq1": {}, "eq9": {}, "M": {}}
    dna = alphabet == P.ALPHA_DNA4
    npbs = 0

    def z_first(i, j):
        return xa[i - 1][0] - yb[j - 1][0]

    def z_second(i, j, e1):
        return scalar(2, xa[i - 1][1] - yb[j - 1][1]) + (one - e1)

    def inside(i, j):
        return P.in_band(i, j, m, n, band)

    def key_of(i, j):
        return (one - v.get((i, j - 1), one)) + scalar(3, one + h.get((i - 1, j), one)) + res["eq9"][(i, j)]

    def key_swapped(i, j):
        return (one - h.get((i - 1, j), one)) + scalar(3, one + v.get((i, j - 1), one)) + res["eq9"][(i, j)]

    def update(i, j, M):
        res["M"][(i, j)] = M
        v[(i, j)] = M - h.get((i - 1, j), one)
        h[(i, j)] = M - v.get((i, j - 1), one)

    if not parallel:
        for j in range(1, n + 1):
            for i in range(1, m + 1):
                if not inside(i, j):
                    continue
                if dna:
                    res["eq9"][(i, j)] = pbs(keys, z_first(i, j), P.LUT_EQ9)
                    npbs += 1
                else:
                    e1 = pbs(keys, z_first(i, j), P.LUT_EQ)
                    res["eq1"][(i, j)] = e1
                    res["eq9"][(i, j)] = pbs(keys, z_second(i, j, e1), P.LUT_EQ9)
                    npbs += 2
                if i + j in refresh:
                    nv = pbs(keys, key_of(i, j), P.LUT_V)
                    nh = pbs(keys, key_swapped(i, j), P.LUT_V)
                    v[(i, j)], h[(i, j)] = nv, nh
                    npbs += 2
                    continue
                update(i, j, pbs(keys, key_of(i, j), P.LUT_MIN))
                npbs += 1
    else:
        cells = [(i, j) for j in range(1, n + 1) for i in range(1, m + 1) if inside(i, j)]
        if dna:
            e9 = _pbs_list(keys, [z_first(i, j) for (i, j) in cells], P.LUT_EQ9)
            npbs += len(cells)
        else:
            e1 = _pbs_list(keys, [z_first(i, j) for (i, j) in cells], P.LUT_EQ)
            for c, e in zip(cells, e1):
                res["eq1"][c] = e
            e9 = _pbs_list(keys, [z_second(i, j, e) for (i, j), e in zip(cells, e1)], P.LUT_EQ9)
            npbs += 2 * len(cells)
        for c, e in zip(cells, e9):
            res["eq9"][c] = e
        for d in range(2, m + n + 1):
            diag = [(i, d - i) for i in range(max(1, d - n), min(m, d - 1) + 1) if inside(i, d - i)]
            if d in refresh:
                nvs = _pbs_list(keys, [key_of(i, j) for (i, j) in diag], P.LUT_V)
                nhs = _pbs_list(keys, [key_swapped(i, j) for (i, j) in diag], P.LUT_V)
                npbs += 2 * len(diag)
                for c, nv, nh in zip(diag, nvs, nhs):
                    v[c], h[c] = nv, nh
                continue
            Ms = _pbs_list(keys, [key_of(i, j) for (i, j) in diag], P.LUT_MIN)
            npbs += len(diag)
            for (i, j), M in zip(diag, Ms):
                update(i, j, M)
    res["h_row"] = [h.get((m, j), one) for j in range(1, n + 1)]
    res["v_col"] = [v.get((i, n), one) for i in range(1, m + 1)]
    if m == n:
        res["diag"] = [c for i in range(1, m + 1) for c in (v.get((i, i - 1), one), h.get((i, i), one))]
    res["path"] = [(v if s == "v" else h).get((i, j), one) for i, j, s in P.readout_path_cells(m, n)]
    res["pbs"] = npbs
    return res


def _pbs_list(keys, cts, lut):
    if not cts:
        return []
    arr = np.stack([np.asarray(c, dtype=U64) for c in cts])
    luts = np.tile(np.asarray(lut, dtype=np.uint32), (len(cts), 1))
    out = pbs_many(keys, arr, luts)
    return [out[i] for i in range(len(cts))]


def decrypt_path(keys, cts, base=0):
    """base + the decrypted differences along a path of the matrix."""
    return base + sum(P.signed(decrypt(keys, c)) for c in cts)


def readout_sum(keys, cts, base):
    """The return of Algorithm algo_complete on ciphertexts: base (trivially
    encrypted) + the sum of the difference ciphertexts, word by word mod 2^64.
    It decrypts to the distance while that stays below 16 (5-bit plaintext
    with its padding bit)."""
    out = [0] * (keys.big_dim + 1)
    for c in cts:
        for t in range(keys.big_dim + 1):
            out[t] = (out[t] + int(c[t])) % 2**64
    out[-1] = (out[-1] + (int(base) % 32) * DELTA) % 2**64
    return np.asarray(out, dtype=U64)


def decrypt_distance(keys, h_row, m):
    """m + sum_j h[m][j], each h decrypted to {-1, 0, 1} (readout of Section 3.2
    with the boundary term taken once)."""
    return m + sum(P.signed(decrypt(keys, c)) for c in h_row)
