"""Noise accounting of the Leuvenshtein DP -- TEST INFRASTRUCTURE ONLY.

Section 3.1.3 ("Limiting the noise growth") counts the noise of the key of
Eq. eq_keyeq2 in units of eps^2_PBS, the variance of one fresh bootstrap
output: every M_ij and every EQ9 is an independent unit, dv and dh are
linear combinations of them (dv_out = M - dh_in, dh_out = M - dv_in), and the
key (1 - dv_in) + 3 (1 + dh_in) + EQ9 has variance sum(coefficient^2).  When a
key would exceed the noise budget, the dv and dh of an earlier anti-diagonal
are refreshed by a bootstrap, which makes them fresh independent units.

- key_variances: the exact linear-combination tracker (the definition).
- key_variance_closed_form: the full-matrix closed form worked out from the
  recursion of Section 3.1.3 (the N_H + 4 N_M + 9 N_L + 1 count).
- refresh_schedule: greedy choice of the anti-diagonals to refresh.
- noise_budget: the largest key variance (in eps^2_PBS units) for which a
  bootstrap fails with probability <= 2^log2_pfail, from the variances of the
  PBS output, the key switch and the modulus switch (Section 2.2).
"""
import math

from .plain import in_band


class _Tracker:
    """Linear combinations over independent unit-variance noises."""

    def __init__(self):
        self.next = 0

    def unit(self):
        self.next += 1
        return {self.next: 1}

    @staticmethod
    def lin(*terms):
        out = {}
        for c, x in terms:
            for u, a in x.items():
                out[u] = out.get(u, 0) + c * a
        return {u: a for u, a in out.items() if a}

    @staticmethod
    def var(x):
        return sum(a * a for a in x.values())


def _track(m, n, band, refresh):
    T = _Tracker()
    zero = {}
    v = {}   # (i, j) -> noise of v[i][j]
    h = {}
    keys = {}
    for d in range(2, m + n + 1):
        for i in range(max(1, d - n), min(m, d - 1) + 1):
            j = d - i
            if not in_band(i, j, m, n, band):
                continue
            dv_in = v.get((i, j - 1), zero)
            dh_in = h.get((i - 1, j), zero)
            eq9 = T.unit()
            key = T.lin((-1, dv_in), (3, dh_in), (1, eq9))
            key_sw = T.lin((3, dv_in), (-1, dh_in), (1, eq9))
            keys[(i, j)] = (T.var(key), T.var(key_sw))
            if d in refresh:
                v[(i, j)] = T.unit()
                h[(i, j)] = T.unit()
            else:
                M = T.unit()
                v[(i, j)] = T.lin((1, M), (-1, dh_in))
                h[(i, j)] = T.lin((1, M), (-1, dv_in))
    return keys, v, h


def key_variances(m, n, band=None, refresh=frozenset()):
    """Variances (eps^2_PBS units) of the key of every computed cell (i, j)
    and of its swapped key (1 - dh_in) + 3 (1 + dv_in) + EQ9, which a
    refreshed cell bootstraps for dh_out.

    Boundary values (v[i][0], h[0][j]) and cells outside the band keep the
    plaintext OneMatrix value 1 and carry no noise.  A cell on a refreshed
    anti-diagonal d = i + j outputs fresh dv, dh.  Returns
    {(i, j): (var_key, var_swapped_key)}."""
    return _track(m, n, band, refresh)[0]


def output_variances(m, n, band=None, refresh=frozenset()):
    """Variances (eps^2_PBS units) of the outputs v[i][j], h[i][j] of every
    computed cell: {(i, j): (var_v, var_h)}."""
    _, v, h = _track(m, n, band, refresh)
    return {c: (_Tracker.var(v[c]), _Tracker.var(h[c])) for c in v}


def key_variance_closed_form(i, j):
    """Full matrix, no refresh: each step back along the diagonal adds
    M_{i,j-1} (1), 3 M_{i-1,j} (9) and -2 M_{i-1,j-1} (4), i.e. 14 per step,
    ended by the boundary term (1 on the main diagonal, 10 below, 2 above)."""
    c = 1 if i == j else (10 if i > j else 2)
    return 14 * (min(i, j) - 1) + c


def refresh_schedule(m, n, band=None, budget=None):
    """Anti-diagonals to refresh so that every key stays <= budget.

    A cell costs the larger of its key's and its swapped key's variance (the
    swapped key is bootstrapped only if the cell is refreshed; counting it
    everywhere keeps the choice simple).  Greedy, as late as possible:
    diagonal d is refreshed when, with d not refreshed, some cell of diagonal
    d + 1 would cost more than the budget.  Raises
    ValueError when even a refresh of the previous diagonal cannot keep a key
    within the budget.  budget None: no refresh.  Returns (sorted list of
    refreshed diagonals, max key variance)."""
    if budget is None:
        return [], _worst(key_variances(m, n, band))
    chosen = set()
    for d in range(2, m + n):
        nxt = _diag_max(m, n, band, chosen, d + 1)
        if nxt > budget:
            chosen.add(d)
            if _diag_max(m, n, band, chosen, d + 1) > budget:
                raise ValueError("noise budget too small")
    worst = _worst(key_variances(m, n, band, frozenset(chosen)))
    if worst > budget:
        raise ValueError("noise budget too small")
    return sorted(chosen), worst


def _worst(var):
    return max((max(x) for x in var.values()), default=0)


def _diag_max(m, n, band, refresh, d):
    var = key_variances(m, n, band, frozenset(refresh))
    return max((max(x) for (i, j), x in var.items() if i + j == d), default=0)


# ---------------------------------------------------------------------------
# variances of one bootstrap (Section 2.2), torus Z_2^64, binary keys of
# expected weight half their length
# ---------------------------------------------------------------------------

def tuniform_variance(b):
    """TUniform(b): values in [-2^b, 2^b], the ends with half weight."""
    return (2.0 ** (2 * b + 1) + 1) / 6.0


def balanced_digit_sq(base_log):
    """E[d^2] of a balanced digit uniform on [-B/2, B/2)."""
    B = 2.0 ** base_log
    return (B * B + 2) / 12.0


def var_pbs(p, weight_lwe=None, weight_glwe=None):
    """Output of the blind rotation + sample extract: gadget rounding of
    X^a ACC - ACC in each CMux whose LWE key bit is set (weight_lwe of them,
    expected n/2), seen through the body and the GLWE key (1 + weight_glwe
    set coefficients, expected kN/2), plus the BSK noise of every CMux."""
    beta = p["pbs_level"] * p["pbs_base_log"]
    rounding = (2.0 ** (63 - beta)) ** 2 / 3.0
    w_lwe = p["n"] / 2.0 if weight_lwe is None else float(weight_lwe)
    w_glwe = p["k"] * p["N"] / 2.0 if weight_glwe is None else float(weight_glwe)
    weight = w_lwe * (1.0 + w_glwe)
    bsk = (p["n"] * (p["k"] + 1) * p["pbs_level"] * p["N"] * balanced_digit_sq(p["pbs_base_log"])
           * tuniform_variance(p["glwe_noise_log2"]))
    return weight * rounding + bsk


def var_keyswitch(p, weight=None):
    """Key switch of a big ciphertext: decomposition rounding (weight = set
    bits of the big key, expected kN/2) plus kN * level KSK rows, each with a
    balanced digit."""
    beta = p["ks_level"] * p["ks_base_log"]
    big = p["k"] * p["N"]
    w = big / 2.0 if weight is None else float(weight)
    rounding = w * (2.0 ** (63 - beta)) ** 2 / 3.0
    ksk = big * p["ks_level"] * balanced_digit_sq(p["ks_base_log"]) * tuniform_variance(p["lwe_noise_log2"])
    return rounding + ksk


def var_modswitch(p, weight=None):
    """Rounding of the n mask values and the body to multiples of 2^64/(2N)
    (weight = set bits of the LWE key, expected n/2)."""
    step = 2.0 ** 64 / (2 * p["N"])
    w = p["n"] / 2.0 if weight is None else float(weight)
    return (1 + w) * step * step / 12.0


def z_for_pfail(log2_pfail):
    """z with P(|X| > z sigma) = 2^log2_pfail for a normal X (bisection)."""
    target = 2.0 ** log2_pfail
    lo, hi = 0.0, 40.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid / math.sqrt(2.0)) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def noise_budget(p, log2_pfail=-64.0):
    """Largest key variance, in units of var_pbs, for which the bootstrap of the
    key (plus key-switch and modulus-switch noise) decodes wrongly with
    probability <= 2^log2_pfail: the error must stay below half a plaintext
    step, 2^58."""
    z = z_for_pfail(log2_pfail)
    room = (2.0 ** 58 / z) ** 2 - var_keyswitch(p) - var_modswitch(p)
    return room / var_pbs(p)


def pfail_of(p, key_var_units):
    """Failure probability of one bootstrap whose key has variance
    key_var_units * var_pbs (plus the key-switch and modulus-switch noise)."""
    s = math.sqrt(key_var_units * var_pbs(p) + var_keyswitch(p) + var_modswitch(p))
    return math.erfc(2.0 ** 58 / s / math.sqrt(2.0))
