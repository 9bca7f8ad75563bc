"""Thin ctypes binding of the C ABI in include/lvs.h (argument marshalling only).

Every function keeps the C name.  Handles are wrapped in small Python objects
that call the matching ``lvs_*_free`` when collected.  Errors raise
``LvsError`` with the library's message.  Device buffers may be passed as
integers (device pointers) or as torch CUDA tensors (their ``data_ptr()``).

The CUDA library is required: importing this module fails loudly if the
shared library cannot be loaded, and compute calls fail with LVS_ERR_CUDA when
no GPU is present.  There is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblvs.so")

LVS_OK, LVS_ERR_ARG, LVS_ERR_OOM, LVS_ERR_CUDA, LVS_ERR_TIMEOUT, LVS_ERR_NOISE_BUDGET, LVS_ERR_STATE = range(7)
LVS_ALPHA_ASCII7, LVS_ALPHA_27, LVS_ALPHA_DNA4 = 0, 1, 2
STATUS_NAMES = ["LVS_OK", "LVS_ERR_ARG", "LVS_ERR_OOM", "LVS_ERR_CUDA", "LVS_ERR_TIMEOUT",
                "LVS_ERR_NOISE_BUDGET", "LVS_ERR_STATE"]

# exported entry points (checked by tests against include/lvs.h)
EXPORTS = [
    "lvs_last_error", "lvs_version", "lvs_params_default", "lvs_params_test", "lvs_opts_default",
    "lvs_keygen", "lvs_client_key_free", "lvs_server_key_free", "lvs_client_key_export",
    "lvs_server_key_export", "lvs_server_key_params", "lvs_server_key_import", "lvs_client_key_import",
    "lvs_decrypt_distance",
    "lvs_ctx_create", "lvs_ctx_free",
    "lvs_ctx_synchronize", "lvs_encrypt_string", "lvs_ct_string_free", "lvs_ct_string_info",
    "lvs_ct_string_export", "lvs_ct_string_import", "lvs_decrypt_lwe", "lvs_encrypt_lwe", "lvs_eq",
    "lvs_edit_distance_batch", "lvs_preprocess", "lvs_eq_table_free",
    "lvs_edit_distance_preprocessed_batch", "lvs_result_info", "lvs_result_export", "lvs_result_free",
    "lvs_result_sum", "lvs_plan_pair", "lvs_plan_table", "lvs_ctx_max_launch_jobs", "lvs_ctx_set_max_launch_jobs",
    "lvs_decrypt", "lvs_decrypt_all", "lvs_pbs_batch_device", "lvs_keyswitch_batch_device",
    "lvs_poly_mul_device", "lvs_ctx_set_timing", "lvs_ctx_kernel_stats", "lvs_ctx_pbs_count",
    "lvs_ctx_launch_count", "lvs_ct_string_upload", "lvs_pbs_batch_device_noalloc",
    "lvs_ctx_prepare_fft64", "lvs_pbs_batch_device_fft64", "lvs_noise_budget", "lvs_noise_plan",
    "lvs_ctx_autotune", "lvs_ctx_ks_plan", "lvs_ctx_set_ks_plan", "lvs_probe_int_mul", "lvs_probe_modmul",
    "lvs_probe_key_product", "lvs_ctx_set_key_staging", "lvs_ctx_key_staging", "lvs_debug_drop_key_copy",
    "lvs_preprocess_batch",
    "lvs_ct_string_pin", "lvs_ctx_br_split", "lvs_ctx_set_br_split", "lvs_ctx_set_wave_fill", "lvs_ctx_wave_fill",
    "lvs_plan_batch",
    "lvs_noise_pfail", "lvs_debug_fail_allocations", "lvs_ctx_ks_gemm_min", "lvs_ctx_set_ks_gemm_min",
    "lvs_server_create", "lvs_server_submit", "lvs_server_poll", "lvs_server_stats_get", "lvs_server_free",
]


class LvsError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


class lvs_params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in (
        "n", "k", "N", "pbs_level", "pbs_base_log", "ks_level", "ks_base_log",
        "lwe_noise_log2", "glwe_noise_log2")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lvs_opts(ctypes.Structure):
    _fields_ = [("band", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("refresh_budget", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class lvs_query(ctypes.Structure):
    _fields_ = [("query", ctypes.c_void_p), ("ref_enc", ctypes.c_void_p), ("ref_plain", ctypes.c_char_p),
                ("ref_plain_len", ctypes.c_size_t)]


class lvs_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "admitted", "completed", "pending", "active", "steps",
                                               "pbs", "max_step_pbs", "mem_in_use")] + [("busy_ms", ctypes.c_double),
                                                                                        ("requeued", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lvs_plan_layout(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("a", "b", "v", "h", "path", "eq1", "eq9", "table", "rows", "steps")]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lvs_plan_job(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("src", ctypes.c_int64 * 3), ("coef", ctypes.c_int64 * 3),
                ("cst", ctypes.c_int64), ("dst", ctypes.c_int64 * 2), ("tap", ctypes.c_int64),
                ("lut", ctypes.c_int32), ("kind", ctypes.c_int32), ("tapsel", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class lvs_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("items", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


_lib = None


def lib():
    """Loads liblvs.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        from . import build as _b
        if not _b.up_to_date():
            _b.build()
        _lib = ctypes.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


def _declare(L):
    vp, u64, u32, sz, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
    vpp = ctypes.POINTER(ctypes.c_void_p)
    u64p, u32p, szp = ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(sz)
    P = ctypes.POINTER(lvs_params)
    sig = {
        "lvs_last_error": ([], ctypes.c_char_p),
        "lvs_version": ([], ctypes.c_char_p),
        "lvs_params_default": ([P], None),
        "lvs_params_test": ([P], None),
        "lvs_opts_default": ([ctypes.POINTER(lvs_opts)], None),
        "lvs_keygen": ([P, u64, vpp, vpp], i32),
        "lvs_client_key_free": ([vp], None),
        "lvs_server_key_free": ([vp], None),
        "lvs_client_key_export": ([vp, u64p, szp, u64p, szp], i32),
        "lvs_server_key_export": ([vp, u64p, szp, u64p, szp], i32),
        "lvs_server_key_import": ([ctypes.POINTER(lvs_params), u64p, sz, u64p, sz, vpp], i32),
        "lvs_client_key_import": ([ctypes.POINTER(lvs_params), u64p, sz, u64p, sz, vpp], i32),
        "lvs_server_key_params": ([vp, P], i32),
        "lvs_ctx_create": ([vp, i32, vp, vpp], i32),
        "lvs_ctx_free": ([vp], None),
        "lvs_ctx_synchronize": ([vp], i32),
        "lvs_encrypt_string": ([vp, ctypes.c_char_p, sz, i32, u64, u64, vpp], i32),
        "lvs_ct_string_free": ([vp], None),
        "lvs_ct_string_info": ([vp, szp, u32p, u32p, ctypes.POINTER(i32)], i32),
        "lvs_ct_string_export": ([vp, u64p, szp], i32),
        "lvs_ct_string_import": ([u64p, sz, i32, u32, vpp], i32),
        "lvs_decrypt_lwe": ([vp, u64p, u32p], i32),
        "lvs_encrypt_lwe": ([vp, u32, u64, u64, u64, u64p], i32),
        "lvs_eq": ([vp, vp, sz, vp, sz, i32, vpp], i32),
        "lvs_edit_distance_batch": ([vp, vpp, vpp, sz, ctypes.POINTER(lvs_opts), vpp], i32),
        "lvs_preprocess": ([vp, vp, ctypes.c_char_p, sz, vpp], i32),
        "lvs_eq_table_free": ([vp], None),
        "lvs_edit_distance_preprocessed_batch": ([vp, vpp, ctypes.POINTER(ctypes.c_char_p), szp, sz,
                                                  ctypes.POINTER(lvs_opts), vpp], i32),
        "lvs_result_info": ([vp, szp, sz, szp, szp], i32),
        "lvs_result_export": ([vp, sz, u64p, szp], i32),
        "lvs_result_free": ([vp], None),
        "lvs_result_sum": ([vp, vp, vpp], i32),
        "lvs_decrypt": ([vp, vp, sz, u32p], i32),
        "lvs_decrypt_all": ([vp, vp, u32p], i32),
        "lvs_decrypt_distance": ([vp, u64p, sz, ctypes.c_int64, u32p], i32),
        "lvs_pbs_batch_device": ([vp, vp, sz, vp, vp, sz, sz], i32),
        "lvs_pbs_batch_device_fft64": ([vp, vp, sz, vp, vp, sz, sz], i32),
        "lvs_ctx_prepare_fft64": ([vp, vp], i32),
        "lvs_ctx_autotune": ([vp], i32),
        "lvs_ct_string_pin": ([vp], i32),
        "lvs_debug_fail_allocations": ([i32], None),
        "lvs_ctx_br_split": ([vp, ctypes.POINTER(sz)], i32),
        "lvs_ctx_ks_gemm_min": ([vp, ctypes.POINTER(sz)], i32),
        "lvs_ctx_set_ks_gemm_min": ([vp, sz], i32),
        "lvs_ctx_max_launch_jobs": ([vp, ctypes.POINTER(sz)], i32),
        "lvs_ctx_set_max_launch_jobs": ([vp, sz], i32),
        "lvs_ctx_set_br_split": ([vp, sz], i32),
        "lvs_preprocess_batch": ([vp, vpp, sz, ctypes.c_char_p, sz, vpp], i32),
        "lvs_ctx_set_wave_fill": ([vp, i32], i32),
        "lvs_ctx_set_key_staging": ([vp, i32], i32),
        "lvs_ctx_key_staging": ([vp, ctypes.POINTER(i32)], i32),
        "lvs_debug_drop_key_copy": ([vp, i32], i32),
        "lvs_ctx_wave_fill": ([vp, ctypes.POINTER(i32)], i32),
        "lvs_plan_batch": ([szp, szp, sz, u32, i32, sz, ctypes.POINTER(ctypes.c_int64), szp, szp], i32),
        "lvs_probe_modmul": ([i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], i32),
        "lvs_probe_key_product": ([i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], i32),
        "lvs_probe_int_mul": ([i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], i32),
        "lvs_ctx_ks_plan": ([vp, sz, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "lvs_ctx_set_ks_plan": ([vp, sz, i32, i32], i32),
        "lvs_noise_budget": ([ctypes.POINTER(lvs_params), ctypes.c_double, ctypes.POINTER(ctypes.c_double)], i32),
        "lvs_noise_pfail": ([ctypes.POINTER(lvs_params), ctypes.c_double, ctypes.POINTER(ctypes.c_double)], i32),
        "lvs_noise_plan": ([sz, sz, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_uint8),
                            ctypes.POINTER(ctypes.c_double)], i32),
        "lvs_plan_pair": ([sz, sz, u32, i32, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, sz,
                           ctypes.POINTER(lvs_plan_layout), ctypes.POINTER(lvs_plan_job), szp], i32),
        "lvs_plan_table": ([sz, i32, ctypes.c_char_p, sz, ctypes.POINTER(lvs_plan_layout),
                            ctypes.POINTER(lvs_plan_job), szp], i32),
        "lvs_keyswitch_batch_device": ([vp, vp, sz, vp, sz], i32),
        "lvs_poly_mul_device": ([vp, vp, vp, vp, sz], i32),
        "lvs_ctx_set_timing": ([vp, i32], i32),
        "lvs_ctx_kernel_stats": ([vp, i32, ctypes.POINTER(lvs_kernel_stats)], i32),
        "lvs_ctx_pbs_count": ([vp, u64p], i32),
        "lvs_ctx_launch_count": ([vp, u64p], i32),
        "lvs_ct_string_upload": ([vp, vp], i32),
        "lvs_pbs_batch_device_noalloc": ([vp, vp, sz, vp, vp, sz, sz], i32),
        "lvs_server_create": ([vp, sz, sz, vpp], i32),
        "lvs_server_submit": ([vp, ctypes.POINTER(lvs_query), ctypes.POINTER(u64)], i32),
        "lvs_server_poll": ([vp, u64, vpp], i32),
        "lvs_server_stats_get": ([vp, ctypes.POINTER(lvs_server_stats)], i32),
        "lvs_server_free": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res


def _check(st):
    if st != LVS_OK:
        raise LvsError(st, lib().lvs_last_error().decode(errors="replace"))


def _ptr(x):
    """Device pointer of an int or a torch tensor."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


class _Handle:
    _free = None

    def __init__(self, ptr, owner=None):
        self.ptr = ptr
        self._owner = owner   # keeps parents alive

    def close(self):
        """Releases the native object now (idempotent)."""
        p, self.ptr = getattr(self, "ptr", None), None
        if p and self._free and _lib is not None:
            getattr(_lib, self._free)(p)

    def __del__(self):
        self.close()

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


class ClientKey(_Handle):
    _free = "lvs_client_key_free"


class ServerKey(_Handle):
    _free = "lvs_server_key_free"


class Context(_Handle):
    _free = "lvs_ctx_free"


class CtString(_Handle):
    _free = "lvs_ct_string_free"


class Result(_Handle):
    _free = "lvs_result_free"


class EqTable(_Handle):
    _free = "lvs_eq_table_free"


class Server(_Handle):
    _free = "lvs_server_free"


# ------------------------------------------------------------------ params

def lvs_params_default():
    p = lvs_params()
    lib().lvs_params_default(ctypes.byref(p))
    return p


def lvs_params_test():
    p = lvs_params()
    lib().lvs_params_test(ctypes.byref(p))
    return p


def lvs_opts_default(use_graph=True, band=-1, refresh_budget=0):
    """band >= 0: only the cells of the band of Section 3.2 (|i - j| <= band,
    widened to the diagonals between 0 and n - m when m != n), the result
    holding the readout path; refresh_budget: 0 from the parameters, > 0
    explicit, < 0 no refresh."""
    o = lvs_opts()
    lib().lvs_opts_default(ctypes.byref(o))
    o.use_graph = 1 if use_graph else 0
    o.band = band
    o.refresh_budget = refresh_budget
    return o


def lvs_noise_budget(params, log2_pfail=-64.0):
    b = ctypes.c_double()
    _check(lib().lvs_noise_budget(ctypes.byref(params), ctypes.c_double(log2_pfail), ctypes.byref(b)))
    return b.value


def lvs_debug_fail_allocations(count):
    lib().lvs_debug_fail_allocations(count)


def lvs_noise_pfail(params, key_var):
    v = ctypes.c_double()
    _check(lib().lvs_noise_pfail(ctypes.byref(params), ctypes.c_double(key_var), ctypes.byref(v)))
    return v.value


def lvs_noise_plan(m, n, band, budget):
    """(list of refreshed anti-diagonals d = i + j, largest key variance)."""
    r = np.zeros(m + n + 1, dtype=np.uint8)
    w = ctypes.c_double()
    _check(lib().lvs_noise_plan(m, n, band, ctypes.c_double(budget),
                                r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(w)))
    return [int(d) for d in np.nonzero(r)[0]], w.value


def lvs_plan_pair(m, n, eq_lookups, band=-1, refresh=None, plain=None, subset=None):
    """(layout dict, list of job dicts) of one pair's wavefront plan (host only)."""
    rf = bytes(bytearray(refresh)) if refresh is not None else None
    pb = _bytes(plain) if plain is not None else None
    sb = _bytes(subset) if subset is not None else None
    lay = lvs_plan_layout()
    cnt = ctypes.c_size_t(0)
    args = (m, n, eq_lookups, band, rf, pb, sb, len(sb) if sb is not None else 0, ctypes.byref(lay))
    _check(lib().lvs_plan_pair(*args, None, ctypes.byref(cnt)))
    jobs = (lvs_plan_job * max(1, cnt.value))()
    _check(lib().lvs_plan_pair(*args, jobs, ctypes.byref(cnt)))
    return lay.as_dict(), _plan_jobs(jobs, cnt.value)


def _plan_jobs(jobs, n):
    return [{"step": j.step, "src": list(j.src), "coef": list(j.coef), "cst": j.cst, "dst": list(j.dst),
             "tap": j.tap, "lut": j.lut, "kind": j.kind, "tapsel": j.tapsel} for j in jobs[:n]]


def lvs_plan_batch(sizes, eq_lookups, band=-1, wave=0):
    """sizes: [(m, n), ...].  Returns (launch of every step, per pair as a
    list, number of launches) of the batch schedule (host only)."""
    np_ = len(sizes)
    m = (ctypes.c_size_t * max(1, np_))(*[a for a, b in sizes])
    n = (ctypes.c_size_t * max(1, np_))(*[b for a, b in sizes])
    cnt, nl = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib().lvs_plan_batch(m, n, np_, eq_lookups, band, wave, None, ctypes.byref(cnt), ctypes.byref(nl)))
    out = (ctypes.c_int64 * max(1, cnt.value))()
    _check(lib().lvs_plan_batch(m, n, np_, eq_lookups, band, wave, out, ctypes.byref(cnt), ctypes.byref(nl)))
    res, k = [], 0
    for a, b in sizes:
        steps = lvs_plan_pair(a, b, eq_lookups, band)[0]["steps"]
        res.append(list(out[k:k + steps]))
        k += steps
    return res, nl.value


def lvs_ctx_set_wave_fill(ctx, enable):
    _check(lib().lvs_ctx_set_wave_fill(ctx, 1 if enable else 0))


def lvs_ctx_wave_fill(ctx):
    v = ctypes.c_int32()
    _check(lib().lvs_ctx_wave_fill(ctx, ctypes.byref(v)))
    return bool(v.value)


def lvs_ctx_set_key_staging(ctx, enable):
    _check(lib().lvs_ctx_set_key_staging(ctx, 1 if enable else 0))


def lvs_ctx_key_staging(ctx):
    v = ctypes.c_int32()
    _check(lib().lvs_ctx_key_staging(ctx, ctypes.byref(v)))
    return bool(v.value)


def lvs_debug_drop_key_copy(ctx, enable):
    _check(lib().lvs_debug_drop_key_copy(ctx, 1 if enable else 0))


def lvs_plan_table(m, alphabet, subset):
    """(layout dict, list of job dicts) of a Section 5 table build (host only)."""
    sb = _bytes(subset)
    lay = lvs_plan_layout()
    cnt = ctypes.c_size_t(0)
    _check(lib().lvs_plan_table(m, alphabet, sb, len(sb), ctypes.byref(lay), None, ctypes.byref(cnt)))
    jobs = (lvs_plan_job * max(1, cnt.value))()
    _check(lib().lvs_plan_table(m, alphabet, sb, len(sb), ctypes.byref(lay), jobs, ctypes.byref(cnt)))
    return lay.as_dict(), _plan_jobs(jobs, cnt.value)


def lvs_version():
    return lib().lvs_version().decode()


# ------------------------------------------------------------------ keys

def lvs_keygen(params, seed):
    ck, sk = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().lvs_keygen(ctypes.byref(params), seed, ctypes.byref(ck), ctypes.byref(sk)))
    return ClientKey(ck.value), ServerKey(sk.value)


def lvs_client_key_export(ck):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().lvs_client_key_export(ck, None, ctypes.byref(a), None, ctypes.byref(b)))
    la, gb = np.zeros(a.value, np.uint64), np.zeros(b.value, np.uint64)
    _check(lib().lvs_client_key_export(ck, _u64p(la), ctypes.byref(a), _u64p(gb), ctypes.byref(b)))
    return la, gb


def lvs_server_key_export(sk):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().lvs_server_key_export(sk, None, ctypes.byref(a), None, ctypes.byref(b)))
    bsk, ksk = np.zeros(a.value, np.uint64), np.zeros(b.value, np.uint64)
    _check(lib().lvs_server_key_export(sk, _u64p(bsk), ctypes.byref(a), _u64p(ksk), ctypes.byref(b)))
    return bsk, ksk


def lvs_server_key_import(params, bsk, ksk):
    bsk = np.ascontiguousarray(bsk, np.uint64)
    ksk = np.ascontiguousarray(ksk, np.uint64)
    out = ctypes.c_void_p()
    _check(lib().lvs_server_key_import(ctypes.byref(params), _u64p(bsk), bsk.size, _u64p(ksk), ksk.size,
                                       ctypes.byref(out)))
    return ServerKey(out.value)


def lvs_client_key_import(params, lwe_key, glwe_key):
    lwe_key = np.ascontiguousarray(lwe_key, np.uint64)
    glwe_key = np.ascontiguousarray(glwe_key, np.uint64)
    out = ctypes.c_void_p()
    _check(lib().lvs_client_key_import(ctypes.byref(params), _u64p(lwe_key), lwe_key.size, _u64p(glwe_key),
                                       glwe_key.size, ctypes.byref(out)))
    return ClientKey(out.value)


def lvs_server_key_params(sk):
    p = lvs_params()
    _check(lib().lvs_server_key_params(sk, ctypes.byref(p)))
    return p


# ------------------------------------------------------------------ context

def lvs_ctx_create(sk, device=0, stream=None):
    """stream: None (library-owned stream), an int cudaStream_t, or a torch.cuda.Stream."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    c = ctypes.c_void_p()
    _check(lib().lvs_ctx_create(sk, device, ctypes.c_void_p(stream) if stream else None, ctypes.byref(c)))
    return Context(c.value, owner=sk)


def lvs_ctx_free(ctx):
    """Frees the context now (otherwise when the handle is collected)."""
    ctx.close()


def lvs_ctx_synchronize(ctx):
    _check(lib().lvs_ctx_synchronize(ctx))


def lvs_ctx_set_timing(ctx, enable):
    _check(lib().lvs_ctx_set_timing(ctx, 1 if enable else 0))


def lvs_ctx_kernel_stats(ctx, kind):
    s = lvs_kernel_stats()
    _check(lib().lvs_ctx_kernel_stats(ctx, kind, ctypes.byref(s)))
    return {"launches": s.launches, "items": s.items, "total_ms": s.total_ms}


def lvs_ctx_pbs_count(ctx):
    v = ctypes.c_uint64()
    _check(lib().lvs_ctx_pbs_count(ctx, ctypes.byref(v)))
    return v.value


def lvs_ctx_launch_count(ctx):
    v = ctypes.c_uint64()
    _check(lib().lvs_ctx_launch_count(ctx, ctypes.byref(v)))
    return v.value


# ------------------------------------------------------------------ client

def _bytes(s):
    return s.encode("latin-1") if isinstance(s, str) else bytes(s)


def lvs_encrypt_string(ck, s, alphabet, noise_seed, string_id):
    b = _bytes(s)
    out = ctypes.c_void_p()
    _check(lib().lvs_encrypt_string(ck, b, len(b), alphabet, noise_seed, string_id, ctypes.byref(out)))
    return CtString(out.value)


def lvs_ct_string_pin(s):
    _check(lib().lvs_ct_string_pin(s))


def lvs_ct_string_upload(ctx, s):
    _check(lib().lvs_ct_string_upload(ctx, s))


def lvs_ct_string_info(s):
    n, sy, big, al = ctypes.c_size_t(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int()
    _check(lib().lvs_ct_string_info(s, ctypes.byref(n), ctypes.byref(sy), ctypes.byref(big), ctypes.byref(al)))
    return {"len": n.value, "symbols": sy.value, "big_dim": big.value, "alphabet": al.value}


def lvs_ct_string_export(s):
    w = ctypes.c_size_t()
    _check(lib().lvs_ct_string_export(s, None, ctypes.byref(w)))
    a = np.zeros(w.value, np.uint64)
    _check(lib().lvs_ct_string_export(s, _u64p(a), ctypes.byref(w)))
    info = lvs_ct_string_info(s)
    return a.reshape(info["len"], info["symbols"], info["big_dim"] + 1)


def lvs_ct_string_import(arr, alphabet):
    arr = np.ascontiguousarray(arr, dtype=np.uint64)
    big = arr.shape[-1] - 1
    out = ctypes.c_void_p()
    _check(lib().lvs_ct_string_import(_u64p(arr), arr.shape[0], alphabet, big, ctypes.byref(out)))
    return CtString(out.value)


def lvs_decrypt_lwe(ck, ct):
    ct = np.ascontiguousarray(ct, dtype=np.uint64)
    v = ctypes.c_uint32()
    _check(lib().lvs_decrypt_lwe(ck, _u64p(ct), ctypes.byref(v)))
    return v.value


def lvs_encrypt_lwe(ck, value, noise_seed, i0, i1, big_dim):
    ct = np.zeros(big_dim + 1, np.uint64)
    _check(lib().lvs_encrypt_lwe(ck, value, noise_seed, i0, i1, _u64p(ct)))
    return ct


# ------------------------------------------------------------------ server

def lvs_eq(ctx, a, i, b, j, times9=True):
    out = ctypes.c_void_p()
    _check(lib().lvs_eq(ctx, a, i, b, j, 1 if times9 else 0, ctypes.byref(out)))
    return Result(out.value)


def lvs_edit_distance_batch(ctx, a_list, b_list, opts=None):
    n = len(a_list)
    assert len(b_list) == n
    A = (ctypes.c_void_p * max(1, n))(*[x.ptr for x in a_list])
    B = (ctypes.c_void_p * max(1, n))(*[x.ptr for x in b_list])
    out = ctypes.c_void_p()
    _check(lib().lvs_edit_distance_batch(ctx, A, B, n, ctypes.byref(opts) if opts else None, ctypes.byref(out)))
    return Result(out.value)


def lvs_preprocess(ctx, enc, subset=None):
    out = ctypes.c_void_p()
    sb = _bytes(subset) if subset is not None else None
    _check(lib().lvs_preprocess(ctx, enc, sb, len(sb) if sb is not None else 0, ctypes.byref(out)))
    return EqTable(out.value, owner=ctx)


def lvs_preprocess_batch(ctx, encs, subset=None):
    n = len(encs)
    E = (ctypes.c_void_p * max(1, n))(*[e.ptr for e in encs])
    outs = (ctypes.c_void_p * max(1, n))()
    sb = _bytes(subset) if subset is not None else None
    _check(lib().lvs_preprocess_batch(ctx, E, n, sb, len(sb) if sb is not None else 0, outs))
    return [EqTable(outs[k], owner=ctx) for k in range(n)]


def lvs_edit_distance_preprocessed_batch(ctx, tables, plains, opts=None):
    n = len(tables)
    T = (ctypes.c_void_p * max(1, n))(*[t.ptr for t in tables])
    bs = [_bytes(p) for p in plains]
    Pp = (ctypes.c_char_p * max(1, n))(*bs)
    L = (ctypes.c_size_t * max(1, n))(*[len(b) for b in bs])
    out = ctypes.c_void_p()
    _check(lib().lvs_edit_distance_preprocessed_batch(ctx, T, Pp, L, n, ctypes.byref(opts) if opts else None,
                                                      ctypes.byref(out)))
    return Result(out.value)


def lvs_result_info(r, pair=0):
    items, m, n = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().lvs_result_info(r, ctypes.byref(items), 0, None, None))
    if items.value == 0:
        return {"items": 0}
    _check(lib().lvs_result_info(r, ctypes.byref(items), pair, ctypes.byref(m), ctypes.byref(n)))
    return {"items": items.value, "m": m.value, "n": n.value}


def lvs_result_export(r, pair, big_dim):
    w = ctypes.c_size_t()
    _check(lib().lvs_result_export(r, pair, None, ctypes.byref(w)))
    a = np.zeros(w.value, np.uint64)
    _check(lib().lvs_result_export(r, pair, _u64p(a), ctypes.byref(w)))
    return a.reshape(-1, big_dim + 1)


def lvs_result_sum(ctx, r):
    out = ctypes.c_void_p()
    _check(lib().lvs_result_sum(ctx, r, ctypes.byref(out)))
    return Result(out.value)


def lvs_decrypt(ck, r, pair):
    v = ctypes.c_uint32()
    _check(lib().lvs_decrypt(ck, r, pair, ctypes.byref(v)))
    return v.value


def lvs_decrypt_distance(ck, rows, base):
    """Distance from exported result rows ([count][k*N+1]) and the base."""
    rows = np.ascontiguousarray(rows, np.uint64)
    count = rows.shape[0] if rows.ndim == 2 else 0
    d = ctypes.c_uint32()
    _check(lib().lvs_decrypt_distance(ck, _u64p(rows), count, int(base), ctypes.byref(d)))
    return d.value


def lvs_decrypt_all(ck, r):
    n = lvs_result_info(r)["items"]
    out = np.zeros(max(1, n), np.uint32)
    _check(lib().lvs_decrypt_all(ck, r, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return [int(x) for x in out[:n]]


# ------------------------------------------------------------------ serving

def lvs_server_create(ctx, mem_budget_bytes, max_active=0):
    out = ctypes.c_void_p()
    _check(lib().lvs_server_create(ctx, mem_budget_bytes, max_active, ctypes.byref(out)))
    return Server(out.value, owner=ctx)


def lvs_server_submit(server, query, ref_enc=None, ref_plain=None):
    """query, ref_enc: CtString; ref_plain: str/bytes (used when ref_enc is None)."""
    rp = _bytes(ref_plain) if ref_plain is not None else None
    q = lvs_query(query.ptr, ref_enc.ptr if ref_enc is not None else None, rp, len(rp) if rp is not None else 0)
    t = ctypes.c_uint64()
    _check(lib().lvs_server_submit(server, ctypes.byref(q), ctypes.byref(t)))
    return t.value


def lvs_server_poll(server, ticket):
    """Result when done, None while pending/running."""
    out = ctypes.c_void_p()
    st = lib().lvs_server_poll(server, ticket, ctypes.byref(out))
    if st == LVS_ERR_STATE:
        return None
    _check(st)
    return Result(out.value)


def lvs_server_free(server):
    """Stops the server's worker and frees it now (otherwise when the handle is collected)."""
    server.close()


def lvs_server_stats_get(server):
    s = lvs_server_stats()
    _check(lib().lvs_server_stats_get(server, ctypes.byref(s)))
    return s.as_dict()


# ------------------------------------------------------------------ low level (device pointers)

def lvs_pbs_batch_device(ctx, d_in, in_stride, d_lut, d_out, out_stride, count):
    _check(lib().lvs_pbs_batch_device(ctx, _ptr(d_in), in_stride, _ptr(d_lut), _ptr(d_out), out_stride, count))


def lvs_probe_int_mul(device=0):
    """(low-half, high-half) 32-bit multiplies per SM per clock, measured."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().lvs_probe_int_mul(device, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def lvs_probe_modmul(device=0):
    """(Shoup products, lazy NTT butterflies) per SM per clock, measured."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().lvs_probe_modmul(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lvs_probe_key_product(device=0):
    """(64-bit multiply-accumulates, L2 -> SM bytes in the key product's shape)
    per SM per clock, measured."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().lvs_probe_key_product(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lvs_ctx_autotune(ctx):
    _check(lib().lvs_ctx_autotune(ctx))


def lvs_ctx_ks_plan(ctx, njobs):
    """(jobs per CTA, split) of the key switch for a launch of njobs PBS."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lvs_ctx_ks_plan(ctx, njobs, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lvs_ctx_ks_gemm_min(ctx):
    v = ctypes.c_size_t()
    _check(lib().lvs_ctx_ks_gemm_min(ctx, ctypes.byref(v)))
    return v.value


def lvs_ctx_set_ks_gemm_min(ctx, min_jobs):
    _check(lib().lvs_ctx_set_ks_gemm_min(ctx, min_jobs))


def lvs_ctx_max_launch_jobs(ctx):
    v = ctypes.c_size_t()
    _check(lib().lvs_ctx_max_launch_jobs(ctx, ctypes.byref(v)))
    return v.value


def lvs_ctx_set_max_launch_jobs(ctx, max_jobs):
    _check(lib().lvs_ctx_set_max_launch_jobs(ctx, max_jobs))


def lvs_ctx_br_split(ctx):
    v = ctypes.c_size_t()
    _check(lib().lvs_ctx_br_split(ctx, ctypes.byref(v)))
    return v.value


def lvs_ctx_set_br_split(ctx, max_jobs):
    _check(lib().lvs_ctx_set_br_split(ctx, max_jobs))


def lvs_ctx_set_ks_plan(ctx, njobs, jobs_per_cta, split):
    _check(lib().lvs_ctx_set_ks_plan(ctx, njobs, jobs_per_cta, split))


def lvs_ctx_prepare_fft64(ctx, sk):
    _check(lib().lvs_ctx_prepare_fft64(ctx, sk))


def lvs_pbs_batch_device_fft64(ctx, d_in, in_stride, d_lut, d_out, out_stride, count):
    _check(lib().lvs_pbs_batch_device_fft64(ctx, _ptr(d_in), in_stride, _ptr(d_lut), _ptr(d_out), out_stride,
                                            count))


def lvs_pbs_batch_device_noalloc(ctx, d_in, in_stride, d_lut, d_out, out_stride, count):
    """Same as lvs_pbs_batch_device, without allocating: scratch in the
    library's static device array (see include/lvs.h for the limit)."""
    _check(lib().lvs_pbs_batch_device_noalloc(ctx, _ptr(d_in), in_stride, _ptr(d_lut), _ptr(d_out), out_stride,
                                              count))


def lvs_keyswitch_batch_device(ctx, d_in, in_stride, d_out, count):
    _check(lib().lvs_keyswitch_batch_device(ctx, _ptr(d_in), in_stride, _ptr(d_out), count))


def lvs_poly_mul_device(ctx, d_dig, d_poly, d_out, count):
    _check(lib().lvs_poly_mul_device(ctx, _ptr(d_dig), _ptr(d_poly), _ptr(d_out), count))
