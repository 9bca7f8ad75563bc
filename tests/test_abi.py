"""The C-ABI library: builds, loads without a GPU, exports every symbol that
include/lvs.h declares, and its host-side logic (key generation, encryption,
decryption, argument checks) matches the oracle -- no GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import plain as P
from oracle import tfhe as T
from paper_2508_14568_gb300 import lvs as L
from tests.conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lvs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(lvs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    declared = declared_functions()
    assert len(declared) >= 30
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(L.EXPORTS) == declared


def test_version_and_params():
    assert "sm_103a" in L.lvs_version()
    p = L.lvs_params_default()
    q = T.params_lvs()
    assert p.as_dict() == q.as_dict()
    assert L.lvs_params_test().as_dict() == T.params_test().as_dict()


def test_keygen_matches_oracle_bit_for_bit_test_params():
    p = L.lvs_params_test()
    ck, sk = L.lvs_keygen(p, 0)
    K = T.Keys(T.params_test(), 0)
    lwe, glwe = L.lvs_client_key_export(ck)
    bsk, ksk = L.lvs_server_key_export(sk)
    assert np.array_equal(lwe, K.lwe_key)
    assert np.array_equal(glwe, K.glwe_key)
    assert np.array_equal(bsk, K.bsk)
    assert np.array_equal(ksk, K.ksk)


@pytest.mark.slow
def test_keygen_matches_oracle_full_params():
    p = L.lvs_params_default()
    ck, sk = L.lvs_keygen(p, 0)
    K = T.Keys(T.params_lvs(), 0)
    lwe, glwe = L.lvs_client_key_export(ck)
    bsk, ksk = L.lvs_server_key_export(sk)
    assert np.array_equal(lwe, K.lwe_key) and np.array_equal(glwe, K.glwe_key)
    assert np.array_equal(ksk, K.ksk)
    assert np.array_equal(bsk, K.bsk)


def test_encrypt_string_matches_oracle():
    p = L.lvs_params_test()
    ck, sk = L.lvs_keygen(p, 3)
    K = T.Keys(T.params_test(), 3)
    for alpha, la, s in [(L.LVS_ALPHA_ASCII7, P.ALPHA_ASCII7, "Hi, there~"),
                         (L.LVS_ALPHA_27, P.ALPHA_27, "AB Z"),
                         (L.LVS_ALPHA_DNA4, P.ALPHA_DNA4, "GATTACA")]:
        cs = L.lvs_encrypt_string(ck, s, alpha, 77, 5)
        got = L.lvs_ct_string_export(cs)
        want = T.encrypt_string(K, s, la, 77, 5)
        assert got.shape[0] == len(s)
        for i in range(len(s)):
            for t in range(got.shape[1]):
                assert np.array_equal(got[i, t], want[i][t])
                assert L.lvs_decrypt_lwe(ck, got[i, t]) == T.decrypt(K, want[i][t])


def test_encrypt_lwe_and_decrypt():
    ck, _ = L.lvs_keygen(L.lvs_params_test(), 4)
    K = T.Keys(T.params_test(), 4)
    for v in range(32):
        ct = L.lvs_encrypt_lwe(ck, v, 9, 1, v, 512)
        assert np.array_equal(ct, T.encrypt(K, v, 9, 1, v))
        assert L.lvs_decrypt_lwe(ck, ct) == v


def test_argument_errors_are_reported():
    p = L.lvs_params_test()
    bad = L.lvs_params()
    ctypes.memmove(ctypes.byref(bad), ctypes.byref(p), ctypes.sizeof(p))
    bad.N = 1000
    with pytest.raises(L.LvsError) as e:
        L.lvs_keygen(bad, 0)
    assert e.value.status == L.LVS_ERR_ARG
    ck, _ = L.lvs_keygen(p, 0)
    with pytest.raises(L.LvsError) as e:
        L.lvs_encrypt_string(ck, "abc", L.LVS_ALPHA_27, 0, 0)      # lowercase not in alphabet
    assert e.value.status == L.LVS_ERR_ARG
    with pytest.raises(L.LvsError) as e:
        L.lvs_encrypt_string(ck, "ACGU", L.LVS_ALPHA_DNA4, 0, 0)
    assert e.value.status == L.LVS_ERR_ARG
    # empty strings are valid
    s = L.lvs_encrypt_string(ck, "", L.LVS_ALPHA_ASCII7, 0, 0)
    assert L.lvs_ct_string_info(s)["len"] == 0


def test_ct_string_import_roundtrip():
    ck, _ = L.lvs_keygen(L.lvs_params_test(), 1)
    s = L.lvs_encrypt_string(ck, "KID", L.LVS_ALPHA_ASCII7, 2, 0)
    arr = L.lvs_ct_string_export(s)
    s2 = L.lvs_ct_string_import(arr, L.LVS_ALPHA_ASCII7)
    assert np.array_equal(L.lvs_ct_string_export(s2), arr)


def test_context_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    _, sk = L.lvs_keygen(L.lvs_params_test(), 0)
    with pytest.raises(L.LvsError) as e:
        L.lvs_ctx_create(sk, 0)
    assert e.value.status == L.LVS_ERR_CUDA


def test_null_arguments_are_rejected_before_any_device_work():
    """Entry points that launch work check their pointers on the host first:
    LVS_ERR_ARG and a message, no CUDA call (this runs without a GPU)."""
    lib = L.lib()
    out = ctypes.c_void_p()
    u = ctypes.c_uint32()
    calls = [
        ("lvs_result_sum", lambda: lib.lvs_result_sum(None, None, ctypes.byref(out))),
        ("lvs_edit_distance_batch", lambda: lib.lvs_edit_distance_batch(None, None, None, 1, None, ctypes.byref(out))),
        ("lvs_decrypt", lambda: lib.lvs_decrypt(None, None, 0, ctypes.byref(u))),
        ("lvs_decrypt_all", lambda: lib.lvs_decrypt_all(None, None, None)),
    ]
    for name, call in calls:
        assert call() == L.LVS_ERR_ARG, name
        assert lib.lvs_last_error().decode(), name
        assert out.value is None


@pytest.mark.parametrize("field,value", [("k", 2), ("N", 1024), ("n", 0), ("n", 5000), ("pbs_level", 1),
                                         ("pbs_level", 3), ("pbs_base_log", 14), ("ks_level", 9),
                                         ("ks_level", 0), ("ks_base_log", 7), ("lwe_noise_log2", 61)])
def test_parameter_limits(field, value):
    """Parameter sets outside what the kernels implement (k = 1, N in {512,
    2048}, a two-level bootstrapping gadget of <= 26 bits for three 30-bit NTT
    primes, a key-switching gadget of <= 8 levels and <= 30 bits) are refused
    on the host with LVS_ERR_ARG, by keygen and by the noise calls."""
    p = L.lvs_params_default()
    setattr(p, field, value)
    with pytest.raises(L.LvsError) as e:
        L.lvs_keygen(p, 0)
    assert e.value.status == L.LVS_ERR_ARG
    with pytest.raises(L.LvsError):
        L.lvs_noise_budget(p, -64)


C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "lvs.h"

int main(void)
{
    lvs_params p;
    lvs_client_key *ck = NULL;
    lvs_server_key *sk = NULL;
    uint64_t ct[513];
    uint32_t v = 99;
    double budget = 0.0;
    size_t count = 0;
    lvs_plan_layout lay;
    lvs_ctx *ctx = NULL;
    lvs_params_test(&p);
    if (lvs_keygen(&p, 7, &ck, &sk) != LVS_OK) return 1;
    for (uint32_t m = 0; m < 32; ++m) {
        if (lvs_encrypt_lwe(ck, m, 3, 0, m, ct) != LVS_OK) return 2;
        if (lvs_decrypt_lwe(ck, ct, &v) != LVS_OK || v != m) return 3;
    }
    lvs_params_default(&p);
    if (lvs_noise_budget(&p, -64.0, &budget) != LVS_OK || budget < 80000.0 || budget > 95000.0) return 4;
    if (lvs_plan_pair(4, 4, 2, -1, NULL, NULL, NULL, 0, &lay, NULL, &count) != LVS_OK || count != 48) return 5;
    if (lvs_keygen(NULL, 0, &ck, &sk) != LVS_ERR_ARG || lvs_last_error()[0] == 0) return 6;
    printf("%s\n", lvs_version());
    lvs_client_key_free(ck);
    lvs_server_key_free(sk);
    lvs_ctx_free(ctx);                       /* NULL is accepted */
    return 0;
}
"""


def test_header_is_plain_c_and_the_abi_links(tmp_path):
    """include/lvs.h compiles as C99 (no C++ in the public interface), and a C
    program linked against liblvs.so runs the host-side calls: keys, LWE
    encryption round trip (Table tab_pbs's 48 PBS for a 4 x 4 ASCII pair in the
    exported plan), the noise budget, error reporting."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    L.lib()                                   # builds liblvs.so if needed
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(L.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                           str(src), "-o", str(exe), "-L", libdir, "-llvs", "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "sm_103a" in out.stdout


def test_key_import_round_trip():
    """Keys rebuilt from their exported words (a server loading the client's
    evaluation keys) export the same words; the imported client key decrypts
    what the original encrypted, and mismatched or non-binary material is
    refused."""
    p = L.lvs_params_test()
    ck, sk = L.lvs_keygen(p, 11)
    lwe, glwe = L.lvs_client_key_export(ck)
    bsk, ksk = L.lvs_server_key_export(sk)
    sk2 = L.lvs_server_key_import(p, bsk, ksk)
    b2, k2 = L.lvs_server_key_export(sk2)
    assert np.array_equal(b2, bsk) and np.array_equal(k2, ksk)
    assert L.lvs_server_key_params(sk2).as_dict() == p.as_dict()
    ck2 = L.lvs_client_key_import(p, lwe, glwe)
    s = L.lvs_encrypt_string(ck, "Hello", L.LVS_ALPHA_ASCII7, 5, 0)
    s2 = L.lvs_encrypt_string(ck2, "Hello", L.LVS_ALPHA_ASCII7, 5, 0)
    assert np.array_equal(L.lvs_ct_string_export(s), L.lvs_ct_string_export(s2))
    for row in L.lvs_ct_string_export(s).reshape(-1, p.N + 1):
        assert L.lvs_decrypt_lwe(ck2, row) == L.lvs_decrypt_lwe(ck, row)
    with pytest.raises(L.LvsError):
        L.lvs_server_key_import(p, bsk[:-1], ksk)
    with pytest.raises(L.LvsError):
        L.lvs_server_key_import(L.lvs_params_default(), bsk, ksk)
    bad = glwe.copy()
    bad[3] = 2
    with pytest.raises(L.LvsError):
        L.lvs_client_key_import(p, lwe, bad)


def test_decrypt_distance_from_exported_rows():
    """The client's readout (Algorithm algo_complete's m + sum of the last row)
    from rows received as words: differences -1 / 0 / 1 as Z_32 residues."""
    p = L.lvs_params_test()
    ck, _ = L.lvs_keygen(p, 12)
    K = T.Keys(T.params_test(), 12)
    a, b = "kitten", "sitting"
    _, h, _, _ = P.lvs_plain(a, b)
    m, n = len(a), len(b)
    rows = np.stack([T.encrypt(K, h[m][j], 4, 0, j) for j in range(1, n + 1)])
    assert L.lvs_decrypt_distance(ck, rows, m) == P.wf_distance(a, b) == 3
    assert L.lvs_decrypt_distance(ck, np.zeros((0, p.N + 1), np.uint64), 5) == 5
    one = np.stack([T.encrypt(K, 3, 4, 1, 0)])
    assert L.lvs_decrypt_distance(ck, one, 0) == 3           # a summed result
