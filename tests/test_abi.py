"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point the header declares, rejects bad arguments before touching
the device, and plans moduli that satisfy the exactness bound."""
import math
import os
import re

import pytest

import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import ffgpu as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"FFGPU_API\s+[\w\s\*]+?\b(ffgpu_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "ffgpu_fgemm" in names and len(names) >= 8
    L = ff.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    # and the binding knows every one of them
    assert names <= set(binding.SIGNATURES)


def test_status_strings_and_version():
    assert ff.version() >= 100
    for code, name in binding.STATUS.items():
        assert ff.status_string(code) == name


def test_invalid_arguments_rejected_without_device():
    f = ff.fgemm_ptr
    assert f(4, 4, 4, 1, 1, 8, 4, 8, 4, 0, 8, 4) == -2          # p < 2
    assert f(4, 4, 4, 2**31, 1, 8, 4, 8, 4, 0, 8, 4) == -2      # p > 2^31 - 1
    assert f(-1, 4, 4, 7, 1, 8, 4, 8, 4, 0, 8, 4) == -1         # negative m
    assert f(4, 4, 4, 7, 1, 8, 3, 8, 4, 0, 8, 4) == -1          # lda < k
    assert f(4, 4, 4, 7, 1, 8, 4, 8, 3, 0, 8, 4) == -1          # ldb < n
    assert f(4, 4, 4, 7, 1, 8, 4, 8, 4, 0, 8, 3) == -1          # ldc < n
    assert f(4, 4, 4, 7, 1, 0, 4, 8, 4, 0, 8, 4) == -1          # null A
    assert f(0, 4, 4, 7, 1, 0, 4, 0, 4, 0, 0, 4) == 0           # m = 0: nothing to do


MODULI_LIMIT = 255


def test_plan_moduli_are_coprime_and_sufficient():
    for p in (2, 3, 5, 251, 256, 257, 65521, 8388593, 2147483647):
        for k in (1, 64, 512, 8192, 65536, 1 << 20):
            pl = ff.fgemm_plan(128, 128, k, p)
            mods = pl["moduli"]
            assert len(mods) == pl["channels"] >= 1
            if p <= MODULI_LIMIT:
                assert pl["mode"] == 1 and mods == [p]
                continue
            # chunk of products summed exactly in f32: reduced value + chunk * max|r|^2 < 2^24
            R = max(m // 2 for m in mods)
            assert pl["k_chunk"] % 64 == 0 and (R + 1) + pl["k_chunk"] * R * R < 2**24
            assert pl["mode"] == 2
            assert all(2 <= m <= MODULI_LIMIT for m in mods)
            for i in range(len(mods)):
                for j in range(i + 1, len(mods)):
                    assert math.gcd(mods[i], mods[j]) == 1
            h = p // 2
            ks = -(-k // pl["k_slices"])
            M = math.prod(mods)
            # the sum of ks products of centred residues stays within M/4
            assert 4 * ks * h * h <= M
            # and one channel fewer would not do (the plan is minimal)
            assert 4 * ks * h * h > math.prod(mods[:-1]) or len(mods) == 1


def test_plan_channel_counts_of_the_sweep():
    # p < 2^31 at n = 8192: 10 channels; p < 2^16: 6; p < 2^8: the prime itself;
    # 1024 products between in-place reductions (residues |r| <= 127)
    assert ff.fgemm_plan(8192, 8192, 8192, 2147483647)["channels"] == 10
    assert ff.fgemm_plan(8192, 8192, 8192, 8388593)["channels"] == 8
    assert ff.fgemm_plan(8192, 8192, 8192, 65521)["channels"] == 6
    assert ff.fgemm_plan(8192, 8192, 8192, 251)["channels"] == 1
    assert ff.fgemm_plan(8192, 8192, 65536, 2147483647)["channels"] == 10
    assert ff.fgemm_plan(8192, 8192, 8192, 2147483647)["k_chunk"] == 1024


def test_workspace_size_monotone():
    a = ff.fgemm_workspace_size(1024, 1024, 1024, 65521)
    b = ff.fgemm_workspace_size(2048, 2048, 2048, 65521)
    assert 0 < a < b
    assert ff.fgemm_workspace_size(1024, 1024, 0, 65521) == 0


def test_argument_checks_of_the_other_routines_without_device():
    """ftrsm, LQUP and its derived routines, the batched call and the request
    server reject bad arguments synchronously, before any device call (these
    run here, on a host with no GPU).  Pointers are placeholders: nothing may
    be dereferenced on these paths."""
    import ctypes
    L = ff.lib()
    r, d, sv = ctypes.c_int64(0), ctypes.c_uint32(0), ctypes.c_void_p()
    P = 8  # a placeholder device pointer
    # ftrsm(side, uplo, diag, m, n, p, alpha, T, ldt, B, ldb, stream)
    assert L.ffgpu_ftrsm(0, 0, 1, 4, 4, 1, 1, P, 4, P, 4, None) == -2        # p < 2
    assert L.ffgpu_ftrsm(2, 0, 1, 4, 4, 7, 1, P, 4, P, 4, None) == -1        # side
    assert L.ffgpu_ftrsm(0, 0, 1, 4, 4, 7, 1, P, 3, P, 4, None) == -1        # ldt < m
    assert L.ffgpu_ftrsm(0, 0, 1, 4, 4, 7, 1, P, 4, P, 3, None) == -1        # ldb < n
    assert L.ffgpu_ftrsm(0, 0, 1, 4, 4, 7, 1, P, 4, None, 4, None) == -1     # null B
    assert L.ffgpu_ftrsm_ex(0, 0, 1, 4, 4, 7, 1, P, 4, P, 4, 5, None) == -1  # unknown algorithm
    # LQUP, rank, determinant, inverse: p must be prime
    assert L.ffgpu_lqup(4, 4, 15, P, 4, ctypes.byref(r), P, P, None) == -2
    assert L.ffgpu_lqup(-1, 4, 7, P, 4, ctypes.byref(r), P, P, None) == -1
    assert L.ffgpu_lqup(4, 4, 7, P, 3, ctypes.byref(r), P, P, None) == -1    # lda < n
    assert L.ffgpu_rank(4, 4, 9, P, 4, ctypes.byref(r), None) == -2
    r.value = 5
    assert L.ffgpu_rank(0, 4, 7, P, 4, ctypes.byref(r), None) == 0 and r.value == 0
    assert L.ffgpu_det(-1, 7, P, 4, ctypes.byref(d), None) == -1
    assert L.ffgpu_det(4, 21, P, 4, ctypes.byref(d), None) == -2
    assert L.ffgpu_inverse(4, 7, P, 4, None, 4, None) == -1                   # null X
    assert L.ffgpu_inverse(4, 7, P, 4, P, 3, None) == -1                      # ldx < n
    # batched and the server
    assert L.ffgpu_fgemm_batched(-1, None, None) == -1
    assert L.ffgpu_fgemm_batched(0, None, None) == 0
    assert L.ffgpu_server_create(0, 1 << 30, ctypes.byref(sv)) == -1          # no stream
    assert L.ffgpu_server_create(2, 100, ctypes.byref(sv)) == -1              # budget below 1 MiB
