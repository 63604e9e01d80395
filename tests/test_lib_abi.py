"""The C-ABI library builds, loads and exports every symbol include/tvs.h declares.

Runs without a GPU: only host-side entry points and argument checks that
return before any CUDA call are exercised.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="needs the CUDA toolkit to build libtvs")


@pytest.fixture(scope="module")
def lib():
    from paper_2602_17494_gb300 import build
    build.build()
    from paper_2602_17494_gb300 import binding
    return binding


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tvs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tvs_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib.lib(), n), n
    assert sorted(lib.EXPORTED) == names


def test_version_and_strings(lib):
    L = lib.lib()
    assert L.tvs_version() >= 100
    assert L.tvs_status_string(0) == b"ok"
    assert b"argument" in L.tvs_status_string(1)


def test_workspace_sizes(lib):
    a = lib.workspace_bytes(1, 64, 64)
    b = lib.workspace_bytes(1, 1024, 1024)
    assert 0 < a < b
    assert lib.workspace_bytes(2, 1024, 1024) < b
    dd = lib.make_decomp(4, 4, 8, 10)
    assert lib.workspace_bytes(2, 1024, 1024, dd) > lib.workspace_bytes(2, 1024, 1024)
    assert lib.workspace_bytes(0, 1024, 1024, dd) > b
    L = lib.lib()
    assert L.tvs_workspace_bytes(1, 1, 64, None, 0) == 0          # too small
    assert L.tvs_workspace_bytes(1, 8193, 64, None, 0) == 0       # too large
    # a 16-bit step-1 dual needs less; Schwarz step 1 keeps an FP32 dual
    assert 0 < L.tvs_workspace_bytes(1, 64, 64, None, 1) < L.tvs_workspace_bytes(1, 64, 64, None, 0)
    dd4 = lib.make_decomp(2, 2, 4, 4)
    assert L.tvs_workspace_bytes(1, 64, 64, ctypes.byref(dd4), 1) == 0
    assert L.tvs_workspace_bytes(2, 64, 64, None, 7) == 0         # no such storage
    assert L.tvs_workspace_bytes(2, 64, 64, None, 3) == lib.workspace_bytes(2, 64, 64, storage=1)
    # 16-bit storage halves the two step-2 dual buffers (and the Schwarz warm starts)
    n = 1024
    f32, bf16, f16 = (lib.workspace_bytes(2, n, n, storage=s) for s in (0, 1, 2))
    assert bf16 == f16 and f32 - bf16 >= 2 * 2 * 2 * n * n
    assert lib.workspace_bytes(2, n, n, dd, storage=1) < lib.workspace_bytes(2, n, n, dd)
    assert lib.workspace_bytes(0, n, n, dd, storage=2) < lib.workspace_bytes(0, n, n, dd)


def test_bad_arguments_rejected_before_any_device_work(lib):
    L = lib.lib()
    it = lib.make_iter(10)
    rep = lib.TvsReport()
    fake = ctypes.c_void_p(0x1000)        # never dereferenced: checks fail first
    # n2 < 2
    assert L.tvs_step1(fake, 1, 8, 0.05, ctypes.byref(it), fake, None, fake, 1 << 30, None, ctypes.byref(rep)) == 1
    # delta <= 0
    assert L.tvs_step1(fake, 8, 8, 0.0, ctypes.byref(it), fake, None, fake, 1 << 30, None, ctypes.byref(rep)) == 1
    # t > 1/8
    bad = lib.make_iter(10, t=0.2)
    assert L.tvs_step2(fake, fake, 8, 8, 10.0, 1e-3, ctypes.byref(bad), fake, None, fake, 1 << 30, None,
                       ctypes.byref(rep)) == 1
    # workspace missing / too small / misaligned
    assert L.tvs_step2(fake, fake, 8, 8, 10.0, 1e-3, ctypes.byref(it), fake, None, None, 1 << 30, None,
                       ctypes.byref(rep)) == 2
    assert L.tvs_step2(fake, fake, 8, 8, 10.0, 1e-3, ctypes.byref(it), fake, None, fake, 16, None,
                       ctypes.byref(rep)) == 2
    assert L.tvs_step2(fake, fake, 8, 8, 10.0, 1e-3, ctypes.byref(it), fake, None, ctypes.c_void_p(0x1004),
                       1 << 30, None, ctypes.byref(rep)) == 2
    # Schwarz: cores narrower than the overlap
    dd = lib.make_decomp(4, 4, 8, 5)
    assert L.tvs_schwarz(2, fake, fake, 20, 20, 10.0, 1e-3, ctypes.byref(dd), ctypes.byref(it), fake, None, fake,
                         1 << 30, None, ctypes.byref(rep)) == 1
    # a 16-bit dual is not an option of Schwarz step 1; unknown storage values are argument errors
    bf = lib.make_iter(10, storage=1)
    dd2 = lib.make_decomp(2, 2, 2, 2)
    assert L.tvs_schwarz(1, fake, None, 16, 16, 0.05, 1e-3, ctypes.byref(dd2), ctypes.byref(bf), fake, None, fake,
                         1 << 30, None, ctypes.byref(rep)) == 6
    odd = lib.make_iter(10, storage=9)
    assert L.tvs_step2(fake, fake, 8, 8, 10.0, 1e-3, ctypes.byref(odd), fake, None, fake, 1 << 30, None,
                       ctypes.byref(rep)) == 1


def test_schwarz1_workspace_and_limits(lib):
    dd = lib.make_decomp(4, 4, 8, 10)
    assert lib.workspace_bytes(1, 1024, 1024, dd) > lib.workspace_bytes(1, 1024, 1024)
    L = lib.lib()
    big = lib.make_decomp(128, 128, 4, 4)     # 16384 subdomains x full-width rows: beyond the scratch limit
    assert L.tvs_workspace_bytes(1, 8192, 8192, ctypes.byref(big), 0) == 0


def test_engine_configuration_checks(lib):
    L = lib.lib()
    it = lib.make_iter(100, 0.125, 1e-4, 10)
    good = lib.make_engine_config(0.05, 10.0, 1e-3, it, it, 64, 4, 16, 8)
    assert L.tvs_engine_pool_overhead(ctypes.byref(good)) > 0
    b1 = L.tvs_engine_request_bytes(ctypes.byref(good), 256, 300)
    b2 = L.tvs_engine_request_bytes(ctypes.byref(good), 1024, 1024)
    assert 0 < b1 < b2
    assert L.tvs_engine_request_bytes(ctypes.byref(good), 1, 300) == 0        # too small
    bad_tile = lib.make_engine_config(0.05, 10.0, 1e-3, it, it, 64, 40, 16, 8)   # 2 overlap >= tile
    assert L.tvs_engine_pool_overhead(ctypes.byref(bad_tile)) == 0
    no_check = lib.make_engine_config(0.05, 10.0, 1e-3, lib.make_iter(100), it, 64, 4, 16, 8)
    assert L.tvs_engine_pool_overhead(ctypes.byref(no_check)) == 0          # check_every must be >= 1
    h = ctypes.c_void_p()
    assert L.tvs_engine_create(ctypes.byref(bad_tile), ctypes.c_void_p(0x1000), 1 << 30, None, ctypes.byref(h)) == 1
    assert L.tvs_engine_create(ctypes.byref(good), None, 1 << 30, None, ctypes.byref(h)) == 2
    huge = lib.make_engine_config(0.05, 10.0, 1e-3, it, it, 200, 4, 16, 8)      # subdomain beyond one CTA
    assert L.tvs_engine_create(ctypes.byref(huge), ctypes.c_void_p(0x1000), 1 << 30, None, ctypes.byref(h)) == 6


def test_tuner_workspace_and_argument_checks(lib):
    L = lib.lib()
    arr = lambda v: (ctypes.c_int * len(v))(*v)
    T, O = arr([32, 64]), arr([2, 4])
    a = L.tvs_tune_workspace_bytes(256, 300, T, 2, O, 2, 0)
    b = L.tvs_tune_workspace_bytes(256, 300, T, 2, O, 2, 3)
    assert a > b > 0                                    # 16-bit duals need less
    assert L.tvs_tune_workspace_bytes(256, 300, T, 0, O, 2, 0) == 0
    best = (ctypes.c_int * 3)()
    it = lib.make_iter(10, 0.125, 0.0, 2)               # no tolerance: nothing to tune against
    fake = ctypes.c_void_p(0x1000)
    assert L.tvs_tune_schwarz2(fake, fake, 64, 64, 10.0, 1e-3, ctypes.byref(it), T, 2, O, 2, arr([4]), 1, fake,
                               1 << 30, None, best, None) == 1


def test_irv2_and_w11_argument_checks(lib):
    L = lib.lib()
    it = lib.make_iter(10)
    rep = lib.TvsReport()
    fake = ctypes.c_void_p(0x1000)
    # IRV2 workspace: plans and the potential on the image grid on top of step 2
    assert lib.workspace_bytes(5, 256, 300) > lib.workspace_bytes(2, 256, 300)
    dd = lib.make_decomp(4, 4, 4, 8)
    assert lib.workspace_bytes(5, 256, 300, dd) > lib.workspace_bytes(5, 256, 300)
    assert L.tvs_workspace_bytes(5, 2, 300, None, 0) == 0          # the potential needs n2, n1 >= 3
    # IRV2: alpha <= 0, n < 3, workspace too small
    assert L.tvs_irv2(fake, fake, 64, 64, 0.0, ctypes.byref(it), None, fake, None, None, fake, 1 << 30, None,
                      ctypes.byref(rep)) == 1
    assert L.tvs_irv2(fake, fake, 2, 64, 10.0, ctypes.byref(it), None, fake, None, None, fake, 1 << 30, None,
                      ctypes.byref(rep)) == 1
    assert L.tvs_irv2(fake, fake, 64, 64, 10.0, ctypes.byref(it), None, fake, None, None, fake, 16, None,
                      ctypes.byref(rep)) == 2
    # W^{1,1}: p is required, eps > 0
    assert L.tvs_step2_w11(fake, fake, 64, 64, 10.0, 1e-3, ctypes.byref(it), fake, None, None, fake, 1 << 30,
                           None, ctypes.byref(rep)) == 1
    assert L.tvs_step2_w11(fake, fake, 64, 64, 10.0, 0.0, ctypes.byref(it), fake, fake, None, fake, 1 << 30,
                           None, ctypes.byref(rep)) == 1
