"""The C-ABI library builds, loads and exports every symbol include/kerdock.h
declares; host-side argument validation works without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2105_05879_gb300 import build as kbuild
from paper_2105_05879_gb300 import kerdock as K

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "kerdock.h")


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return K.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kerdock_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_list():
    assert declared_functions() == sorted(K.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_plan_info_sizes(lib):
    h = K.kerdock_plan_create(1024, 1024, K.KERDOCK_F32, 375, 2, 160)
    info = K.kerdock_plan_info(h)
    assert info["d"] == 1024 and info["k"] == 10 and info["num_bases"] == 513
    assert info["L"] == 1024 * 513 and info["ldr"] == 1024
    assert info["repr_bytes"] == 513 * 1024 * 1024 * 4
    # a 1 KiB status area (status word, scheduling counters), then the sign
    # table twice: p order and lane-transposed, 32 words per basis each
    assert info["table_bytes"] == 1024 + 512 * (32 + 32) * 4
    K.kerdock_plan_destroy(h)
    # padding: n = 2048 -> d = 4096 (power of four), m ragged -> ldr multiple of 8
    h = K.kerdock_plan_create(1001, 2048, K.KERDOCK_BF16, 10, 3, 5000)
    info = K.kerdock_plan_info(h)
    assert info["d"] == 4096 and info["ldr"] == 1008 and info["S"] == 1001
    assert info["repr_bytes"] == 2049 * 4096 * 1008 * 2
    K.kerdock_plan_destroy(h)
    for n, d in [(1, 4), (4, 4), (5, 16), (17, 64), (65, 256), (257, 1024), (1025, 4096)]:
        h = K.kerdock_plan_create(8, n, 0, 1, 1, 1)
        assert K.kerdock_plan_info(h)["d"] == d
        K.kerdock_plan_destroy(h)


@pytest.mark.parametrize("args,code", [
    ((0, 4, 0, 1, 1, 1), -1), ((4, 0, 0, 1, 1, 1), -1), ((4, 4, 2, 1, 1, 1), -1),
    ((4, 4, 0, 0, 1, 1), -1), ((4, 4, 0, 1, 0, 1), -1), ((4, 4, 0, 1, 1, 0), -1),
    ((4097, 4, 0, 1, 1, 1), -2), ((4, 4097, 0, 1, 1, 1), -2), ((4, 4, 0, 1, 33, 1), -2),
    ((4, 4, 0, 1 << 21, 16, 1), -2),
])
def test_create_rejects_bad_arguments(lib, args, code):
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_plan_create(*args)
    assert e.value.code == code


def test_calls_before_bind_fail_cleanly(lib):
    h = K.kerdock_plan_create(16, 16, 0, 4, 2, 4)
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_preprocess(h, 1 << 20, 16)
    assert e.value.code == -3
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_apply(h, 1 << 20, 1, 16, 0.1, 0, 0, 1 << 20, 1 << 20, 1 << 20, None, 0)
    assert e.value.code == -3
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_sync(h)
    assert e.value.code == -3
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_plan_bind(h, None, 0, None, 0, None)
    assert e.value.code == -1
    info = K.kerdock_plan_info(h)
    with pytest.raises(K.KerdockError) as e:   # too small
        K.kerdock_plan_bind(h, 256, info["repr_bytes"] - 1, 512, info["table_bytes"], None)
    assert e.value.code == -5
    with pytest.raises(K.KerdockError) as e:   # misaligned
        K.kerdock_plan_bind(h, 256 + 16, info["repr_bytes"], 512, info["table_bytes"], None)
    assert e.value.code == -8
    K.kerdock_plan_destroy(h)
    K.kerdock_plan_destroy(None)


def test_batch_schedule_calls_null_handle(lib):
    # a null batch is refused before any device work
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_batch_set_costs(None, np.ones(4))
    assert e.value.code == -1
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_batch_set_schedule(None, [[0, 1], [2]])
    assert e.value.code == -1
    assert K.kerdock_batch_ctas(None) == 0


def test_strerror_and_version(lib):
    assert K.kerdock_strerror(0) == "ok"
    assert "timed out" in K.kerdock_strerror(-7)
    assert K.kerdock_strerror(-99) == "unknown error"
    assert K.kerdock_version() >= 100


def test_theory_parameters_match_theorem3(lib):
    # the library's host computation against the oracle's restatement of
    # Theorem 3 (whose guarantee tests/test_oracle_query.py checks by Monte Carlo)
    from oracle import query as oq
    for a, eps, delta, eta, m in [(1.0, 0.5, 0.0, 0.2, 16), (1.0, 0.25, 0.0, 0.5, 64),
                                  (0.7, 0.6, 0.1, 0.9, 1000), (1.0, 0.9, 0.2, 1.0, 2048)]:
        J, Kb = K.kerdock_theory_parameters(a, eps, delta, eta, m)
        assert (J, Kb) == oq.theorem3_parameters(a, eps, delta, eta, m)
    # and against values worked by hand from Theorem 3's statement
    assert K.kerdock_theory_parameters(1.0, 0.5, 0.0, 0.2, 16) == (473, 9)
    assert K.kerdock_theory_parameters(2.0, 1.0, 0.5, 0.2, 16) == (1892, 9)
    assert K.kerdock_theory_parameters(0.5, 0.5, 0.0, 0.5, 2) == (119, 3)


def test_theory_parameters_errors(lib):
    for args in [(0.0, 0.5, 0.0, 0.1, 10), (1.0, 0.1, 0.2, 0.1, 10), (1.0, 0.5, -0.1, 0.1, 10),
                 (1.0, 0.5, 0.0, 0.0, 10), (1.0, 0.5, 0.0, 1.5, 10), (1.0, 0.5, 0.0, 0.1, 0)]:
        with pytest.raises(K.KerdockError) as ei:
            K.kerdock_theory_parameters(*args)
        assert ei.value.code == -1  # KERDOCK_ERR_INVALID_ARG
    # the guarantee at n = 1024, eps = 0.125, eta = 0.01 needs K = 24 batches,
    # within the library's 32; eta = 1e-9 at m = 4096 needs K = 59 > 32
    assert K.kerdock_theory_parameters(1.0, 0.125, 0.0, 0.01, 1024)[1] == 24
    with pytest.raises(K.KerdockError) as ei:
        K.kerdock_theory_parameters(1.0, 0.125, 0.0, 1e-9, 4096)
    assert ei.value.code == -2  # KERDOCK_ERR_UNSUPPORTED


def test_ring_tuning_values(lib):
    # rows per chunk 1, 2, 4 or 8 (0 = default); a geometry whose ring cannot
    # hold more chunks than the query kernel has coefficient warps is refused
    small = K.kerdock_plan_create(16, 16, 0, 4, 2, 4)        # 64-byte rows
    for cr in (0, 1, 2, 4, 8):
        K.kerdock_plan_set_tuning(small, 160, cr)
    for cr in (3, 5, 6, 16):
        with pytest.raises(K.KerdockError) as e:
            K.kerdock_plan_set_tuning(small, 160, cr)
        assert e.value.code == -1
    large = K.kerdock_plan_create(4096, 4096, 0, 4, 2, 4)    # 16 KiB float32 rows
    K.kerdock_plan_set_tuning(large, 160, 1)
    with pytest.raises(K.KerdockError) as e:                 # 9 slots: one chunk of 8
        K.kerdock_plan_set_tuning(large, 160, 8)
    assert e.value.code == -2
    K.kerdock_plan_destroy(small)
    K.kerdock_plan_destroy(large)
