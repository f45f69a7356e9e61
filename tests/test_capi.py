"""CPU checks of the C ABI: the library loads, exports every function that
include/aao.h declares, validates arguments before touching the GPU, and its
host-side g_k setup agrees with the oracle (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_2003_07020_gb300 import aao
from oracle import fcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(aao.LIB_PATH):
        __graft_entry__.build()
    return aao.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "aao.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aao_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_list():
    assert header_functions() == sorted(aao.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_setup_coeffs_matches_oracle(lib):
    # the oracle goes through log|Gamma|, whose relative error grows like |log Gamma(k)| eps
    # (about 4e-12 at k = 4096); the first weights agree to rounding
    for alpha in (1.2, 1.5, 1.8):
        g = aao.aao_setup_coeffs(alpha, 4096)
        ref = fcd.fcd_weights(alpha, 4096)
        np.testing.assert_allclose(g[:64], ref[:64], rtol=3e-13, atol=0)
        np.testing.assert_allclose(g, ref, rtol=5e-11, atol=0)


def test_setup_coeffs_rejects_bad_arguments(lib):
    buf = np.zeros(4)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    assert lib.aao_setup_coeffs(1.5, 0, p) == aao.AAO_EINVAL
    assert lib.aao_setup_coeffs(1.5, 4, None) == aao.AAO_EINVAL
    assert lib.aao_setup_coeffs(2.5, 4, p) == aao.AAO_EINVAL
    assert b"alpha" in lib.aao_last_error(None)


def test_default_opts(lib):
    o = aao.default_opts(aao.AAO_PREC_MIXED)
    assert (o.restart, o.tol, o.inner_tol, o.inner) == (20, 1e-10, 1e-6, aao.AAO_INNER_STRANG)
    o = aao.default_opts(aao.AAO_PREC_FP64)
    assert o.inner_tol == 1e-12 and o.prec == aao.AAO_PREC_FP64


@pytest.mark.parametrize("field,value,word", [
    ("M", 0, "M must"), ("Nt", 48, "Nt must"), ("Nt", 2, "Nt must"), ("dim", 3, "dim"), ("dim", 2, "My")])
def test_plan_create_validates_problem_without_gpu(lib, field, value, word):
    prob = aao.AaoProblem(1, 63, 64, 1.0, 1.5, 1.0, 0.0)
    setattr(prob, field, value)
    o = aao.default_opts()
    h = ctypes.c_void_p()
    st = lib.aao_plan_create(ctypes.byref(prob), ctypes.byref(o), None, ctypes.byref(h))
    assert st == aao.AAO_EINVAL and not h.value
    assert word.encode() in lib.aao_last_error(None)


def test_plan_create_validates_options_without_gpu(lib):
    prob = aao.AaoProblem(1, 64, 64, 1.0, 1.5, 1.0, 0.0)
    o = aao.default_opts(inner=aao.AAO_INNER_TAU)  # needs M+1 a power of two
    h = ctypes.c_void_p()
    assert lib.aao_plan_create(ctypes.byref(prob), ctypes.byref(o), None, ctypes.byref(h)) == aao.AAO_EINVAL
    o = aao.default_opts(restart=0)
    prob.M = 63
    assert lib.aao_plan_create(ctypes.byref(prob), ctypes.byref(o), None, ctypes.byref(h)) == aao.AAO_EINVAL


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.aao_matvec(None, None, None) == aao.AAO_EINVAL
    assert lib.aao_plan_destroy(None) == aao.AAO_OK
    assert lib.aao_plan_workspace_bytes(None) == 0


def test_fno_parameter_count_matches_oracle_layout(lib):
    from oracle import fno
    assert lib.aao_fno_num_params() == fno.num_params(32, 16, 4)


def test_fno_and_warm_start_calls_validate_without_gpu(lib):
    h = ctypes.c_void_p()
    # grid too small for 16 modes, and a null output handle
    assert lib.aao_fno_create(16, 4, 0, ctypes.byref(h)) == aao.AAO_EINVAL
    assert lib.aao_fno_create(63, 4, 0, None) == aao.AAO_EINVAL
    assert lib.aao_fno_destroy(None) == aao.AAO_OK
    assert lib.aao_fno_predict(None, 1, None, None, None, None, None) == aao.AAO_EINVAL
    assert lib.aao_fno_save(None, b"x") == aao.AAO_EINVAL
    assert lib.aao_plan_set_warm_start(None, None) == aao.AAO_EINVAL
    assert lib.aao_plan_record_pairs(None, 0, None, None, None) == aao.AAO_EINVAL
    n = ctypes.c_int64(-1)
    assert lib.aao_plan_recorded_pairs(None, ctypes.byref(n)) == aao.AAO_EINVAL


def test_plan_create_validates_launch_options_without_gpu(lib):
    prob = aao.AaoProblem(1, 2047, 64, 1.0, 1.5, 1.0, 0.0, 0, 1.5, 1.0)
    h = ctypes.c_void_p()
    for kw in (dict(cocg_threads=100), dict(cocg_threads=64), dict(use_graphs=2)):
        o = aao.default_opts(**kw)
        assert lib.aao_plan_create(ctypes.byref(prob), ctypes.byref(o), None, ctypes.byref(h)) == aao.AAO_EINVAL, kw
    assert lib.aao_plan_get_tuning(None, None) == aao.AAO_EINVAL


def test_plan_create_rejects_bad_matvec_kind_without_gpu(lib):
    prob = aao.AaoProblem(1, 63, 16, 1.0, 1.5, 1.0, 0.0, 0, 1.5, 1.0)
    h = ctypes.c_void_p()
    o = aao.default_opts(matvec=7)
    assert lib.aao_plan_create(ctypes.byref(prob), ctypes.byref(o), None, ctypes.byref(h)) == aao.AAO_EINVAL
    o = aao.default_opts()
    assert o.matvec == aao.AAO_MATVEC_NTT and o.use_graphs == 1 and o.cocg_threads == 0
