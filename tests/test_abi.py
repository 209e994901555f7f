"""The C-ABI library builds, loads and exports every entry point that
include/lyap.h declares (CPU only: no compute calls)."""
import ctypes

import pytest

import paper_2312_08201_gb300 as ly


@pytest.fixture(scope="module")
def lib():
    ly.build()
    return ly.load()


def test_header_declares_the_paper_boundary():
    names = ly.header_functions()
    for fn in ["lyap_seed_factor", "lyap_param_solve", "lyap_trace_EX", "lyap_grad", "lyap_serve_submit",
               "lyap_serve_poll", "lyap_ctx_create", "lyap_strerror"]:
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in ly.header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    assert set(ly.header_functions()) == set(ly._SIGS), set(ly.header_functions()) ^ set(ly._SIGS)


def test_opts_defaults_follow_paper_settings(lib):
    o = ly.default_opts()
    assert o.maxit == 300 and o.s == 10  # §4, Ex. 1 settings (also p̄ = 50)
    assert o.m == 40 and o.precision == ly.FP64 and o.pbar == 50 and o.inner_tol == 1e-3
    assert 0 < o.tol <= 1e-10
    assert o.residual == ly.RESID_TC


def test_strerror(lib):
    assert lib.lyap_strerror(0) == b"ok"
    assert b"invalid" in lib.lyap_strerror(ly.EINVAL)
    assert lib.lyap_strerror(12345) == b"unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    # argument validation happens before any device work
    assert lib.lyap_ctx_create(0, None) == ly.EINVAL
    assert lib.lyap_seed_free(None) == ly.EINVAL
    assert lib.lyap_trace_EX(None, 0, None, 0, None, None, None) == ly.EINVAL
    o = ly.default_opts()
    h = ctypes.c_void_p()
    assert lib.lyap_seed_factor(None, 4, 1, 1, None, None, None, None, None, 0, ctypes.byref(o), ctypes.byref(h), None) == ly.EINVAL
