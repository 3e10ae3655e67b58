"""The C ABI library loads and exports every entry point include/ezo.h
declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ezo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ezo_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_10783_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["ezo_check_collision", "ezo_hit_and_run", "ezo_batch_create", "ezo_batch_run",
                 "ezo_batch_run_path", "ezo_robot_create", "ezo_env_create", "ezo_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_default_and_last_error_without_gpu(lib):
    from paper_2504_10783_gb300 import ezo
    p = ezo.Params.make()
    assert (p.eps, p.delta, p.tau, p.n_p, p.n_f, p.n_b, p.n_mix, p.n_it_max) == (0.05, 0.05, 0.5, 10000, 10, 10, 60, 50)
    ezo.lib().ezo_last_error.restype = ctypes.c_char_p
    assert isinstance(ezo.lib().ezo_last_error(), bytes)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_2504_10783_gb300 import ezo
    out = ctypes.c_void_p()
    st = ezo.lib().ezo_env_create(-1, None, ctypes.byref(out))
    assert st == 1 and not out.value
    st = ezo.lib().ezo_robot_create(0, None, None, None, None, None, None, 0, None, None, None, 0, None, None,
                                    ctypes.byref(out))
    assert st == 1
    assert b"n must be" in ezo.lib().ezo_last_error()
    st = ezo.lib().ezo_probe_fp32_fma(None, None)
    assert st == 1
    assert b"tflops" in ezo.lib().ezo_last_error()
    st = ezo.lib().ezo_surrogate_status(None, None, 0, None)
    assert st == 1
