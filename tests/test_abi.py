"""C-ABI library: builds, loads, exports every declared symbol, and the host-only
entry points behave as documented (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2511_12051_gb300 import build as plk_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libplk():
    path = plk_build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "plk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plk_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(libplk):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libplk, n), n


def test_binding_covers_the_header():
    from paper_2511_12051_gb300 import plk
    assert sorted(plk.EXPORTS) == declared_functions()


def test_glrt_threshold_library_matches_oracle(libplk):
    import oracle
    f = libplk.plk_glrt_threshold
    f.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    for alpha in (1e-4, 1e-3, 0.05):
        for n in (1, 2, 5, 10, 15, 18, 30, 60, 120, 400):
            c = ctypes.c_double()
            assert f(alpha, n, ctypes.byref(c)) == 0
            ref = oracle.glrt_threshold(alpha, n)
            assert abs(c.value - ref) <= 1e-10 * ref, (alpha, n, c.value, ref)
            # the kernels compare in single precision: the float threshold must agree
            assert np.float32(c.value) == np.float32(ref)
    c = ctypes.c_double()
    assert f(0.0, 10, ctypes.byref(c)) == 1
    assert f(0.5, 0, ctypes.byref(c)) == 1


def test_host_helpers(libplk):
    from paper_2511_12051_gb300 import plk
    p = plk.default_params()
    assert p.alpha == pytest.approx(1e-3) and p.mu == pytest.approx(0.99) and p.max_iter == 100 and p.err_max == pytest.approx(0.1)
    assert plk.mask_words((5, 11, 3, 6)) == 1
    assert plk.mask_words((19, 37, 3, 6)) == 11
    Ho, Wo = ctypes.c_int(), ctypes.c_int()
    assert plk.lib().plk_output_shape(4096, 16384, plk.window((5, 11, 3, 6)), ctypes.byref(Ho), ctypes.byref(Wo)) == 0
    assert (Ho.value, Wo.value) == (1365, 2730)
    # even windows and zero strides are rejected
    assert plk.lib().plk_output_shape(10, 10, plk.window((4, 11, 1, 1)), ctypes.byref(Ho), ctypes.byref(Wo)) == 1
    assert plk.lib().plk_output_shape(10, 10, plk.window((5, 11, 0, 1)), ctypes.byref(Ho), ctypes.byref(Wo)) == 1


def test_null_context_is_rejected(libplk):
    from paper_2511_12051_gb300 import plk
    L = plk.lib()
    assert L.plk_amp_stats(None, None, 1, 1, 1, None, None, 0) == 1
    assert L.plk_phase_link(None, None, 2, 1, 0, None, None, None, None, None) == 1
    assert b"null ctx" in L.plk_last_error(None)


def test_glrt_threshold_for_real_looks_matches_oracle(libplk):
    """plk_glrt_threshold_looks (decaying image weights, nu = W1^2 / W2) against
    the oracle's F quantile (scipy), and equal to the integer form at integer nu."""
    import oracle
    f = libplk.plk_glrt_threshold_looks
    f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    for alpha in (1e-3, 0.05):
        for nu in (1.0, 1.7, 4.25, 9.18, 14.88, 17.45, 29.5):
            c = ctypes.c_double()
            assert f(alpha, nu, ctypes.byref(c)) == 0
            ref = oracle.glrt_threshold_real(alpha, nu)
            assert abs(c.value - ref) <= 1e-9 * ref, (alpha, nu, c.value, ref)
            assert np.float32(c.value) == np.float32(ref)
    c = ctypes.c_double()
    assert f(1e-3, 0.5, ctypes.byref(c)) == 1 and f(1.5, 3.0, ctypes.byref(c)) == 1   # PLK_EINVAL


def test_device_allocation_counter_is_host_only(libplk):
    f = libplk.plk_device_allocations
    f.argtypes = []
    f.restype = ctypes.c_int64
    assert f() == 0   # nothing allocated in a process that made no context
