"""The C-ABI library loads and exports every symbol include/lfmm.h declares
(no device needed), and its host-only quadrature helper is right."""
import ctypes
import os
import re

import numpy as np
import pytest
from scipy.special import roots_laguerre

from paper_1908_10863_gb300 import lfmm as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lfmm.h")).read()
    return sorted(set(re.findall(r"\b(lfmm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["lfmm_create", "lfmm_build", "lfmm_evaluate", "lfmm_destroy", "lfmm_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == _declared()


def test_library_path_is_in_tree():
    path = os.path.realpath(binding.library_path())
    assert path.startswith(os.path.realpath(ROOT))
    assert os.path.exists(path)


@pytest.mark.parametrize("Q", [16, 32, 64, 128])
def test_gauss_laguerre_rule(Q):
    t, w = binding.gauss_laguerre(Q)
    t2, w2 = roots_laguerre(Q)
    assert np.max(np.abs(t - t2) / t2) < 1e-12
    big = w2 > 1e-30
    assert np.max(np.abs(w - w2)[big] / w2[big]) < 1e-11
    # exact for polynomials of degree 2Q-1
    for k in (0, 1, 5, 2 * Q - 1 if Q <= 32 else 40):
        from math import factorial, lgamma, exp
        exact = factorial(k) if k < 170 else exp(lgamma(k + 1))
        assert np.sum(w * t ** k) == pytest.approx(exact, rel=1e-10)


def test_gauss_laguerre_rejects_bad_order():
    with pytest.raises(binding.LfmmError):
        binding.gauss_laguerre(0)


def test_batch_create_rejects_bad_arguments_without_a_device():
    # argument checks come before any CUDA call
    lib = binding.load()
    h = ctypes.c_void_p()
    assert lib.lfmm_batch_create(None, 3, None, 1, ctypes.byref(h)) == binding.EINVAL
    assert lib.lfmm_batch_create((ctypes.c_void_p * 1)(None), 1, None, 1, ctypes.byref(h)) == binding.EINVAL
    assert lib.lfmm_batch_create((ctypes.c_void_p * 1)(None), 0, None, 1, None) == binding.EINVAL
    assert not h.value
    lib.lfmm_batch_destroy(None)
    assert lib.lfmm_batch_last_error(None) == b"null batch"
