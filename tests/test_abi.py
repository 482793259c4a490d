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


C_PROGRAM = r"""
#include <stdio.h>
#include "lfmm.h"
/* the boundary from plain C: the header is C11, every call takes plain
 * pointers and sizes; only the host-only helper runs without a device */
int main(void) {
    double t[32], w[32];
    if (lfmm_gauss_laguerre(32, t, w) != LFMM_OK) return 2;
    if (lfmm_gauss_laguerre(0, t, w) != LFMM_EINVAL) return 3;
    double m0 = 0.0, m1 = 0.0;
    for (int i = 0; i < 32; ++i) { m0 += w[i]; m1 += w[i] * t[i]; }
    printf("%.17g %.17g\n", m0, m1);   /* int e^{-t} = 1, int t e^{-t} = 1 */
    lfmm_destroy(NULL);                /* NULL-safe */
    return 0;
}
"""


def test_header_is_plain_c_and_links(tmp_path):
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib = os.path.realpath(binding.library_path())
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", os.path.dirname(lib), "-llfmm", "-Wl,-rpath," + os.path.dirname(lib),
                    "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert abs(float(out[0]) - 1.0) < 1e-13 and abs(float(out[1]) - 1.0) < 1e-13
