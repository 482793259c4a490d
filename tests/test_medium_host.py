"""The medium set-up of the CUDA library (host code, no device needed):
every component's polarization map, interface, leading term C e^{-k zeta}
and remainder rate zeta_r, as ``lfmm_medium_components`` reports them,
against the oracle's densities and the paper's exponent definitions."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LfmmError
from paper_1908_10863_gb300.lfmm import medium_components

MEDIA = [([], [2.0]), ([0.0], [3.0, 11.0]), ([0.0, -1.2], [1.0, 5.0, 10.0]), ([0.0, -1.2], [1.0, 80.0, 2.0]),
         ([0.0, -1.2], [21.2, 47.5, 62.8]), ([0.0, -0.6, -1.2], [2.0, 7.0, 1.5, 12.0]),
         ([0.0, -0.55, -1.2371], [1.0, 80.0, 2.0, 5.0]), ([0.3, -0.2, -1.0], [5.0, 1.0, 30.0, 2.0]),
         ([0.0, -0.6, -1.2, -1.8], [2.0, 7.0, 1.5, 12.0, 4.0]),
         ([0.0, -0.45, -1.1, -1.6], [1.0, 40.0, 3.0, 9.0, 1.5])]


def _exponent(d, l, lp, a, b, z, zp):
    # eqs. generalcomponents / zexponential: the target side e^{-k(z - d_l)}
    # (a = 1) or e^{-k(d_{l-1} - z)} (a = 2), the source side e^{-k(z' - d_lp)}
    # (b = 1) or e^{-k(d_{lp-1} - z')} (b = 2)
    ht = (z - d[l]) if a == 1 else (d[l - 1] - z)
    hs = (zp - d[lp]) if b == 1 else (d[lp - 1] - zp)
    return ht + hs


def _inside(d, l, rng):
    top = d[l - 1] if l > 0 else d[0] + 1.0
    bot = d[l] if l < len(d) else d[-1] - 1.0
    return rng.uniform(bot + 0.01 * (top - bot), top - 0.01 * (top - bot))


@pytest.mark.parametrize("d,eps", MEDIA)
def test_components_match_oracle(d, eps):
    L = len(d)
    comps = medium_components(d, eps)
    free = [c for c in comps if c["is_free"]]
    react = [c for c in comps if not c["is_free"]]
    assert [c["l"] for c in free] == list(range(L + 1)) and all(c["lp"] == c["l"] for c in free)
    assert len(react) == (2 * L) ** 2
    rng = np.random.default_rng(61)
    dmin = min([d[j - 1] - d[j] for j in range(1, L)], default=1.0)
    for c in react:
        l, lp, a, b = c["l"], c["lp"], c["a"], c["b"]
        assert not ((a == 1 and l == L) or (a == 2 and l == 0) or (b == 1 and lp == L) or (b == 2 and lp == 0))
        assert c["iface"] == (d[l] if a == 1 else d[l - 1])
        # the polarization map reproduces the paper's exponent for any pair of the two layers
        for _ in range(4):
            z, zp = _inside(d, l, rng), _inside(d, lp, rng)
            zpp = c["s"] * zp + c["o"]
            h = (z - zpp) if a == 1 else (zpp - z)
            assert h == pytest.approx(_exponent(d, l, lp, a, b, z, zp), abs=1e-12)
        # the leading term is the large-k limit of the density
        zeta, zr, C = c["zeta"], c["zeta_r"], c["C"]
        sig = lambda k: oracle.sigma(d, eps, k, lp)[l, a - 1, b - 1]
        if zr < 0:  # no remainder: the density is exactly C e^{-k zeta}
            for k in (0.01, 0.5, 3.0):
                assert sig(k) * np.exp(k * zeta) == pytest.approx(C, rel=1e-12, abs=1e-14)
            continue
        assert zr >= zeta + 2.0 * dmin - 1e-12
        k1 = min(40.0 / (zr - zeta), 600.0 / max(zeta, 1e-300))
        assert abs(sig(k1) * np.exp(k1 * zeta) - C) <= 1e-10 * (1.0 + abs(C))
        # the remainder, scaled by e^{k zeta_r}, stays bounded while the subtraction is accurate
        for k in np.linspace(0.0, 20.0 / (zr - zeta), 9)[1:]:
            g = (sig(k) * np.exp(k * zeta) - C) * np.exp(k * (zr - zeta))
            assert abs(g) < 50.0 * (1.0 + abs(C)), (l, lp, a, b, k, g)


@pytest.mark.parametrize("d,eps", [([0.0, -1.0, -2.0, -3.0, -4.0], [1.0] * 6), ([0.0, -1.0, -0.5], [1.0] * 4),
                                   ([0.0, -1.0], [1.0, -2.0, 3.0]), ([0.0, np.nan], [1.0, 2.0, 3.0])])
def test_invalid_media_rejected(d, eps):
    with pytest.raises(LfmmError):
        medium_components(d, eps)


def test_short_output_is_refused_with_the_full_count():
    # four layers have 4 free + 36 reaction components; a buffer for 10 rows
    # is refused (nothing written) and the count still comes back
    import ctypes
    from paper_1908_10863_gb300 import lfmm
    d = np.array([0.0, -0.6, -1.2]); eps = np.array([2.0, 7.0, 1.5, 12.0])
    dp = ctypes.POINTER(ctypes.c_double)
    out = np.full((10, len(lfmm.MEDIUM_COLS)), 7.0)
    n = ctypes.c_int(-1)
    st = lfmm.load().lfmm_medium_components(d.ctypes.data_as(dp), 3, eps.ctypes.data_as(dp),
                                            out.ctypes.data_as(dp), 10, ctypes.byref(n))
    assert st == lfmm.EINVAL and n.value == 40
    assert np.all(out == 7.0)
    assert len(medium_components(d, eps)) == 40
