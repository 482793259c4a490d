"""The four- and five-layer density routines of the CUDA library (``lf_sigma_solve`` and
the coupling-series remainder ``lf_sigma_rem<true>``, host-and-device code in
``lfmm_internal.cuh``) compiled for the host and checked against the oracle's
independent solve of the interface problem.  No GPU is needed: nvcc compiles
the header's host side."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_1908_10863_gb300", "csrc", "lfmm_internal.cuh")

PROGRAM = r'''
#include <cstdio>
#include <cstdlib>
#include "%s"
// stdin: L, d[L], eps[L+1], then lines "l lp a b C zeta zeta_r nterm nk k..."
// stdout: per k, sigma and the scaled remainder
int main() {
    int L; if (scanf("%%d", &L) != 1) return 1;
    double d[LFMM_MAXL], e[LFMM_MAXL + 1];
    for (int j = 0; j < L; ++j) if (scanf("%%lf", &d[j]) != 1) return 1;
    for (int j = 0; j <= L; ++j) if (scanf("%%lf", &e[j]) != 1) return 1;
    int l, lp, a, b, nterm, nk;
    double C, zeta, zr;
    while (scanf("%%d %%d %%d %%d %%lf %%lf %%lf %%d %%d", &l, &lp, &a, &b, &C, &zeta, &zr, &nterm, &nk) == 9) {
        LfmmComp c = {};
        c.l = l; c.lp = lp; c.a = a; c.b = b; c.nif = L; c.C = C; c.zeta = zeta; c.zeta_r = zr; c.nterm = nterm;
        for (int j = 0; j < L; ++j) c.md[j] = d[j];
        for (int j = 0; j <= L; ++j) c.me[j] = e[j];
        for (int i = 0; i < nk; ++i) {
            double k; if (scanf("%%lf", &k) != 1) return 1;
            printf("%%.17g %%.17g\n", lf_sigma_solve(c, k), lf_sigma_rem<true>(c, k));
        }
    }
    return 0;
}
''' % HDR.replace("\\", "/")

MEDIA = [([0.0, -0.6, -1.2], [2.0, 7.0, 1.5, 12.0]), ([0.0, -0.55, -1.2371], [1.0, 80.0, 2.0, 5.0]),
         ([0.3, -0.2, -1.0], [5.0, 1.0, 30.0, 2.0]),
         ([0.0, -0.6, -1.2, -1.8], [2.0, 7.0, 1.5, 12.0, 4.0]),
         ([0.0, -0.45, -1.1, -1.6], [1.0, 40.0, 3.0, 9.0, 1.5])]


@pytest.fixture(scope="module")
def host_program(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("density")
    src, exe = d / "density.cu", d / "density"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), str(src)], check=True, capture_output=True)
    return str(exe)


def _components(L):
    return [(l, lp, a, b) for l in range(L + 1) for lp in range(L + 1) for a in (1, 2) for b in (1, 2)
            if not (a == 1 and l == L) and not (a == 2 and l == 0)
            and not (b == 1 and lp == L) and not (b == 2 and lp == 0)]


@pytest.mark.parametrize("d,eps", MEDIA)
def test_density_and_remainder_series_match_oracle(host_program, d, eps):
    L = len(d)
    dmin = min(d[j - 1] - d[j] for j in range(1, L))
    ks = [0.01, 0.3, 1.0, 3.0, 7.0, 15.0, 40.0, 120.0]
    g = lambda v: "%.17g" % float(v)
    lines = ["%d" % L, " ".join(map(g, d)), " ".join(map(g, eps))]
    rows = []
    for (l, lp, a, b) in _components(L):
        i_s = lp if b == 1 else lp - 1
        i_t = l if a == 1 else l - 1
        zeta = abs(d[i_s] - d[i_t])
        zr = zeta + 2.0 * dmin
        k1 = 30.0 / dmin
        C = oracle.sigma(d, eps, k1, lp)[l, a - 1, b - 1] * np.exp(k1 * zeta)  # leading constant, from the oracle
        nterm = int(np.ceil(zr / dmin)) + 1
        lines.append("%d %d %d %d %s %s %s %d %d %s" % (l, lp, a, b, g(C), g(zeta), g(zr), nterm, len(ks),
                                                       " ".join(map(g, ks))))
        rows.append((l, lp, a, b, C, zeta, zr))
    out = subprocess.run([host_program], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    vals = np.array([[float(x) for x in ln.split()] for ln in out.stdout.strip().splitlines()])
    assert vals.shape == (len(rows) * len(ks), 2)
    for i, (l, lp, a, b, C, zeta, zr) in enumerate(rows):
        for j, k in enumerate(ks):
            sig, rem = vals[i * len(ks) + j]
            ref = oracle.sigma(d, eps, k, lp)[l, a - 1, b - 1]
            assert abs(sig - ref) <= 1e-13 * max(abs(ref), 1e-300) + 1e-300, (l, lp, a, b, k, sig, ref)
            assert np.isfinite(rem) and abs(rem) < 1e3, (l, lp, a, b, k, rem)
            if k * 2.0 * dmin < 8.0:  # where the plain subtraction still holds 1e-11
                direct = (ref * np.exp(k * zeta) - C) * np.exp(k * (zr - zeta))
                assert abs(rem - direct) <= 1e-9 * (1.0 + abs(direct)), (l, lp, a, b, k, rem, direct)
