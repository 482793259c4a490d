"""Building blocks of the CUDA kernels that are host-and-device code in
``lfmm_internal.cuh``, compiled for the host with nvcc and checked against
independent references (no GPU needed):

* the Morton interleave of the box keys, against bit-by-bit interleaving;
* the packed (n, m, Re/Im) index of every expansion, against its definition;
* the irregular solid harmonics T_N^mu of every M2L table and the regular
  ones U_n^m of the shift operators and P2M / L2P, against scipy's associated
  Legendre functions (T_N^mu = (N-mu)! P_N^mu(cos t) / r^{N+1},
  U_n^m = r^n P_n^m(cos t) e^{i m f} / (n+m)!, P without the Condon-Shortley
  phase)."""
import os
import shutil
import subprocess
from math import factorial

import numpy as np
import pytest
from scipy.special import lpmv

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_1908_10863_gb300", "csrc", "lfmm_internal.cuh")

PROGRAM = r'''
#include <cstdio>
#include <vector>
#include "%s"
int main() {
    char op;
    while (scanf(" %%c", &op) == 1) {
        if (op == 'M') {
            unsigned v; if (scanf("%%u", &v) != 1) return 1;
            unsigned s = lf_spread3(v);
            printf("%%u %%u\n", s, lf_compact3(s));
        } else if (op == 'D') {
            int p; if (scanf("%%d", &p) != 1) return 1;
            for (int j = 0; j < lf_nc(p); ++j) {
                int n, m, im;
                lf_decode(p, j, n, m, im);
                printf("%%d %%d %%d %%d %%d\n", n, m, im, lf_re(n, m), im ? lf_im(p, n, m) : -1);
            }
        } else if (op == 'T') {
            double rho, z; int nmax;
            if (scanf("%%lf %%lf %%d", &rho, &z, &nmax) != 3) return 1;
            const int ld = nmax + 1;
            std::vector<double> t((size_t)ld * ld, 0.0);
            for (int mu = 0; mu <= nmax; ++mu) lf_theta_column(rho, z, mu, nmax, 1.0, t.data(), ld);
            for (int N = 0; N <= nmax; ++N)
                for (int mu = 0; mu <= N; ++mu) printf("%%.17g\n", t[(size_t)N * ld + mu]);
        } else if (op == 'U') {
            int p; double x, y, z;
            if (scanf("%%d %%lf %%lf %%lf", &p, &x, &y, &z) != 4) return 1;
            std::vector<double> re(lf_nre(p)), im(lf_nre(p));
            lf_regular<double>(p, x, y, z, re.data(), im.data());
            for (int n = 0; n <= p; ++n)
                for (int m = 0; m <= n; ++m) printf("%%.17g %%.17g\n", re[lf_re(n, m)], im[lf_re(n, m)]);
        }
    }
    return 0;
}
''' % HDR.replace("\\", "/")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("devmath")
    src, exe = d / "devmath.cu", d / "devmath"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), str(src)], check=True, capture_output=True)

    def call(text):
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
        return [ln.split() for ln in out.strip().splitlines()]
    return call


def _pbar(m, n, x):
    return (-1.0) ** m * lpmv(m, n, x)  # scipy includes the Condon-Shortley phase


def test_morton_interleave(run):
    vals = list(range(0, 1024, 7)) + [1023, 512, 1]
    rows = run("".join("M %d\n" % v for v in vals))
    for v, (s, back) in zip(vals, rows):
        ref = 0
        for b in range(10):
            ref |= ((v >> b) & 1) << (3 * b)
        assert int(s) == ref and int(back) == v


@pytest.mark.parametrize("p", [1, 4, 10, 20])
def test_packed_index(run, p):
    rows = run("D %d\n" % p)
    nre = (p + 1) * (p + 2) // 2
    seen = set()
    for j, (n, m, im, jre, jim) in enumerate(map(lambda r: tuple(map(int, r)), rows)):
        assert 0 <= m <= n <= p and (im == 0 or m >= 1)
        if im:
            assert j == nre + n * (n - 1) // 2 + m - 1 == jim
        else:
            assert j == n * (n + 1) // 2 + m == jre
        seen.add((n, m, im))
    assert len(seen) == (p + 1) ** 2


@pytest.mark.parametrize("rho,z", [(0.0, 2.0), (1.0, 2.0), (2.0 ** 0.5, 3.0), (3.0, 0.3), (0.7, -1.9)])
def test_irregular_solid_harmonics(run, rho, z):
    nmax = 20
    vals = np.array([float(r[0]) for r in run("T %r %r %d\n" % (rho, z, nmax))])
    r = np.hypot(rho, z)
    k = 0
    for N in range(nmax + 1):
        row = np.array([factorial(N - mu) * _pbar(mu, N, z / r) / r ** (N + 1) for mu in range(N + 1)])
        got = vals[k:k + N + 1]
        k += N + 1
        assert np.max(np.abs(got - row)) <= 1e-13 * np.max(np.abs(row)), (N, got, row)


@pytest.mark.parametrize("x,y,z", [(0.3, -0.2, 0.4), (0.0, 0.0, -0.25), (-0.25, 0.25, 0.25), (1.2, 0.7, -0.9)])
def test_regular_solid_harmonics(run, x, y, z):
    p = 20
    vals = np.array([[float(a), float(b)] for a, b in run("U %d %r %r %r\n" % (p, x, y, z))])
    r = np.sqrt(x * x + y * y + z * z)
    phi = np.arctan2(y, x)
    k = 0
    for n in range(p + 1):
        ref = np.array([r ** n * _pbar(m, n, z / r) * np.exp(1j * m * phi) / factorial(n + m) for m in range(n + 1)])
        got = vals[k:k + n + 1, 0] + 1j * vals[k:k + n + 1, 1]
        k += n + 1
        assert np.max(np.abs(got - ref)) <= 1e-13 * max(np.max(np.abs(ref)), 1e-300), (n, got, ref)
