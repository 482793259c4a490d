"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form printed in the paper, a textbook identity evaluated by scipy, a
physical invariant, or an independent evaluation route.
"""
import json
import os
from math import factorial, pi, sqrt

import numpy as np
import pytest
from scipy.special import lpmv

import oracle
from oracle import expansions

HERE = os.path.dirname(os.path.abspath(__file__))
D3 = [0.0, -1.2]
MEDIA = [[1.0, 5.0, 10.0], [1.0, 80.0, 2.0], [21.2, 47.5, 62.8]]
COMPONENTS3 = [(l, lp, a, b) for l in range(3) for lp in range(3) for a in (1, 2) for b in (1, 2)
               if not (a == 1 and l == 2) and not (a == 2 and l == 0)
               and not (b == 1 and lp == 2) and not (b == 2 and lp == 0)]


def test_sixteen_components_for_three_layers():
    # Section 4: three free-space and sixteen reaction components for 3 layers
    assert len(COMPONENTS3) == 16


@pytest.mark.parametrize("eps", MEDIA)
@pytest.mark.parametrize("k", [0.05, 0.3, 1.0, 2.5, 9.0])
def test_sigma_solve_matches_appendix_closed_forms(eps, k):
    # Appendix A, densitythreelayer1-3 (with the kappa / sigma22_22 corrections)
    for (l, lp, a, b) in COMPONENTS3:
        s = oracle.sigma(D3, eps, k, lp)[l, a - 1, b - 1]
        c = oracle.sigma3_closed(D3, eps, k, l, lp, a, b)
        assert abs(s - c) <= 1e-14 * max(1.0, abs(c)), (l, lp, a, b, s, c)


def test_printed_typos_disagree_with_solve():
    # The printed kappa (with (eps2-eps1)) and the printed sigma^{22}_{22} are
    # inconsistent with the interface problem; the corrected forms are used.
    e0, e1, e2 = 1.0, 5.0, 10.0
    k = 1.0
    x = np.exp(D3[1] * k)
    kap_printed = 0.5 * ((e0 + e1) * (e1 + e2) + (e0 - e1) * (e2 - e1) * x * x)
    s11_printed = (e1 - e2) * (e1 + e0) / (2 * kap_printed)
    s_solve = oracle.sigma(D3, [e0, e1, e2], k, 1)[1, 0, 0]
    assert abs(s11_printed - s_solve) > 1e-3
    kap = 0.5 * ((e0 + e1) * (e1 + e2) + (e0 - e1) * (e1 - e2) * x * x)
    s22_printed = ((e1 - e0) * (e1 + e2) + (e0 + e1) * (e2 - e1) * x * x) / (2 * kap)
    assert abs(s22_printed - oracle.sigma(D3, [e0, e1, e2], k, 2)[2, 1, 1]) > 1e-3


def test_sigma_limits():
    # equal permittivities: same-layer densities vanish, and the cross-layer
    # components add up to the plain Coulomb kernel 1/|r - r'|
    for lp in range(3):
        s = oracle.sigma(D3, [3.0, 3.0, 3.0], 0.7, lp)
        assert np.max(np.abs(s[lp])) < 1e-15
    zr = {0: 0.4, 1: -0.5, 2: -1.9}
    for l in range(3):
        for lp in range(3):
            r = np.array([0.1, 0.2, zr[l]]); rp = np.array([-0.3, 0.05, zr[lp] + 0.1])
            u, g = oracle.reaction_pair(D3, [3.0, 3.0, 3.0], l, lp, r, rp, mode=oracle.MODE_QUAD)
            ref = 0.0 if l == lp else 1.0 / np.linalg.norm(r - rp)
            assert u == pytest.approx(ref, abs=1e-13)
    # two layers: constant reflection / transmission coefficients (image charge)
    e0, e1 = 2.0, 7.0
    for k in (0.1, 1.0, 10.0):
        s0 = oracle.sigma([0.0], [e0, e1], k, 0)
        s1 = oracle.sigma([0.0], [e0, e1], k, 1)
        assert s0[0, 0, 0] == pytest.approx((e0 - e1) / (e0 + e1), abs=1e-15)
        assert s0[1, 1, 0] == pytest.approx(2 * e0 / (e0 + e1), abs=1e-15)
        assert s1[1, 1, 1] == pytest.approx((e1 - e0) / (e0 + e1), abs=1e-15)
        assert s1[0, 0, 1] == pytest.approx(2 * e1 / (e0 + e1), abs=1e-15)
    # middle permittivity -> 0 or -> infinity (Appendix A closed forms' limits)
    assert oracle.sigma(D3, [1.0, 1e-9, 10.0], 1.0, 0)[0, 0, 0] == pytest.approx(1.0, abs=1e-7)
    assert oracle.sigma(D3, [1.0, 1e9, 10.0], 1.0, 0)[0, 0, 0] == pytest.approx(-1.0, abs=1e-7)


def _K_closed(N, mu, rho, z):
    # int_0^inf J_mu(k rho) k^N e^{-kz} dk = (N-mu)! Pbar_N^mu(z/r) / r^{N+1}
    # (Pbar without Condon-Shortley phase); scipy's lpmv carries the phase.
    r = np.hypot(rho, z)
    return factorial(N - mu) * (-1) ** mu * lpmv(mu, N, z / r) / r ** (N + 1)


@pytest.mark.parametrize("rho,z", [(0.0, 0.7), (0.3, 0.5), (0.5, 0.5), (0.2, 1.3)])
def test_sommerfeld_sigma_one_closed_form(rho, z):
    # sigma == 1: the closed form quoted before Table 3.1 (eq. wavefunspectralform)
    for N in range(0, 21, 3):
        for mu in range(0, N + 1, 2):
            ref = _K_closed(N, mu, rho, z)
            got = oracle.sommerfeld_K(D3, MEDIA[0], 0, 0, 1, 1, N, mu, rho, z, sigma_one=True)
            scale = max(abs(_K_closed(N, m2, rho, z)) for m2 in range(N + 1))
            assert abs(got - ref) <= 1e-11 * scale, (N, mu, got, ref)


def test_table31_cases_rho_below_z():
    # Table 3.1, sigma == 1, z = 0.001; the real-axis quadrature applies when
    # rho <= z (the paper switches to the contour form for rho > z).
    g = json.load(open(os.path.join(HERE, "golden", "table31_quadrature_cases.json")))
    z = g["z"]
    n_checked = 0
    for c in g["cases"]:
        if c["rho"] > z:
            continue
        n, m, rho = c["n"], c["m"], c["rho"]
        r = np.hypot(rho, z)
        # paper's normalisation: r^n I_nm = sqrt(4 pi/(2n+1)) Phat_n^m(z/r)/r
        phat = (-1) ** m * sqrt((2 * n + 1) / (4 * pi) * factorial(n - m) / factorial(n + m)) * lpmv(m, n, z / r)
        ref = sqrt(4 * pi / (2 * n + 1)) * phat / r
        K = oracle.sommerfeld_K(D3, MEDIA[0], 0, 0, 1, 1, n, m, rho, z, sigma_one=True, tol=1e-14)
        got = r ** n * K / sqrt(factorial(n + m) * factorial(n - m))
        # at least as accurate as the paper's mixed DE-SE result for the case
        assert abs(got - ref) <= max(abs(c["desE_error"]), 1e-13 * abs(ref)), (c, got, ref)
        n_checked += 1
    assert n_checked == 4


def test_legendre_matches_scipy():
    for n in range(0, 30, 4):
        for m in range(0, n + 1, 3):
            for x in (-0.9, -0.2, 0.3, 0.99):
                ref = (-1) ** m * lpmv(m, n, x)
                assert oracle.legendre_nocs(n, m, x) == pytest.approx(ref, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("eps", MEDIA)
def test_image_series_matches_quadrature_integrals(eps):
    # two independent evaluations of K_{N,mu}: closed-form image series of the
    # Appendix A densities vs adaptive quadrature of the spectral-solve density
    rng = np.random.default_rng(7)
    for (l, lp, a, b) in COMPONENTS3[::3]:
        for _ in range(2):
            rho, z = rng.uniform(0.0, 0.6), rng.uniform(0.4, 1.5)
            for N, mu in [(0, 0), (1, 1), (4, 2), (9, 5)]:
                qv = oracle.sommerfeld_K(D3, eps, l, lp, a, b, N, mu, rho, z)
                iv = oracle.sommerfeld_K_images(D3, eps, l, lp, a, b, N, mu, rho, z)
                scale = abs(oracle.sommerfeld_K_images(D3, eps, l, lp, a, b, N, 0, rho, z)) + abs(iv)
                assert abs(qv - iv) <= 1e-11 * scale, (l, lp, a, b, N, mu, qv, iv)


def _mixed_points(rng, n):
    zr = {0: (0.1, 1.1), 1: (-1.1, -0.1), 2: (-2.3, -1.3)}
    lay = rng.integers(0, 3, n).astype(np.int32)
    xyz = np.zeros((n, 3))
    xyz[:, :2] = rng.uniform(-0.5, 0.5, (n, 2))
    for i in range(n):
        xyz[i, 2] = rng.uniform(*zr[int(lay[i])])
    return xyz, lay


@pytest.mark.parametrize("eps", MEDIA[:2])
def test_direct_quadrature_matches_image_series(eps):
    rng = np.random.default_rng(11)
    xyz, lay = _mixed_points(rng, 60)
    q = rng.uniform(-1, 1, 60)
    p0, f0 = oracle.direct(D3, eps, xyz, lay, q, mode=oracle.MODE_QUAD)
    p1, f1 = oracle.direct(D3, eps, xyz, lay, q, mode=oracle.MODE_IMAGES)
    assert oracle.err2(p1, p0) < 1e-11
    assert np.max(np.abs(f1 - f0)) < 1e-10 * np.max(np.abs(f1))


@pytest.mark.parametrize("eps", [MEDIA[0], MEDIA[1]])
def test_quadrature_next_to_interfaces_matches_image_series(eps):
    # Charges 1e-5 .. 1e-2 from an interface, the regime of the near field
    # (Section 3.1's components with a short exponent distance h): the
    # quadrature of the spectral-solve density must agree with the exact
    # three-layer image series in potential and gradient, for every pair of
    # layers and every side of each interface.
    sides = [(0, lambda h: 0.0 + h), (1, lambda h: 0.0 - h), (1, lambda h: -1.2 + h), (2, lambda h: -1.2 - h)]
    worst = 0.0
    for ht in (1e-5, 1e-4, 1e-3, 1e-2):
        for hs in (1e-5, 1e-3):
            for lt, zt in sides:
                for ls, zs in sides:
                    for rho in (0.0, 0.03, 0.4, 1.0):
                        r = np.array([0.1, -0.2, zt(ht)])
                        rp = np.array([0.1 + rho * 0.6, -0.2 + rho * 0.8, zs(hs)])
                        uq, gq = oracle.reaction_pair(D3, eps, lt, ls, r, rp, mode=oracle.MODE_QUAD, tol=1e-13)
                        ui, gi = oracle.reaction_pair(D3, eps, lt, ls, r, rp, mode=oracle.MODE_IMAGES)
                        assert abs(uq - ui) <= 1e-10 * abs(ui) + 1e-13, (ht, hs, lt, ls, rho)
                        assert np.linalg.norm(gq - gi) <= 1e-10 * np.linalg.norm(gi) + 1e-13, (ht, hs, lt, ls, rho)
                        worst = max(worst, abs(uq - ui) / abs(ui))
    assert worst < 1e-10


def test_quadrature_reports_non_convergence():
    # A planted failure: the unsplit integral of J0(k rho) e^{-kh} (the sigma == 1
    # mode) at h = 1e-8 and rho = 1 spans ~1e9 Bessel oscillations, far beyond
    # the panel budget.  The oracle must refuse, not return the partial sum.
    r = np.array([0.0, 0.0, -0.6]); rp = np.array([1.0, 0.0, -0.6])
    d_near = [-0.6 + 5e-9, -1.2]
    with pytest.raises(oracle.OracleNotConverged):
        oracle.reaction_pair(d_near, MEDIA[0], 1, 1, r, rp, mode=oracle.MODE_SIGMA_ONE)
    xyz = np.array([r, rp]); lay = np.array([1, 1], np.int32)
    with pytest.raises(oracle.OracleNotConverged):
        oracle.direct(d_near, MEDIA[0], xyz, lay, np.ones(2), mode=oracle.MODE_SIGMA_ONE)
    # the same pair with the spectral-solve density converges (split form)
    u, g = oracle.reaction_pair(d_near, MEDIA[0], 1, 1, r, rp, mode=oracle.MODE_QUAD)
    ui, gi = oracle.reaction_pair(d_near, MEDIA[0], 1, 1, r, rp, mode=oracle.MODE_IMAGES)
    assert u == pytest.approx(ui, rel=1e-11)
    assert np.allclose(g, gi, rtol=1e-10, atol=1e-12 * np.linalg.norm(gi))


def test_homogeneous_medium_is_coulomb():
    rng = np.random.default_rng(5)
    n = 40
    xyz = rng.uniform(-1, 1, (n, 3))
    q = rng.uniform(-1, 1, n)
    p, f = oracle.direct([], [2.0], xyz, np.zeros(n, np.int32), q)
    diff = xyz[:, None, :] - xyz[None, :, :]
    R = np.linalg.norm(diff, axis=2)
    np.fill_diagonal(R, np.inf)
    ref = (q[None, :] / R).sum(1) / (4 * pi)
    E = (q[None, :, None] * diff / R[:, :, None] ** 3).sum(1) / (4 * pi)
    assert np.max(np.abs(p - ref)) < 1e-14 * np.max(np.abs(ref))
    assert np.max(np.abs(f - E)) < 1e-13 * np.max(np.abs(E))


def test_two_layer_image_charge():
    # one interface at z=0: the reaction field is one image charge scaled by
    # (eps_s - eps_o)/(eps_s + eps_o); across the interface the total field is
    # 2 eps_s/(eps_s+eps_o) times the free-space one
    e0, e1 = 3.0, 11.0
    rng = np.random.default_rng(3)
    n = 30
    lay = rng.integers(0, 2, n).astype(np.int32)
    xyz = rng.uniform(-1, 1, (n, 3))
    xyz[:, 2] = np.where(lay == 0, rng.uniform(0.05, 1.0, n), -rng.uniform(0.05, 1.0, n))
    q = rng.uniform(-1, 1, n)
    p, f = oracle.direct([0.0], [e0, e1], xyz, lay, q)
    eps = [e0, e1]
    ref = np.zeros(n)
    for i in range(n):
        s = 0.0
        for j in range(n):
            es, eo = eps[lay[j]], eps[1 - lay[j]]
            if lay[i] == lay[j]:
                if i != j:
                    s += q[j] / np.linalg.norm(xyz[i] - xyz[j])
                img = xyz[j] * np.array([1, 1, -1])
                s += q[j] * (es - eo) / (es + eo) / np.linalg.norm(xyz[i] - img)
            else:
                s += q[j] * 2 * es / (es + eo) / np.linalg.norm(xyz[i] - xyz[j])
        ref[i] = s / (4 * pi)
    assert np.max(np.abs(p - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("eps", MEDIA)
def test_reciprocity_eps_weighted(eps):
    # eps_l u_{l l'}(r, r') = eps_l' u_{l' l}(r', r)  (from the self-adjoint
    # form of the interface problem, eqs. Laplaceeqlayer, transmissioncond)
    rng = np.random.default_rng(9)
    zr = {0: (0.1, 1.1), 1: (-1.1, -0.1), 2: (-2.3, -1.3)}
    for l in range(3):
        for lp in range(3):
            r = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[l])])
            rp = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[lp])])
            u1, _ = oracle.reaction_pair(D3, eps, l, lp, r, rp)
            u2, _ = oracle.reaction_pair(D3, eps, lp, l, rp, r)
            free = 1.0 / np.linalg.norm(r - rp) if l == lp else 0.0
            assert eps[l] * (u1 + free) == pytest.approx(eps[lp] * (u2 + free), rel=1e-11)


def test_harmonic_away_from_sources():
    eps = MEDIA[0]
    h = 2e-3
    rp = np.array([0.1, -0.2, -0.5])
    for l, r in [(0, np.array([0.3, 0.1, 0.6])), (1, np.array([-0.2, 0.2, -0.9])), (2, np.array([0.0, 0.1, -1.8]))]:
        f = lambda x: oracle.reaction_pair(D3, eps, l, 1, x, rp, mode=oracle.MODE_IMAGES)[0]
        lap = -6 * f(r)
        for k in range(3):
            e = np.zeros(3); e[k] = h
            lap += f(r + e) + f(r - e)
        lap /= h * h
        assert abs(lap) < 1e-5 * abs(f(r)) / h ** 0 + 1e-4, (l, lap)


@pytest.mark.parametrize("eps", MEDIA[:2])
def test_transmission_conditions(eps):
    # eq. transmissioncond: u and eps du/dz continuous across each interface
    rp = np.array([0.05, -0.1, -0.45])
    q = 1.0
    for j, dj in enumerate(D3):
        above, below = j, j + 1
        x = np.array([0.2, 0.15, dj])
        def total(l, pt):
            u, g = oracle.reaction_pair(D3, eps, l, 1, pt, rp, mode=oracle.MODE_IMAGES)
            if l == 1:
                R = pt - rp
                u += 1 / np.linalg.norm(R)
                g = g - R / np.linalg.norm(R) ** 3
            return q * u, q * g
        ua, ga = total(above, x)
        ub, gb = total(below, x)
        assert ua == pytest.approx(ub, rel=1e-10)
        assert eps[above] * ga[2] == pytest.approx(eps[below] * gb[2], rel=1e-9)
        assert ga[0] == pytest.approx(gb[0], rel=1e-9)


def test_field_is_minus_gradient_of_potential():
    # E = -grad Phi: a zero-charge probe point moved by +-h in each direction
    rng = np.random.default_rng(21)
    xyz, lay = _mixed_points(rng, 25)
    q = rng.uniform(-1, 1, 25)
    eps = MEDIA[0]
    for probe, lp in [(np.array([0.12, -0.07, -0.52]), 1), (np.array([-0.2, 0.3, 0.45]), 0)]:
        pts = np.vstack([xyz, probe])
        lays = np.append(lay, lp).astype(np.int32)
        qs = np.append(q, 0.0)
        _, f = oracle.direct(D3, eps, pts, lays, qs, targets=[25], mode=oracle.MODE_IMAGES)
        h = 1e-5
        g = np.zeros(3)
        for k in range(3):
            vals = []
            for sgn in (1, -1):
                moved = pts.copy()
                moved[25, k] += sgn * h
                v, _ = oracle.direct(D3, eps, moved, lays, qs, targets=[25], mode=oracle.MODE_IMAGES)
                vals.append(v[0])
            g[k] = (vals[0] - vals[1]) / (2 * h)
        assert np.allclose(f[0], -g, rtol=1e-6, atol=1e-8 * np.max(np.abs(f[0])))


def test_paper_forward_recurrence_stability_regimes():
    # eq. recurrence on S^n I_nm with exact sigma == 1 seeds.  Stable when
    # rho >= 1.5 z; for rho < z rounding errors grow by many orders.
    P, S = 10, 1.0

    def table(rho, z):
        r = np.hypot(rho, z)
        T = np.zeros((2 * P + 1, 2 * P + 1))
        for n in range(2 * P + 1):
            for m in range(n + 1):
                T[n, m] = S ** n * _K_closed(n, m, rho, z) / sqrt(factorial(n + m) * factorial(n - m))
        return T

    for rho, z, stable in [(3.0, 1.0, True), (3.0, 2.0, True), (1.0, 3.0, False), (0.5, 2.0, False), (1.0, 6.0, False)]:
        ex = table(rho, z)
        got = oracle.forward_recurrence(P, S, rho, ex[:, 0], ex[:, 1])
        err = max(np.max(np.abs(got[n, :n + 1] - ex[n, :n + 1])) / np.max(np.abs(ex[n, :n + 1]))
                  for n in range(2 * P + 1))
        if stable:
            assert err < 1e-12, (rho, z, err)
        else:
            assert err > 1e-9, (rho, z, err)  # >= 7 digits lost


def test_reaction_me_convergence_e1():
    # Section 3.3 example: the ME of u^{11}_{11} and u^{22}_{11} converges
    # like (|r'_ab - r_c| / |r - r_c|)^(p+1)
    g = json.load(open(os.path.join(HERE, "golden", "me_convergence_e1.json")))
    d, eps = g["d"], g["eps"]
    assert np.linalg.norm(np.subtract(g["polarization_source_11"], g["center_11"])) == pytest.approx(
        g["distance_source_center"], abs=1e-4)
    for comp, rp, rc in [((1, 1, 1, 1), g["polarization_source_11"], g["center_11"]),
                         ((1, 1, 2, 2), g["polarization_source_22"], g["center_22"])]:
        for r in g["targets"]:
            exact = expansions.reaction_exact(d, eps, *comp, r, rp)
            rate = np.linalg.norm(np.subtract(rp, rc)) / np.linalg.norm(np.subtract(r, rc))
            errs = []
            for p in (1, 3, 5, 7):
                e = abs(expansions.reaction_me(d, eps, *comp, r, rp, rc, p) - exact) / abs(exact)
                errs.append(e)
                assert e <= 1.5 * rate ** (p + 1) + 1e-14, (comp, r, p, e, rate)
            assert errs[-1] < errs[0] * rate ** 4


def test_polarization_coordinates():
    # eq. eqpolarizedsource: z'_ab for a middle-layer source, and the
    # separation by an interface of Section 3.2
    d = D3
    zp = -0.4
    l, lp = 1, 1
    z11 = d[l] - (zp - d[lp])
    z22 = d[l - 1] + (d[lp - 1] - zp)
    assert z11 == pytest.approx(-2.0)
    assert z22 == pytest.approx(0.4)
    # u^{11}_{11}(r, r') = sigma-weighted kernel at distance z - z'_11
    r = np.array([0.1, 0.0, -0.7]); rp = np.array([0.0, 0.0, zp])
    u, _ = oracle.reaction_pair(d, MEDIA[0], 1, 1, r, rp, mode=oracle.MODE_IMAGES)
    parts = 0.0
    for (a, b, zz) in [(1, 1, z11), (2, 2, z22), (1, 2, d[l] - (d[lp - 1] - zp)), (2, 1, d[l - 1] + (zp - d[lp]))]:
        parts += oracle.sommerfeld_K_images(d, MEDIA[0], 1, 1, a, b, 0, 0, 0.1, abs(r[2] - zz))
    assert u == pytest.approx(parts, rel=1e-13)


def test_mlp_reference_gradient_matches_finite_differences_and_autograd():
    # the surrogate network's reference backward pass (oracle/mlp.py)
    from oracle import mlp
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 0.3, mlp.NPARAM)
    x = rng.uniform(-1, 1, (17, 4))
    y = rng.normal(0, 1, (17, 3))
    loss, grad = mlp.loss_and_grad(theta, x, y, quantize=False)
    idx = rng.choice(mlp.NPARAM, 40, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mlp.loss_and_grad(tp, x, y, quantize=False)[0] - mlp.loss_and_grad(tm, x, y, quantize=False)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])
    torch = pytest.importorskip("torch")
    t = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    parts, o = {}, 0
    for name, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        parts[name] = t[o:o + n].reshape(shp)
        o += n
    X = torch.tensor(x)
    a = X
    for k in ("1", "2", "3"):
        a = torch.nn.functional.silu(a @ parts["W" + k].T + parts["b" + k])
    out = a @ parts["W4"].T + parts["b4"]
    L = ((out - torch.tensor(y)) ** 2).sum() / x.shape[0]
    L.backward()
    assert abs(float(L) - loss) < 1e-12
    assert np.max(np.abs(t.grad.numpy() - grad)) < 1e-12


def test_bf16_rounding_reference():
    from oracle import mlp
    v = np.array([1.0, 1.00390625, 1.001953125, 3.14159, -2.5e-3], dtype=np.float32)
    r = mlp.bf16_round(v)
    torch = pytest.importorskip("torch")
    ref = torch.tensor(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r, ref)


# ---------------------------------------------------------------------------
# General media (more than two interfaces): the oracle's per-k linear solve of
# Appendix A covers any number of layers.  These pins fix it for four layers.
# ---------------------------------------------------------------------------
D4 = [0.0, -0.6, -1.2]
ZR4 = {0: (0.1, 1.1), 1: (-0.55, -0.05), 2: (-1.15, -0.65), 3: (-2.3, -1.3)}


def _points4(rng, n):
    lay = rng.integers(0, 4, n).astype(np.int32)
    xyz = np.zeros((n, 3))
    xyz[:, :2] = rng.uniform(-0.5, 0.5, (n, 2))
    for i in range(n):
        xyz[i, 2] = rng.uniform(*ZR4[int(lay[i])])
    return xyz, lay


def test_thirty_six_components_for_four_layers():
    # a layer has a reaction term per bounding interface (eqs. generalcomponents,
    # zexponential): 2L of them over all layers, so (2L)^2 reaction components
    L = 3
    comps = [(l, lp, a, b) for l in range(L + 1) for lp in range(L + 1) for a in (1, 2) for b in (1, 2)
             if not (a == 1 and l == L) and not (a == 2 and l == 0)
             and not (b == 1 and lp == L) and not (b == 2 and lp == 0)]
    assert len(comps) == 36
    for k in (0.1, 1.0, 4.0):
        for lp in range(4):
            s = oracle.sigma(D4, [1.0, 5.0, 2.0, 10.0], k, lp)
            for l in range(4):
                for a in (1, 2):
                    for b in (1, 2):
                        if (l, lp, a, b) not in comps:
                            assert s[l, a - 1, b - 1] == 0.0


@pytest.mark.parametrize("merge", ["inner", "top"])
def test_equal_eps_interface_disappears(merge):
    # an interface between two layers of the same permittivity is no interface:
    # the four-layer potential equals the three-layer one, which the exact image
    # series evaluates independently of the linear solve
    rng = np.random.default_rng(41)
    xyz, lay = _points4(rng, 80)
    q = rng.uniform(-1, 1, 80)
    if merge == "inner":      # layers 1 and 2 share eps = 5: interfaces (0, -1.2) remain
        eps4, d3, lay3 = [1.0, 5.0, 5.0, 10.0], [0.0, -1.2], np.where(lay >= 2, lay - 1, lay)
    else:                      # layers 0 and 1 share eps = 1: interfaces (-0.6, -1.2) remain
        eps4, d3, lay3 = [1.0, 1.0, 5.0, 10.0], [-0.6, -1.2], np.maximum(lay - 1, 0)
    eps3 = [eps4[0], eps4[2], eps4[3]] if merge == "inner" else [eps4[1], eps4[2], eps4[3]]
    t = np.arange(30)
    p4, f4 = oracle.direct(D4, eps4, xyz, lay, q, targets=t, mode=oracle.MODE_QUAD)
    p3, f3 = oracle.direct(d3, eps3, xyz, lay3.astype(np.int32), q, targets=t, mode=oracle.MODE_IMAGES)
    assert oracle.err2(p3, p4) < 1e-11
    assert oracle.err2(f3, f4) < 1e-10


def test_uniform_four_layer_medium_is_coulomb():
    rng = np.random.default_rng(43)
    xyz, lay = _points4(rng, 40)
    q = rng.uniform(-1, 1, 40)
    p4, f4 = oracle.direct(D4, [3.0] * 4, xyz, lay, q, mode=oracle.MODE_QUAD)
    p0, f0 = oracle.direct([], [3.0], xyz, np.zeros(40, np.int32), q)
    assert np.max(np.abs(p4 - p0)) < 1e-13 * np.max(np.abs(p0))
    assert np.max(np.abs(f4 - f0)) < 1e-12 * np.max(np.abs(f0))


@pytest.mark.parametrize("src_layer", [1, 2])
def test_transmission_conditions_four_layers(src_layer):
    # eq. transmissioncond at every interface of a four-layer medium
    eps = [2.0, 7.0, 1.5, 12.0]
    rp = np.array([0.05, -0.1, -0.3 if src_layer == 1 else -0.9])
    for j, dj in enumerate(D4):
        above, below = j, j + 1
        x = np.array([0.2, 0.15, dj])

        def total(l, pt):
            u, g = oracle.reaction_pair(D4, eps, l, src_layer, pt, rp, mode=oracle.MODE_QUAD)
            if l == src_layer:
                R = pt - rp
                u += 1 / np.linalg.norm(R)
                g = g - R / np.linalg.norm(R) ** 3
            return u, g
        ua, ga = total(above, x)
        ub, gb = total(below, x)
        assert ua == pytest.approx(ub, rel=1e-10)
        assert eps[above] * ga[2] == pytest.approx(eps[below] * gb[2], rel=1e-9)
        assert ga[0] == pytest.approx(gb[0], rel=1e-9)


@pytest.mark.parametrize("h", [1e-3, 1e-4])
def test_transmission_conditions_four_layers_next_to_interfaces(h):
    # eq. transmissioncond at each interface, with the source a distance h
    # below it and the evaluation point right above the source (rho = 0.01):
    # the exponent distances are ~h, the regime of the near field
    eps = [2.0, 7.0, 1.5, 12.0]
    for j, dj in enumerate(D4):
        above, below = j, j + 1
        rp = np.array([0.05, -0.1, dj - h])
        x = np.array([0.06, -0.1, dj])

        def total(l, pt):
            u, g = oracle.reaction_pair(D4, eps, l, below, pt, rp, mode=oracle.MODE_QUAD)
            if l == below:
                R = pt - rp
                u += 1 / np.linalg.norm(R)
                g = g - R / np.linalg.norm(R) ** 3
            return u, g
        ua, ga = total(above, x)
        ub, gb = total(below, x)
        assert ua == pytest.approx(ub, rel=1e-10)
        assert eps[above] * ga[2] == pytest.approx(eps[below] * gb[2], rel=1e-9)
        assert ga[0] == pytest.approx(gb[0], rel=1e-9)


def test_equal_eps_interface_disappears_next_to_interfaces():
    # eps = (1, 5, 5, 10): the interface at -0.6 disappears, and charges 1e-4
    # from the remaining interfaces (0 and -1.2) must see the three-layer
    # image series' potential and field
    rng = np.random.default_rng(53)
    n = 60
    lay = rng.integers(0, 4, n).astype(np.int32)
    side = {0: (0.0, 1.0), 1: (0.0, -1.0), 2: (-1.2, 1.0), 3: (-1.2, -1.0)}
    xyz = np.zeros((n, 3))
    xyz[:, :2] = rng.uniform(-0.5, 0.5, (n, 2))
    for i in range(n):
        base, sgn = side[int(lay[i])]
        xyz[i, 2] = base + sgn * 10 ** rng.uniform(-4, -2)
    q = rng.uniform(-1, 1, n)
    lay3 = np.where(lay >= 2, lay - 1, lay).astype(np.int32)
    t = np.arange(20)
    p4, f4 = oracle.direct(D4, [1.0, 5.0, 5.0, 10.0], xyz, lay, q, targets=t, mode=oracle.MODE_QUAD)
    p3, f3 = oracle.direct(D3, [1.0, 5.0, 10.0], xyz, lay3, q, targets=t, mode=oracle.MODE_IMAGES)
    assert oracle.err2(p3, p4) < 1e-11
    assert oracle.err2(f3, f4) < 1e-10


def test_reciprocity_four_layers():
    eps = [2.0, 7.0, 1.5, 12.0]
    rng = np.random.default_rng(47)
    for l in range(4):
        for lp in range(4):
            r = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(*ZR4[l])])
            rp = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(*ZR4[lp])])
            u1, _ = oracle.reaction_pair(D4, eps, l, lp, r, rp)
            u2, _ = oracle.reaction_pair(D4, eps, lp, l, rp, r)
            free = 1.0 / np.linalg.norm(r - rp) if l == lp else 0.0
            assert eps[l] * (u1 + free) == pytest.approx(eps[lp] * (u2 + free), rel=1e-11)


D5 = [0.0, -0.6, -1.2, -1.8]


@pytest.mark.parametrize("src_layer", [1, 3])
def test_transmission_conditions_five_layers(src_layer):
    # eq. transmissioncond at every interface of a five-layer medium
    eps = [2.0, 7.0, 1.5, 12.0, 4.0]
    rp = np.array([0.05, -0.1, -0.3 if src_layer == 1 else -1.5])
    for j, dj in enumerate(D5):
        above, below = j, j + 1
        x = np.array([0.2, 0.15, dj])

        def total(l, pt):
            u, g = oracle.reaction_pair(D5, eps, l, src_layer, pt, rp, mode=oracle.MODE_QUAD)
            if l == src_layer:
                R = pt - rp
                u += 1 / np.linalg.norm(R)
                g = g - R / np.linalg.norm(R) ** 3
            return u, g
        ua, ga = total(above, x)
        ub, gb = total(below, x)
        assert ua == pytest.approx(ub, rel=1e-10)
        assert eps[above] * ga[2] == pytest.approx(eps[below] * gb[2], rel=1e-9)
        assert ga[0] == pytest.approx(gb[0], rel=1e-9)


def test_five_layers_with_two_vanishing_interfaces_match_three_layer_images():
    # eps = (1, 5, 5, 10, 10): the interfaces at -0.6 and -1.8 separate equal
    # permittivities and disappear, leaving the three-layer medium (1, 5, 10)
    # with interfaces 0 and -1.2, whose exact image series is independent
    rng = np.random.default_rng(59)
    n = 50
    lay = rng.integers(0, 5, n).astype(np.int32)
    zr = {0: (0.05, 1.0), 1: (-0.55, -0.05), 2: (-1.15, -0.65), 3: (-1.75, -1.25), 4: (-2.8, -1.85)}
    xyz = np.zeros((n, 3))
    xyz[:, :2] = rng.uniform(-0.5, 0.5, (n, 2))
    for i in range(n):
        xyz[i, 2] = rng.uniform(*zr[int(lay[i])])
    q = rng.uniform(-1, 1, n)
    lay3 = np.array([0, 1, 1, 2, 2], np.int32)[lay]
    t = np.arange(20)
    p5, f5 = oracle.direct(D5, [1.0, 5.0, 5.0, 10.0, 10.0], xyz, lay, q, targets=t, mode=oracle.MODE_QUAD)
    p3, f3 = oracle.direct(D3, [1.0, 5.0, 10.0], xyz, lay3, q, targets=t, mode=oracle.MODE_IMAGES)
    assert oracle.err2(p3, p5) < 1e-11
    assert oracle.err2(f3, f5) < 1e-10


def test_reciprocity_five_layers():
    eps = [2.0, 7.0, 1.5, 12.0, 4.0]
    zr = {0: (0.1, 1.0), 1: (-0.55, -0.05), 2: (-1.15, -0.65), 3: (-1.75, -1.25), 4: (-2.8, -1.9)}
    rng = np.random.default_rng(67)
    for l in range(5):
        for lp in range(5):
            r = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[l])])
            rp = np.array([*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[lp])])
            u1, _ = oracle.reaction_pair(D5, eps, l, lp, r, rp)
            u2, _ = oracle.reaction_pair(D5, eps, lp, l, rp, r)
            free = 1.0 / np.linalg.norm(r - rp) if l == lp else 0.0
            assert eps[l] * (u1 + free) == pytest.approx(eps[lp] * (u2 + free), rel=1e-11)
