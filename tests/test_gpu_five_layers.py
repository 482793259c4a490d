"""GPU parity for media of five layers (four interfaces, the general L-layer
interface problem of Appendix A solved at each quadrature node; the box key
gives the layer three bits, so trees stop at level 9).  Every reference is the
CPU oracle: its adaptive quadrature of its own per-k linear solve, or, where
interfaces separate equal permittivities, the exact image series of the
three-layer medium the five layers reduce to."""
import os

import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, workloads

pytestmark = pytest.mark.gpu
D5 = list(workloads.D_FIVE)
EPS5 = list(workloads.EPS_FIVE)


def _components(L):
    return [(l, lp, a, b) for l in range(L + 1) for lp in range(L + 1) for a in (1, 2) for b in (1, 2)
            if not (a == 1 and l == L) and not (a == 2 and l == 0)
            and not (b == 1 and lp == L) and not (b == 2 and lp == 0)]


COMPS5 = _components(4)


def test_medium_and_components():
    assert len(COMPS5) == 64
    w = workloads.five_layers(500)
    with LayeredFMM(w.d, w.eps, 4) as f:
        f.build(w.xyz, w.layer)
        st = f.stats()
        assert st["components"] == 5 + 64 and st["depth"] <= 9


def test_reaction_near_kernel_matches_oracle():
    rng = np.random.default_rng(15)
    rho = rng.uniform(0.0, 0.6, 8)
    h = rng.uniform(0.1, 2.0, 8)
    with LayeredFMM(D5, EPS5, 4) as f:
        for comp in COMPS5[::3]:
            got = f.reaction_kernel(*comp, rho, h)
            ref = np.array([[oracle.sommerfeld_K(D5, EPS5, *comp, N, mu, r, z) for N, mu in ((0, 0), (1, 0), (1, 1))]
                            for r, z in zip(rho, h)])
            err = np.max(np.abs(got - ref) / (np.abs(ref[:, :1]) + 1e-300))
            assert err < 1e-11, (comp, err)


def _oracle(w, t, mode=oracle.MODE_QUAD):
    return oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=mode, threads=os.cpu_count() or 1)


@pytest.mark.parametrize("aligned", [True, False])
# measured Err2 (phi, field): aligned 5.8e-7 3.4e-6 (FP64), 7.4e-7 3.4e-6 (float32);
# unaligned 5.8e-7 1.9e-6, 6.2e-7 2.2e-6
@pytest.mark.parametrize("precision,tol_phi,tol_fld", [(0, 2e-6, 8e-6), (1, 2e-6, 8e-6)])
def test_fmm_matches_oracle(aligned, precision, tol_phi, tol_fld):
    d = workloads.D_FIVE if aligned else workloads.D_FIVE_UNALIGNED
    w = workloads.five_layers(3000, d=d)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build(w.xyz, w.layer)
        st = f.stats()
        phi, E = f.evaluate(w.q)
    assert st["m2l_reaction"] > 0 and st["p2p_reaction"] > 0 and st["timeouts"] == 0
    t = workloads.subsample(w.n, 48)
    ref, refE = _oracle(w, t)
    e_phi, e_fld = oracle.err2(ref, phi[t]), oracle.err2(refE, E[t])
    print("five layers aligned=%s precision=%d: Err2 phi %.2e field %.2e (depth %d, m2l_reaction %d, "
          "p2p_reaction %d)" % (aligned, precision, e_phi, e_fld, st["depth"], st["m2l_reaction"],
                                st["p2p_reaction"]))
    assert e_phi < tol_phi and e_fld < tol_fld


@pytest.mark.parametrize("precision", [0, 1])
def test_near_interfaces_matches_oracle(precision):
    # every charge 1e-3 .. 0.02 from an interface: reaction pairs of every layer pair in the near field
    w = workloads.five_layers(3200, near=0.02)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build(w.xyz, w.layer)
        st = f.stats()
        phi, E = f.evaluate(w.q)
    assert st["p2p_reaction"] > 0
    t = workloads.subsample(w.n, 40)
    ref, refE = _oracle(w, t)
    e_phi, e_fld = oracle.err2(ref, phi[t]), oracle.err2(refE, E[t])
    print("five layers near interfaces precision=%d: Err2 phi %.2e field %.2e" % (precision, e_phi, e_fld))
    # measured 3.8e-6 / 9.5e-7 (FP64), 4.1e-6 / 9.6e-6 (float32)
    assert e_phi < 8e-6 and e_fld < 2e-5


def test_vanishing_interfaces_match_three_layer_images():
    # eps = (1, 5, 5, 10, 10): the interfaces at -0.6 and -1.8 disappear; the
    # FMM must reproduce the exact image series of the three-layer medium
    w = workloads.five_layers(8000, eps=(1.0, 5.0, 5.0, 10.0, 10.0))
    with LayeredFMM(w.d, w.eps, 10) as f:
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q)
    t = workloads.subsample(w.n, 200)
    lay3 = np.array([0, 1, 1, 2, 2], np.int32)[w.layer]
    ref, refE = oracle.direct([0.0, -1.2], [1.0, 5.0, 10.0], w.xyz, lay3, w.q, targets=t, mode=oracle.MODE_IMAGES)
    e_phi, e_fld = oracle.err2(ref, phi[t]), oracle.err2(refE, E[t])
    print("five layers, two vanishing interfaces: Err2 phi %.2e field %.2e" % (e_phi, e_fld))
    assert e_phi < 2e-6 and e_fld < 1e-5  # measured 6.1e-7 / 4.2e-6


def test_large_problem():
    # N = 262,144 in five layers, float32 form: against the three-layer image
    # series through two vanishing interfaces, on sampled targets
    w = workloads.five_layers(1 << 18, eps=(1.0, 5.0, 5.0, 10.0, 10.0))
    with LayeredFMM(w.d, w.eps, 10, precision=1) as f:
        f.build(w.xyz, w.layer)
        st = f.stats()
        phi, E = f.evaluate(w.q)
    assert st["timeouts"] == 0 and st["components"] == 69
    t = workloads.subsample(w.n, 40)
    lay3 = np.array([0, 1, 1, 2, 2], np.int32)[w.layer]
    ref, refE = oracle.direct([0.0, -1.2], [1.0, 5.0, 10.0], w.xyz, lay3, w.q, targets=t, mode=oracle.MODE_IMAGES,
                              threads=os.cpu_count() or 1)
    e_phi, e_fld = oracle.err2(ref, phi[t]), oracle.err2(refE, E[t])
    print("five layers N=262144 float32: Err2 phi %.2e field %.2e (depth %d)" % (e_phi, e_fld, st["depth"]))
    assert e_phi < 8e-6 and e_fld < 2e-5  # measured 3.5e-6 / 7.5e-6
