"""GPU tests of the pre-computed remainder tables of the near-field reaction
kernels: their interpolation error against the quadrature, the FMM with them
against the FMM with the quadrature and against the oracle, and what they
gain in the near field."""
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, LfmmError, workloads
from paper_1908_10863_gb300.lfmm import OPT_NEAR_TABLES, OPT_PROFILE

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps,tol", [(workloads.EPS_CONFIG, 1e-7), (workloads.EPS_HIGH_CONTRAST, 1e-6)])
def test_table_interpolation_error(eps, tol):
    with LayeredFMM(workloads.D_CONFIG, eps, 8) as f:
        e = f.near_tables()
        e2 = f.near_tables()  # built once; checked again
    print("eps %s: largest relative deviation from the quadrature %.2e" % (eps, e))
    assert e == e2 and e < tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_fmm_with_tables_matches_quadrature_and_oracle(precision, tol):
    w = workloads.near_interface(12000)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build(w.xyz, w.layer)
        assert f.stats()["p2p_reaction"] > 0
        f.set_option(OPT_NEAR_TABLES, 0)
        phi0, E0 = f.evaluate(w.q)
        f.set_option(OPT_NEAR_TABLES, 1)
        phi1, E1 = f.evaluate(w.q)
        f.set_option(OPT_NEAR_TABLES, 0)
        phi2, _ = f.evaluate(w.q)
        with pytest.raises(LfmmError):
            f.set_option(OPT_NEAR_TABLES, 3)
    d_phi, d_fld = oracle.err2(phi0, phi1), oracle.err2(E0, E1)
    print("precision %d: tables vs quadrature Err2 phi %.2e field %.2e" % (precision, d_phi, d_fld))
    assert d_phi < tol and d_fld < 10 * tol
    assert oracle.err2(phi0, phi2) < (1e-13 if precision == 0 else 1e-6)  # switched off again: the quadrature
    t = workloads.subsample(w.n, 200)
    ref, _ = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES)
    assert oracle.err2(ref, phi1[t]) < 1e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_tables_gain_in_near_field(precision):
    w = workloads.near_interface(1 << 17)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.set_option(OPT_PROFILE, 1)
        f.build(w.xyz, w.layer)
        res = {}
        for use in (0, 1):
            f.set_option(OPT_NEAR_TABLES, use)
            f.evaluate(w.q)
            ts = []
            for _ in range(3):
                phi, _ = f.evaluate(w.q)
                ts.append(f.timings()["p2p"])
            res[use] = (min(ts), phi)
    print("precision %d: near field %.3f ms by quadrature, %.3f ms with tables (%.2fx); Err2 %.2e"
          % (precision, res[0][0], res[1][0], res[0][0] / res[1][0], oracle.err2(res[0][1], res[1][1])))
    assert oracle.err2(res[0][1], res[1][1]) < (1e-8 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_default_near_tables_automatic(precision):
    # the default (2) takes the tables in the float32 form once the near lists
    # hold reaction pairs and keeps the quadrature in the FP64 form
    w = workloads.near_interface(12000)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build(w.xyz, w.layer)
        assert f.stats()["p2p_reaction"] > 0
        phi_d, _ = f.evaluate(w.q)
        f.set_option(OPT_NEAR_TABLES, 0)
        phi_q, _ = f.evaluate(w.q)
        f.set_option(OPT_NEAR_TABLES, 1)
        phi_t, _ = f.evaluate(w.q)
        f.set_option(OPT_NEAR_TABLES, 2)
        phi_a, _ = f.evaluate(w.q)
    if precision == 0:
        # tables and quadrature differ by ~2e-11 here: the default is the quadrature
        assert oracle.err2(phi_q, phi_d) < 1e-14 and oracle.err2(phi_q, phi_a) < 1e-14
        assert oracle.err2(phi_t, phi_d) > 1e-13
    else:
        assert oracle.err2(phi_t, phi_d) < 1e-6 and oracle.err2(phi_t, phi_a) < 1e-6
