"""GPU tests of the launch settings: the near-list split of the P2P kernels
and the autotuner that picks leaf capacity, M2L engine and split.  Settings
change how work is distributed, never the result beyond summation order."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, LfmmError, workloads
from paper_1908_10863_gb300.lfmm import EINVAL, OPT_P2P_SPLIT, OPT_SURROGATE

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_near_list_split_keeps_results(precision, tol):
    w = workloads.near_interface(6000)  # reaction pairs in the near field too
    with LayeredFMM(w.d, w.eps, 8, precision=precision) as f:
        f.set_option(OPT_P2P_SPLIT, 1)
        f.build(w.xyz, w.layer)
        ref = f.evaluate(w.q)
        for k in (0, 2, 4, 16):
            f.set_option(OPT_P2P_SPLIT, k)
            phi, E = f.evaluate(w.q)
            e = (oracle.err2(ref[0], phi), oracle.err2(ref[1], E))
            print("precision %d split %d: Err2 vs split 1 phi %.2e field %.2e" % (precision, k, *e))
            assert e[0] < tol and e[1] < tol
        # several right-hand sides share the zeroed outputs
        Q = np.random.default_rng(3).uniform(-1, 1, (3, w.n))
        f.set_option(OPT_P2P_SPLIT, 8)
        phi_b, _ = f.evaluate(Q)
        f.set_option(OPT_P2P_SPLIT, 1)
        phi_1, _ = f.evaluate(Q)
        assert oracle.err2(phi_1, phi_b) < tol


def test_near_list_split_with_network():
    w = workloads.near_interface(6000)
    with LayeredFMM(w.d, w.eps, 8) as f:
        f.surrogate_train(1 << 15, 4, 3)
        f.set_option(OPT_SURROGATE, 1)
        f.set_option(OPT_P2P_SPLIT, 1)
        f.build(w.xyz, w.layer)
        ref, _ = f.evaluate(w.q)
        f.set_option(OPT_P2P_SPLIT, 16)
        phi, _ = f.evaluate(w.q)
        assert f.stats()["surr_net_pairs"] > 0
    assert oracle.err2(ref, phi) < 1e-12


def test_split_option_is_checked():
    w = workloads.config2(2000)
    with LayeredFMM(w.d, w.eps, 6) as f:
        for bad in (3, -1, 32, 0.5):
            with pytest.raises(LfmmError) as ei:
                f.set_option(OPT_P2P_SPLIT, bad)
            assert ei.value.status == EINVAL


@pytest.mark.parametrize("precision,mode", [(1, 0), (0, 1)])
def test_autotune_picks_a_timed_setting_and_stays_correct(precision, mode):
    w = workloads.config2(12000)
    t = workloads.subsample(w.n, 100)
    ref, _ = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES)
    with LayeredFMM(w.d, w.eps, 8, precision=precision) as f:
        rows = f.autotune(w.xyz, w.layer, mode=mode, reps=2)
        for r in rows:
            print(r)
        chosen = [r for r in rows if r["chosen"] == 1.0]
        assert len(chosen) == 1
        assert chosen[0]["ms"] == min(r["ms"] for r in rows)
        assert len({r["depth"] for r in rows}) >= 2  # several tree depths were timed
        assert f.stats()["depth"] == int(chosen[0]["depth"])
        phi, _ = f.evaluate(w.q)
    e = oracle.err2(ref, phi[t])
    print("tuned: Err2 vs oracle %.2e" % e)
    assert e < 1e-4  # p = 8
