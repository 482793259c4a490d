"""The float32 near field with the whole near list staged per warp against
the kernel that stages per source box (same pairs, float32 rounding apart)
and against the oracle, including leaves whose near lists exceed the staging
capacity (rounds of whole boxes, and a box larger than the capacity staged
in pieces)."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, workloads
from paper_1908_10863_gb300.lfmm import OPT_P2P_SPLIT, OPT_P2P_STAGED

pytestmark = pytest.mark.gpu

# two evaluations of the float32 form differ by the order of the far field's
# float atomics alone at Err2 ~2-3e-7 (measured up to 3.05e-7); the near-field
# kernels are compared within that noise
NOISE = 5e-7


def _both(w, p=8, split=0, leaf_cap=40):
    out = []
    with LayeredFMM(w.d, w.eps, p, precision=1, leaf_cap=leaf_cap) as f:
        if split:
            f.set_option(OPT_P2P_SPLIT, split)
        f.build(w.xyz, w.layer)
        st = f.stats()
        for staged in (0, 1):
            f.set_option(OPT_P2P_STAGED, staged)
            out.append(f.evaluate(w.q))
    return out, st


def _clustered(n=1 << 18, extra=3000, seed=5):
    # config2 plus a dense cluster in the middle layer: one leaf holds
    # thousands of charges, so its near lists overflow the staging capacity
    # (N = 262,144: deep enough that no reaction pair is near)
    w = workloads.config2(n, seed=seed)
    rng = np.random.default_rng(seed)
    c = np.column_stack([rng.uniform(0.1, 0.1005, extra), rng.uniform(-0.2, -0.1995, extra),
                         rng.uniform(-0.6, -0.5995, extra)])
    w.xyz = np.concatenate([w.xyz, c])
    w.layer = np.concatenate([w.layer, np.ones(extra, np.int32)])
    w.q = np.concatenate([w.q, rng.uniform(-1, 1, extra)])
    return w


# the staged kernel serves trees whose near lists hold no reaction pair
# (N >~ 100k for this workload); smaller trees keep the per-box kernel
@pytest.mark.parametrize("case", ["config2_131072", "config2_262144", "config2_262144_split4"])
def test_staged_matches_per_box_staging(case):
    parts = case.split("_")
    w = workloads.config2(int(parts[1]))
    split = int(parts[2][5:]) if len(parts) > 2 else 0
    ((p0, E0), (p1, E1)), st = _both(w, split=split)
    assert st["p2p_reaction"] == 0
    e, eE = oracle.err2(p0, p1), oracle.err2(E0, E1)
    print("%s: staged vs per-box Err2 phi %.2e field %.2e (leaves %d, mean %.1f per leaf)"
          % (case, e, eE, st["leaves"], w.n / st["leaves"]))
    assert e < NOISE and eE < NOISE


@pytest.mark.parametrize("cap", [6, 16, 64, 160])
def test_staged_leaf_sizes(cap):
    # the lanes of a warp are laid out per leaf as target slots x source
    # slices with up to three targets per lane; leaf capacities from 6 to 160
    # give leaves of a few charges (many slices) up to more than 96 (several
    # passes over the targets)
    w = workloads.config2(1 << 18)
    ((p0, E0), (p1, E1)), st = _both(w, leaf_cap=cap)
    assert st["p2p_reaction"] == 0
    e, eE = oracle.err2(p0, p1), oracle.err2(E0, E1)
    print("leaf cap %d (mean %.1f per leaf): staged vs per-box Err2 phi %.2e field %.2e"
          % (cap, w.n / st["leaves"], e, eE))
    assert e < NOISE and eE < NOISE


def test_staged_not_used_with_near_reaction_pairs():
    # N = 20,000: the near lists hold reaction pairs, so both settings run the
    # per-box kernel; the float atomics of the far field make two evaluations
    # differ only at the float32 noise level
    w = workloads.config2(20000)
    ((p0, E0), (p1, E1)), st = _both(w)
    assert st["p2p_reaction"] > 0
    assert oracle.err2(p0, p1) < NOISE and oracle.err2(E0, E1) < NOISE


def test_staged_clustered_against_oracle():
    # A leaf of 3,000 charges within 5e-4 of each other: its near lists
    # overflow the staging capacity (rounds of whole boxes, and the leaf's own
    # box staged in pieces).  Pair distances of ~1e-4 against float32 offsets
    # of ~1e-2 from the leaf centre limit the float32 form there (both kernels
    # measured Err2(phi) 9.1e-5, field 8.0e-4 on these targets): each kernel is
    # compared with the oracle, and the staged one must be as accurate as
    # the per-box one.
    import os
    w = _clustered()
    n0 = w.n - 3000
    ((p0, E0), (p1, E1)), st = _both(w, p=10)
    assert st["p2p_reaction"] == 0
    # targets in the cluster and elsewhere
    t = np.concatenate([workloads.subsample(n0, 150), n0 + np.arange(0, 3000, 20)])
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES,
                              threads=os.cpu_count() or 1)
    e0, e1 = oracle.err2(ref, p0[t]), oracle.err2(ref, p1[t])
    f0, f1 = oracle.err2(refE, E0[t]), oracle.err2(refE, E1[t])
    print("clustered: Err2 phi per-box %.2e staged %.2e; field per-box %.2e staged %.2e" % (e0, e1, f0, f1))
    assert e1 < 2e-4 and f1 < 2e-3
    assert e1 <= 1.05 * e0 + 1e-8 and f1 <= 1.05 * f0 + 1e-8
