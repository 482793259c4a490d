"""The integral-equation layer with the GPU FMM as the product: potentials at
charge-free target points, and a capacitance matrix solved by GMRES, both
against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, workloads
from paper_1908_10863_gb300.solve import PanelSystem, TargetSet, capacitance, plate_panels

pytestmark = pytest.mark.gpu


class _OracleSum:
    def __init__(self, d, eps):
        self.d, self.eps = list(d), list(eps)

    def build(self, xyz, layer):
        self.xyz, self.layer = np.asarray(xyz), np.asarray(layer, dtype=np.int32)

    def evaluate(self, q, field=True):
        phi, E = oracle.direct(self.d, self.eps, self.xyz, self.layer, q, mode=oracle.MODE_IMAGES)
        return phi, (E if field else None)


def test_targets_without_charge():
    # measured: Err2(phi) 1.8e-6, Err2(E) 2.1e-5
    w = workloads.config2(20000, seed=11)
    rng = np.random.default_rng(5)
    nt = 50
    zr = {0: (0.1, 1.1), 1: (-1.1, -0.1), 2: (-2.3, -1.3)}
    tl = rng.integers(0, 3, nt).astype(np.int32)
    txyz = np.array([[*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[int(l)])] for l in tl])
    with LayeredFMM(w.d, w.eps, 10) as f:
        phi, E = TargetSet(f, w.xyz, w.layer, txyz, tl).evaluate(w.q)
    ref, refE = oracle.direct(w.d, w.eps, np.concatenate([w.xyz, txyz]), np.concatenate([w.layer, tl]),
                              np.concatenate([w.q, np.zeros(nt)]), targets=np.arange(w.n, w.n + nt),
                              mode=oracle.MODE_IMAGES)
    assert oracle.err2(ref, phi) < 1e-5 and oracle.err2(refE, E) < 2e-4


def test_capacitance_with_fmm_product():
    # two plates in the middle layer; measured: 20 GMRES products per column,
    # 3.9e-9 from the capacitance solved with the oracle's direct sum
    w = workloads.config2(8, seed=11)  # the medium only
    a = plate_panels((0.0, 0.0, -0.3), 0.6, 8, 1)
    b = plate_panels((0.1, -0.05, -0.8), 0.5, 8, 1)
    xyz = np.concatenate([a[0], b[0]])
    rad = np.concatenate([a[1], b[1]])
    lay = np.concatenate([a[2], b[2]])
    cond = np.repeat([0, 1], 64)
    with LayeredFMM(w.d, w.eps, 12) as f:
        C, infos = capacitance(PanelSystem(f, w.eps, xyz, lay, rad), cond, tol=1e-10)
    C2, _ = capacitance(PanelSystem(_OracleSum(w.d, w.eps), w.eps, xyz, lay, rad), cond, tol=1e-10)
    assert all(i["converged"] for i in infos)
    assert np.max(np.abs(C - C2)) < 1e-7 * np.max(np.abs(C2))
    assert abs(C[0, 1] - C[1, 0]) < 1e-7 * C[0, 0] and C[0, 1] < 0 < C[0, 0]
