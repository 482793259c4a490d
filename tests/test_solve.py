"""The integral-equation layer (GMRES and the panel system) on the CPU, with
the oracle's direct sum standing in for the FMM as the matrix-vector product:
the solver against dense solves, the panel system against the dense matrix of
the oracle, and the capacitance matrix against what the physics fixes
(symmetry of the eps-weighted Green's function, signs, scaling with eps)."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300.solve import PanelSystem, capacitance, gmres, plate_panels

D3 = [0.0, -1.2]


class OracleSum:
    """Direct summation by the oracle behind the FMM's build / evaluate calls."""

    def __init__(self, d, eps, mode=oracle.MODE_IMAGES):
        self.d, self.eps, self.mode = list(d), list(eps), mode

    def build(self, xyz, layer):
        self.xyz, self.layer = np.asarray(xyz), np.asarray(layer, dtype=np.int32)

    def evaluate(self, q, field=True):
        q = np.asarray(q)
        if q.ndim == 2:  # several charge vectors, like the FMM's [nrhs, n]
            res = [self.evaluate(row, field) for row in q]
            return np.stack([r[0] for r in res]), (np.stack([r[1] for r in res]) if field else None)
        phi, E = oracle.direct(self.d, self.eps, self.xyz, self.layer, q, mode=self.mode)
        return phi, (E if field else None)


def _two_plates(z0, z1, l0, l1, nside=6):
    a = plate_panels((0.0, 0.0, z0), 0.6, nside, l0)
    b = plate_panels((0.1, -0.05, z1), 0.5, nside, l1)
    xyz = np.concatenate([a[0], b[0]])
    rad = np.concatenate([a[1], b[1]])
    lay = np.concatenate([a[2], b[2]])
    cond = np.repeat([0, 1], nside * nside)
    return xyz, rad, lay, cond


@pytest.mark.parametrize("restart", [5, 40])
def test_gmres_matches_dense_solve(restart):
    rng = np.random.default_rng(3)
    n = 150
    A = 3.0 * np.eye(n) + rng.normal(0.0, 1.0, (n, n)) / np.sqrt(n)
    b = rng.normal(size=n)
    x, info = gmres(lambda v: A @ v, b, tol=1e-12, restart=restart)
    ref = np.linalg.solve(A, b)
    assert info["converged"] and np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b) * 1.0001


def test_gmres_stops_and_edge_cases():
    rng = np.random.default_rng(4)
    n = 60
    A = np.eye(n) + 0.9 * rng.normal(0.0, 1.0, (n, n)) / np.sqrt(n)
    b = rng.normal(size=n)
    _, info = gmres(lambda v: A @ v, b, tol=1e-14, restart=3, maxiter=7)
    assert not info["converged"] and info["iterations"] == 7
    x, info = gmres(lambda v: v, b)                 # identity: one product solves it
    assert info["converged"] and info["iterations"] == 1 and np.allclose(x, b)
    x, info = gmres(lambda v: A @ v, np.zeros(n))   # zero right-hand side
    assert info["converged"] and not x.any()
    ref = np.linalg.solve(A, b)
    x, info = gmres(lambda v: A @ v, b, x0=ref, tol=1e-10)  # already solved
    assert info["iterations"] == 0
    D = np.diag(np.linspace(1.0, 100.0, n))         # right preconditioning keeps the true residual
    x, info = gmres(lambda v: D @ v, b, precond=lambda r: r / np.diag(D), tol=1e-12)
    assert info["iterations"] == 1 and np.allclose(x, b / np.diag(D))


def test_panel_system_matches_dense_oracle_matrix():
    eps = [1.0, 5.0, 10.0]
    xyz, rad, lay, cond = _two_plates(-0.3, -0.8, 1, 1, nside=5)
    sysm = PanelSystem(OracleSum(D3, eps), eps, xyz, lay, rad)
    n = sysm.n
    U = np.column_stack([oracle.direct(D3, eps, xyz, lay, np.eye(n)[j], mode=oracle.MODE_IMAGES)[0]
                         for j in range(n)])
    A = U + np.diag(1.0 / (2.0 * np.pi * rad))
    v = (cond == 0).astype(float)
    q, info = sysm.solve(v, tol=1e-12)
    ref = np.asarray(eps)[lay] * np.linalg.solve(A, v)
    assert info["converged"]
    assert np.max(np.abs(q - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("z0,z1,l0,l1", [(-0.3, -0.8, 1, 1), (0.4, -0.5, 0, 1), (-0.9, -1.7, 1, 2)])
def test_capacitance_symmetric_and_signed(z0, z1, l0, l1):
    # the physical Green's function u / eps_source is symmetric, so is C; a
    # conductor at unit potential carries positive charge and induces negative
    # charge on the grounded one
    eps = [1.0, 5.0, 10.0]
    xyz, rad, lay, cond = _two_plates(z0, z1, l0, l1)
    C, infos = capacitance(PanelSystem(OracleSum(D3, eps), eps, xyz, lay, rad), cond, tol=1e-11)
    assert all(i["converged"] for i in infos)
    assert abs(C[0, 1] - C[1, 0]) < 1e-8 * abs(C[0, 0])
    assert C[0, 0] > 0 and C[1, 1] > 0 and C[0, 1] < 0
    assert C[0, 0] + C[0, 1] > 0 and C[1, 1] + C[1, 0] > 0


def test_capacitance_scales_with_permittivity():
    # in a uniform medium the reaction part vanishes and every charge scales with eps
    xyz, rad, lay, cond = _two_plates(-0.3, -0.8, 1, 1)
    C1, _ = capacitance(PanelSystem(OracleSum(D3, [1.0] * 3), [1.0] * 3, xyz, lay, rad), cond, tol=1e-12)
    C3, _ = capacitance(PanelSystem(OracleSum(D3, [3.0] * 3), [3.0] * 3, xyz, lay, rad), cond, tol=1e-12)
    assert np.allclose(C3, 3.0 * C1, rtol=1e-9, atol=0)


def test_separate_targets_match_pair_sums():
    # potential and field at charge-free points, against the oracle's reaction
    # kernel summed pair by pair (plus the Coulomb term for sources in the
    # target's layer): independent of the zero-charge construction
    from paper_1908_10863_gb300.solve import TargetSet
    eps = [1.0, 5.0, 10.0]
    rng = np.random.default_rng(21)
    zr = {0: (0.1, 1.1), 1: (-1.1, -0.1), 2: (-2.3, -1.3)}
    n, nt = 40, 7
    lay = rng.integers(0, 3, n).astype(np.int32)
    xyz = np.array([[*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[int(l)])] for l in lay])
    tl = rng.integers(0, 3, nt).astype(np.int32)
    txyz = np.array([[*rng.uniform(-0.5, 0.5, 2), rng.uniform(*zr[int(l)])] for l in tl])
    q = rng.uniform(-1.0, 1.0, n)
    ts = TargetSet(OracleSum(D3, eps), xyz, lay, txyz, tl)
    phi, E = ts.evaluate(q)
    ref_phi, ref_E = np.zeros(nt), np.zeros((nt, 3))
    for i in range(nt):
        for j in range(n):
            u, g = oracle.reaction_pair(D3, eps, int(tl[i]), int(lay[j]), txyz[i], xyz[j], mode=oracle.MODE_IMAGES)
            if tl[i] == lay[j]:
                R = txyz[i] - xyz[j]
                u += 1.0 / np.linalg.norm(R)
                g = g - R / np.linalg.norm(R) ** 3
            ref_phi[i] += q[j] * u / (4 * np.pi)
            ref_E[i] -= q[j] * g / (4 * np.pi)
    assert np.max(np.abs(phi - ref_phi)) < 1e-12 * np.max(np.abs(ref_phi))
    assert np.max(np.abs(E - ref_E)) < 1e-11 * np.max(np.abs(ref_E))
    phi2, _ = ts.evaluate(np.stack([q, 2.0 * q]))  # several charge vectors at once
    assert phi2.shape == (2, nt) and np.allclose(phi2[1], 2.0 * phi, rtol=1e-13, atol=0)
