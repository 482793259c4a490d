"""Integral equations with the layered-media FMM as the matrix-vector product.

The paper's introduction motivates the method by boundary-integral
formulations of capacitance extraction in layered (IC-like) media, solved by a
Krylov method whose matrix-vector product is the fast summation.  This module
is that outer layer: a restarted GMRES and a collocation system of flat panels
lumped to point charges, whose product is one call of
``LayeredFMM.evaluate`` (any object with the same ``build`` / ``evaluate``
methods works, which is how the tests drive it with the CPU oracle).

Units follow the library: the layered Green's function u solves
Delta u = -delta in every layer with eps only in the interface conditions
(Section 3.1), so the physical potential of a charge Q in layer l' is
Q u / eps_l'.  The unknowns of the panel system are therefore the scaled
charges Q / eps of the source layer; the physical Green's function
u(r, r') / eps_l' is symmetric (eps-weighted reciprocity of the interface
problem), so the capacitance matrix is too.
"""
from __future__ import annotations

import math

import numpy as np


def gmres(matvec, b, x0=None, tol: float = 1e-8, restart: int = 50, maxiter: int = 1000, precond=None):
    """Solve A x = b by restarted GMRES(restart) with modified Gram-Schmidt
    Arnoldi and Givens rotations; right preconditioning by ``precond``
    (a callable applying M^{-1}), so the residual is the true one.

    Returns (x, info) with info = {"iterations", "residual" (relative, of the
    last iterate), "converged", "cycles" (Arnoldi cycles run)}.  Stops when
    ||b - A x|| <= tol ||b|| or after ``maxiter`` products.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    M = (lambda v: v) if precond is None else precond
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), {"iterations": 0, "residual": 0.0, "converged": True, "cycles": 0}
    m = max(1, int(restart))
    its, cycles = 0, 0
    r = b - matvec(x)
    beta = float(np.linalg.norm(r))
    while True:
        if beta <= tol * bnorm or its >= maxiter:
            return x, {"iterations": its, "residual": beta / bnorm, "converged": beta <= tol * bnorm,
                       "cycles": cycles}
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        while k < m and its < maxiter:
            Z[k] = M(V[k])
            w = matvec(Z[k])
            its += 1
            for j in range(k + 1):
                H[j, k] = float(np.dot(w, V[j]))
                w = w - H[j, k] * V[j]
            hnext = float(np.linalg.norm(w))
            H[k + 1, k] = hnext
            if hnext > 0.0:
                V[k + 1] = w / hnext
            # apply the earlier rotations to the new column, then make its own
            for j in range(k):
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = (1.0, 0.0) if den == 0.0 else (H[k, k] / den, H[k + 1, k] / den)
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k += 1
            # converged, or the Krylov space is invariant (the solution lies in it)
            if abs(g[k]) <= tol * bnorm or hnext == 0.0:
                break
        # x += Z^T y with H[:k, :k] y = g[:k] (upper triangular)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - float(np.dot(H[i, i + 1:k], y[i + 1:k]))) / H[i, i] if H[i, i] != 0.0 else 0.0
        x = x + Z[:k].T @ y
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
        cycles += 1


class PanelSystem:
    """Collocation of a single-layer charge density on N flat panels, each
    lumped to a point charge at its centroid r_i (in layer l_i, radius a_i of
    the disk of equal area):

        (S + U) s = v,   S_ii = 1 / (2 pi a_i),   U_ij = u(r_i, r_j),

    where s_j = Q_j / eps_{l_j} are the scaled charges, v the prescribed
    physical potentials, 1/(2 pi a) the potential at the centre of a uniformly
    charged disk of unit charge, and U the layered Green's function between
    centroids without the free-space self term and with the reaction self term
    (exactly what the FMM evaluates at its charges).  ``solve`` returns the
    physical charges Q = eps s.
    """

    def __init__(self, fmm, eps, xyz, layer, radius):
        self.fmm = fmm
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.layer = np.ascontiguousarray(layer, dtype=np.int32)
        self.radius = np.asarray(radius, dtype=np.float64) * np.ones(self.xyz.shape[0])
        if np.any(self.radius <= 0.0):
            raise ValueError("panel radii must be positive")
        self.eps_panel = np.asarray(eps, dtype=np.float64)[self.layer]
        self.self_coef = 1.0 / (2.0 * math.pi * self.radius)
        self.products = 0
        fmm.build(self.xyz, self.layer)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def matvec(self, s):
        self.products += 1
        phi, _ = self.fmm.evaluate(np.ascontiguousarray(s, dtype=np.float64), field=False)
        return phi + self.self_coef * s

    def solve(self, v, tol: float = 1e-8, restart: int = 50, maxiter: int = 1000):
        """Physical panel charges for prescribed potentials v (Jacobi-preconditioned GMRES)."""
        inv = 1.0 / self.self_coef
        s, info = gmres(self.matvec, v, tol=tol, restart=restart, maxiter=maxiter, precond=lambda r: inv * r)
        return self.eps_panel * s, info


def capacitance(system: PanelSystem, conductor, tol: float = 1e-8, **kw):
    """Capacitance matrix of the conductors labelled 0..K-1 by ``conductor``
    (one label per panel): column j holds the total charge on each conductor
    when conductor j is at unit potential and the others at zero."""
    conductor = np.asarray(conductor)
    K = int(conductor.max()) + 1
    C = np.zeros((K, K))
    infos = []
    for j in range(K):
        q, info = system.solve((conductor == j).astype(np.float64), tol=tol, **kw)
        infos.append(info)
        C[:, j] = np.bincount(conductor, weights=q, minlength=K)
    return C, infos


def plate_panels(center, size, nside: int, layer: int):
    """Centroids of an nside x nside grid of square panels covering a
    horizontal plate (size x size, centred at ``center``), the radius of the
    disk of equal area, and the layer id: a synthetic conductor."""
    h = size / nside
    u = (np.arange(nside) + 0.5) * h - size / 2
    X, Y = np.meshgrid(u, u, indexing="ij")
    xyz = np.column_stack([X.ravel() + center[0], Y.ravel() + center[1], np.full(nside * nside, center[2])])
    return xyz, np.full(nside * nside, h / math.sqrt(math.pi)), np.full(nside * nside, layer, dtype=np.int32)


class TargetSet:
    """Potential and field at points that carry no charge (targets separate
    from the sources, as an integral-equation or post-processing step needs).
    The targets join the tree as zero charges: the FMM's sum at a charge is
    the layered-Green's-function sum over every other charge, and a zero
    charge adds nothing to anyone else's.  A target placed exactly on a
    source skips that source's singular free-space term, as the charges'
    own self terms are skipped.

    ``evaluate(q)`` takes the source charges ([n] or [nrhs, n]) and returns
    (phi, E) at the targets ([nt] / [nrhs, nt] and [..., nt, 3]).
    """

    def __init__(self, fmm, xyz, layer, target_xyz, target_layer):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        txyz = np.ascontiguousarray(target_xyz, dtype=np.float64).reshape(-1, 3)
        self.n, self.nt = int(xyz.shape[0]), int(txyz.shape[0])
        self.fmm = fmm
        fmm.build(np.concatenate([xyz, txyz]),
                  np.concatenate([np.asarray(layer, dtype=np.int32), np.asarray(target_layer, dtype=np.int32)]))

    def evaluate(self, q, field: bool = True):
        q = np.asarray(q, dtype=np.float64)
        if q.shape[-1] != self.n:
            raise ValueError("expected %d source charges, got %d" % (self.n, q.shape[-1]))
        pad = np.zeros(q.shape[:-1] + (self.nt,))
        phi, E = self.fmm.evaluate(np.ascontiguousarray(np.concatenate([q, pad], axis=-1)), field=field)
        return phi[..., self.n:], (E[..., self.n:, :] if field else None)
