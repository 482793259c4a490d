"""Seeded synthetic charge sets shaped like the paper's test problems.

These generators hold none of the method's arithmetic: they only draw points,
layer ids and charges.  Both the tests and the benchmark use them, for the GPU
library and for the CPU oracle alike.

* :func:`config1` -- three-layer medium (interfaces z=0, z=-1.2, eps=(1,5,10)),
  N charges uniform in [-0.5,0.5]^2 x [-1.1,-0.1] (middle layer).
* :func:`config2` -- same medium, N split equally between the three layers
  (remainder to the middle one): top z in [0.1,1.1], middle [-1.1,-0.1],
  bottom [-2.3,-1.3], x, y uniform in [-0.5,0.5].
* :func:`near_interface` -- same medium, every charge between ``hmin`` and
  ``delta`` from an interface on its own side (top [hmin, delta], middle
  [-delta, -hmin] and [-1.2 + hmin, -1.2 + delta], bottom
  [-1.2 - delta, -1.2 - hmin]); the near field then holds reaction
  interactions, which the other workloads' trees admit to the far field.
  ``hmin`` (default 1e-3) keeps each charge a finite distance from its own
  polarization image, as a charge of finite size would be.
* :func:`paper_p4` -- the irregular domains of Section 4: charges uniform in
  r(theta) = 0.5 - a + a P_4(cos theta), a = (0.1, 0.15, 0.05), centred at
  z = 0.6, -0.6, -1.8, eps = (21.2, 47.5, 62.8), by rejection from the
  bounding cube.
* :func:`four_layers` / :func:`four_layers_near_interface` -- media of four
  layers: slabs away from the interfaces, or every charge within ``delta``
  of an interface on its own side.
* :func:`five_layers` -- media of five layers, slabs or charges next to the
  interfaces.
* :func:`uneven_problems` -- k independent config2-shaped problems whose
  sizes are log-uniform in [nmin, nmax] (the batched form's many uneven
  problems), each with its own seed.
Charges are uniform in [-1, 1].  Every generator uses numpy's PCG64 with
seed 20190829 + config index unless a seed is given.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

D_CONFIG = (0.0, -1.2)
EPS_CONFIG = (1.0, 5.0, 10.0)
EPS_HIGH_CONTRAST = (1.0, 80.0, 2.0)
EPS_PAPER = (21.2, 47.5, 62.8)
SEED_BASE = 20190829


@dataclass
class Workload:
    name: str
    d: np.ndarray        # interface z positions, strictly decreasing
    eps: np.ndarray      # permittivity per layer, layer 0 on top
    xyz: np.ndarray      # [N, 3] float64
    layer: np.ndarray    # [N] int32
    q: np.ndarray        # [N] float64

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def _box(rng, n, zlo, zhi):
    xy = rng.uniform(-0.5, 0.5, size=(n, 2))
    z = rng.uniform(zlo, zhi, size=n)
    return np.column_stack([xy, z])


def config1(n: int = 1000, seed: int | None = None, eps=EPS_CONFIG) -> Workload:
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1 if seed is None else seed))
    xyz = _box(rng, n, -1.1, -0.1)
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("config1_n%d" % n, np.array(D_CONFIG), np.array(eps, dtype=np.float64), xyz,
                    np.ones(n, dtype=np.int32), q)


def config2(n: int = 1 << 20, seed: int | None = None, eps=EPS_CONFIG) -> Workload:
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2 if seed is None else seed))
    n0 = n // 3
    n2 = n // 3
    n1 = n - n0 - n2
    parts = [(_box(rng, n0, 0.1, 1.1), 0), (_box(rng, n1, -1.1, -0.1), 1), (_box(rng, n2, -2.3, -1.3), 2)]
    xyz = np.concatenate([p for p, _ in parts])
    layer = np.concatenate([np.full(p.shape[0], l, dtype=np.int32) for p, l in parts])
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("config2_n%d" % n, np.array(D_CONFIG), np.array(eps, dtype=np.float64), xyz, layer, q)


def near_interface(n: int = 1 << 18, delta: float = 0.02, hmin: float = 1e-3, seed: int | None = None,
                   eps=EPS_CONFIG) -> Workload:
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4 if seed is None else seed))
    d0, d1 = D_CONFIG
    sizes = [n // 4, n // 4, n // 4, n - 3 * (n // 4)]
    spans = [((d0 + hmin, d0 + delta), 0), ((d0 - delta, d0 - hmin), 1), ((d1 + hmin, d1 + delta), 1),
             ((d1 - delta, d1 - hmin), 2)]
    parts = [(_box(rng, cnt, lo, hi), l) for cnt, ((lo, hi), l) in zip(sizes, spans)]
    xyz = np.concatenate([p for p, _ in parts])
    layer = np.concatenate([np.full(p.shape[0], l, dtype=np.int32) for p, l in parts])
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("near_interface_n%d_d%g" % (n, delta), np.array(D_CONFIG), np.array(eps, dtype=np.float64),
                    xyz, layer, q)


def paper_p4(counts=(912, 640, 1296), seed: int | None = None) -> Workload:
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 6 if seed is None else seed))
    avals = (0.1, 0.15, 0.05)
    centres = (0.6, -0.6, -1.8)
    pts, lay = [], []
    for l, (cnt, a, zc) in enumerate(zip(counts, avals, centres)):
        got = []
        while sum(g.shape[0] for g in got) < cnt:
            c = rng.uniform(-0.5, 0.5, size=(4 * cnt, 3))
            r = np.linalg.norm(c, axis=1)
            ct = np.divide(c[:, 2], r, out=np.zeros_like(r), where=r > 0)
            p4 = (35 * ct ** 4 - 30 * ct ** 2 + 3) / 8.0
            keep = r < 0.5 - a + a * p4
            got.append(c[keep])
        g = np.concatenate(got)[:cnt]
        g[:, 2] += zc
        pts.append(g)
        lay.append(np.full(cnt, l, dtype=np.int32))
    xyz = np.concatenate(pts)
    layer = np.concatenate(lay)
    q = rng.uniform(-1.0, 1.0, size=xyz.shape[0])
    return Workload("paper_p4_%d" % xyz.shape[0], np.array(D_CONFIG), np.array(EPS_PAPER), xyz, layer, q)


def uneven_problems(k: int = 48, nmin: int = 2000, nmax: int = 100000, seed: int | None = None,
                    eps=EPS_CONFIG) -> list:
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 7 if seed is None else seed))
    sizes = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=k)).astype(np.int64)
    seeds = rng.integers(0, 2 ** 31, size=k)
    return [config2(int(n), seed=int(sd), eps=eps) for n, sd in zip(sizes, seeds)]


D_FOUR = (0.0, -0.6, -1.2)          # inner layers of equal thickness: interfaces are grid planes
D_FOUR_UNALIGNED = (0.0, -0.55, -1.2371)  # gaps with no common unit: cells straddle interfaces
EPS_FOUR = (2.0, 7.0, 1.5, 12.0)


def four_layers(n: int = 4000, seed: int | None = None, d=D_FOUR, eps=EPS_FOUR, margin: float = 0.05) -> Workload:
    """Four layers, N split equally: a unit-thick slab above d0, the two inner
    layers (each kept `margin` from its interfaces) and a unit-thick slab
    below the last interface, x, y in [-0.5, 0.5], q ~ U[-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 8 if seed is None else seed))
    d = tuple(float(v) for v in d)
    spans = [(d[0] + 0.1, d[0] + 1.1), (d[1] + margin, d[0] - margin), (d[2] + margin, d[1] - margin),
             (d[2] - 1.1, d[2] - 0.1)]
    sizes = [n // 4] * 3 + [n - 3 * (n // 4)]
    parts = [(_box(rng, cnt, lo, hi), l) for l, (cnt, (lo, hi)) in enumerate(zip(sizes, spans))]
    xyz = np.concatenate([p for p, _ in parts])
    layer = np.concatenate([np.full(p.shape[0], l, dtype=np.int32) for p, l in parts])
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("four_layers_n%d" % n, np.array(d), np.array(eps, dtype=np.float64), xyz, layer, q)


D_FIVE = (0.0, -0.6, -1.2, -1.8)         # inner layers of equal thickness
D_FIVE_UNALIGNED = (0.0, -0.45, -1.1, -1.6371)
EPS_FIVE = (2.0, 7.0, 1.5, 12.0, 4.0)


def five_layers(n: int = 5000, seed: int | None = None, d=D_FIVE, eps=EPS_FIVE, margin: float = 0.05,
                near: float = 0.0) -> Workload:
    """Five layers, N split equally: a unit-thick slab above d0, the three
    inner layers (each kept `margin` from its interfaces) and a unit-thick
    slab below the last interface, x, y in [-0.5, 0.5], q ~ U[-1, 1].  With
    near > 0 every charge lies instead between 1e-3 and `near` from an
    interface on its own side (the eight sides split equally)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 10 if seed is None else seed))
    d = tuple(float(v) for v in d)
    if near > 0.0:
        spans = []
        for j, dj in enumerate(d):
            spans.append(((dj + 1e-3, dj + near), j))
            spans.append(((dj - near, dj - 1e-3), j + 1))
        sizes = [n // 8] * 7 + [n - 7 * (n // 8)]
        parts = [(_box(rng, cnt, lo, hi), l) for cnt, ((lo, hi), l) in zip(sizes, spans)]
    else:
        spans = [(d[0] + 0.1, d[0] + 1.1)] + [(d[j] + margin, d[j - 1] - margin) for j in range(1, 4)] + \
                [(d[3] - 1.1, d[3] - 0.1)]
        sizes = [n // 5] * 4 + [n - 4 * (n // 5)]
        parts = [(_box(rng, cnt, lo, hi), l) for l, (cnt, (lo, hi)) in enumerate(zip(sizes, spans))]
    xyz = np.concatenate([p for p, _ in parts])
    layer = np.concatenate([np.full(p.shape[0], l, dtype=np.int32) for p, l in parts])
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("five_layers_n%d" % n, np.array(d), np.array(eps, dtype=np.float64), xyz, layer, q)


def four_layers_near_interface(n: int = 3000, delta: float = 0.02, hmin: float = 1e-3, seed: int | None = None,
                               d=D_FOUR, eps=EPS_FOUR) -> Workload:
    """Four layers, every charge between ``hmin`` and ``delta`` from an
    interface on its own side: N split equally between the six sides of the
    three interfaces (above and below each), x, y in [-0.5, 0.5],
    q ~ U[-1, 1].  The near field then holds reaction interactions of every
    layer pair, which the general-medium near-field kernels evaluate."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 9 if seed is None else seed))
    d = tuple(float(v) for v in d)
    spans = []
    for j, dj in enumerate(d):
        spans.append(((dj + hmin, dj + delta), j))          # layer j, above interface j
        spans.append(((dj - delta, dj - hmin), j + 1))      # layer j + 1, below it
    sizes = [n // 6] * 5 + [n - 5 * (n // 6)]
    parts = [(_box(rng, cnt, lo, hi), l) for cnt, ((lo, hi), l) in zip(sizes, spans)]
    xyz = np.concatenate([p for p, _ in parts])
    layer = np.concatenate([np.full(p.shape[0], l, dtype=np.int32) for p, l in parts])
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("four_layers_near_interface_n%d" % n, np.array(d), np.array(eps, dtype=np.float64), xyz,
                    layer, q)


def slab(n: int = 4000, half_width: float = 50.0, seed: int | None = None, eps=EPS_CONFIG,
         margin: float = 0.01) -> Workload:
    """A flat, wide layout (interconnect-like): x over [-half_width, half_width],
    y over [-0.1, 0.1], z over [-2.5, 1.0] across the three layers of config 2,
    every charge at least `margin` from an interface.  Most reaction pairs are
    then laterally far (rho up to 2 half_width) and shallow, so they stay in
    the near field."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 11 if seed is None else seed))
    d0, d1 = D_CONFIG
    x = rng.uniform(-half_width, half_width, n)
    y = rng.uniform(-0.1, 0.1, n)
    z = rng.uniform(-2.5, 1.0, n)
    for di in (d0, d1):  # keep the margin: push charges off the interfaces
        close = np.abs(z - di) < margin
        z[close] = di + np.where(z[close] >= di, margin, -margin)
    layer = np.where(z > d0, 0, np.where(z > d1, 1, 2)).astype(np.int32)
    q = rng.uniform(-1.0, 1.0, size=n)
    return Workload("slab_n%d_w%g" % (n, half_width), np.array(D_CONFIG), np.array(eps, dtype=np.float64),
                    np.column_stack([x, y, z]), layer, q)


def subsample(n: int, count: int, seed: int = SEED_BASE + 3) -> np.ndarray:
    """The first ``count`` indices of a seeded permutation of range(n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.permutation(n)[:count]).astype(np.int64)
