"""Wall-clock timing of the CPU oracle (test infrastructure, like the rest of
this package): the cost of the plain O(N^2) definition that the GPU path is
checked against.

    python -m oracle.timing [--quick]

Prints one JSON line per case:
  * full N^2 sums (every charge a target) on the three-layer workload of
    Section 4's accuracy tests, N in {250, 500, 1000, 2000, 4000}, exact image
    series, on one thread and on all host threads, with the fitted exponent
    alpha of t ~ N^alpha;
  * the same with the adaptive-quadrature densities for N <= 500 (the mode
    that also covers media without a closed form);
  * a 2,000-target subsample against all sources at N = 65,536, 262,144 and
    1,048,576 (image series), the way the benchmark's accuracy is measured.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import MODE_IMAGES, MODE_QUAD, direct


def _workload(n: int, seed: int):
    # three layers d = (0, -1.2), eps = (1, 5, 10), N split equally between
    # the layers (top z in [0.1, 1.1], middle [-1.1, -0.1], bottom [-2.3, -1.3]),
    # x, y in [-0.5, 0.5], q ~ U[-1, 1]
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [n // 3, n - 2 * (n // 3), n // 3]
    spans = [(0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3)]
    xyz = np.concatenate([np.column_stack([rng.uniform(-0.5, 0.5, (k, 2)), rng.uniform(lo, hi, k)])
                          for k, (lo, hi) in zip(sizes, spans)])
    layer = np.concatenate([np.full(k, l, dtype=np.int32) for l, k in enumerate(sizes)])
    q = rng.uniform(-1.0, 1.0, n)
    return [0.0, -1.2], [1.0, 5.0, 10.0], xyz, layer, q


def _time(fn, reps=1):
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        best = min(best, time.perf_counter() - t0)
    return best


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="smaller sizes (a few seconds)")
    args = ap.parse_args()
    cores = os.cpu_count() or 1
    sizes = [250, 500, 1000] if args.quick else [250, 500, 1000, 2000, 4000]
    for mode, mname, ns in ((MODE_IMAGES, "image series", sizes), (MODE_QUAD, "adaptive quadrature", sizes[:2])):
        for threads in (1, cores):
            ts = []
            for n in ns:
                d, eps, xyz, lay, q = _workload(n, 20190829 + n)
                ts.append(_time(lambda: direct(d, eps, xyz, lay, q, mode=mode, threads=threads)))
            alpha = float(np.polyfit(np.log(ns), np.log(ts), 1)[0]) if len(ns) > 1 else None
            print(json.dumps({"case": "full N^2", "mode": mname, "threads": threads, "N": ns,
                              "seconds": [round(t, 4) for t in ts],
                              "pairs_per_s": [round(n * n / t) for n, t in zip(ns, ts)],
                              "alpha": None if alpha is None else round(alpha, 3)}), flush=True)
    subs = [65536] if args.quick else [65536, 262144, 1048576]
    for n in subs:
        d, eps, xyz, lay, q = _workload(n, 20190829 + 2)
        t = np.sort(np.random.default_rng(20190829 + 3).choice(n, 2000, replace=False))
        sec = _time(lambda: direct(d, eps, xyz, lay, q, targets=t, mode=MODE_IMAGES, threads=cores))
        print(json.dumps({"case": "2000-target subsample", "mode": "image series", "threads": cores, "N": n,
                          "seconds": round(sec, 3), "pairs_per_s": round(2000 * n / sec)}), flush=True)


if __name__ == "__main__":
    main()
