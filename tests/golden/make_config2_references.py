"""Write the CPU oracle's potentials and fields at seeded target subsamples
of the N = 1,048,576 three-layer workload (charges split equally between
the layers), for the GPU accuracy tests at full size.

Calls only ``oracle`` (exact three-layer image series, FP64 direct sum over
all sources) and the seeded input generators; no GPU code.  Each output file
also records a fingerprint of the workload (sums of the targets' positions
and of all charges) so that a test can check that the generator still draws
the same inputs before it trusts the stored values.

    python tests/golden/make_config2_references.py [threads]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1908_10863_gb300 import workloads  # noqa: E402

CASES = [  # (file, eps, targets)
    ("config2_n1m_eps1_5_10_targets2000.json", workloads.EPS_CONFIG, 2000),
    ("config2_n1m_eps1_80_2_targets400.json", workloads.EPS_HIGH_CONTRAST, 400),
]
N = 1 << 20


def fingerprint(w, t):
    return {"n": int(w.n), "sum_xyz_targets": float(np.sum(w.xyz[t])), "sum_q": float(np.sum(w.q)),
            "sum_abs_q_targets": float(np.sum(np.abs(w.q[t])))}


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    for fname, eps, count in CASES:
        path = os.path.join(HERE, fname)
        w = workloads.config2(N, eps=eps)
        t = workloads.subsample(w.n, count)
        t0 = time.perf_counter()
        phi, E = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES,
                               threads=threads)
        dt = time.perf_counter() - t0
        out = {"workload": "config2 (three-layer split), N=%d, d=(0,-1.2), eps=%s, q~U[-1,1]" % (N, list(eps)),
               "generator": "paper_1908_10863_gb300.workloads.config2(%d, eps=%s); targets "
                            "workloads.subsample(%d, %d)" % (N, tuple(eps), N, count),
               "oracle": "oracle.direct(mode=MODE_IMAGES): FP64 direct sum, exact three-layer image series",
               "oracle_seconds": round(dt, 1), "threads": threads,
               "fingerprint": fingerprint(w, t),
               "targets": [int(v) for v in t],
               "phi": [float(v) for v in phi],
               "field": [[float(v) for v in row] for row in E]}
        with open(path, "w") as fh:
            json.dump(out, fh, separators=(",", ":"))
        print("%s: %d targets in %.1f s" % (fname, count, dt), flush=True)


if __name__ == "__main__":
    main()
