"""Host-side helpers of bench.py (no device): the per-layer split of Err2."""
import numpy as np

import bench


def test_err2_per_layer_splits_the_combined_error():
    rng = np.random.default_rng(2)
    n = 300
    layers = rng.integers(0, 3, n)
    ref = rng.normal(size=n) * (1 + layers)
    got = ref + 1e-6 * rng.normal(size=n)
    per = bench.err2_per_layer(ref, got, layers)
    assert sorted(per) == ["0", "1", "2"]
    for l, e in per.items():
        m = layers == int(l)
        assert e == np.sqrt(np.sum((ref[m] - got[m]) ** 2) / np.sum(ref[m] ** 2))
    # the squared errors and norms add up to the combined Err2
    num = sum(per[str(l)] ** 2 * np.sum(ref[layers == l] ** 2) for l in range(3))
    assert np.isclose(np.sqrt(num / np.sum(ref ** 2)), np.sqrt(np.sum((ref - got) ** 2) / np.sum(ref ** 2)))
    # vector-valued fields ([n, 3]) split the same way
    E = rng.normal(size=(n, 3))
    perE = bench.err2_per_layer(E, E * (1 + 1e-7), layers)
    assert all(abs(v - 1e-7) < 1e-12 for v in perE.values())
