"""Host-side helpers of bench.py (no device): the per-layer split of Err2, the
roofline arithmetic and the label of the headline form."""
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


def test_roofline_arithmetic():
    # dense complex M2L: (p+1)^2 inputs x (p+1)(p+2)/2 outputs, 8 flops per complex MAC
    assert bench.m2l_flops_per_pair(10) == 63888
    assert bench.m2l_flops_per_pair(6) == 8 * 49 * 28
    # FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flops x clock
    assert np.isclose(bench.fp32_peak_tflops(2070.0), 152 * 128 * 2 * 2070e6 / 1e12)
    # dense TF32 peak: the measured bf16 burst times the nominal 1.1 / 2.25 ratio
    import json
    import os
    peak, src = bench.tf32_peak_tflops()
    path = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        assert src == "of measured" and np.isclose(peak, bf16 * 1.1 / 2.25)
    else:
        assert src == "of fallback" and np.isclose(peak, 1900.0 * 1.1 / 2.25)
    # DRAM traffic per free M2L pair from the committed capture: 278.4 MB for 10,905,072 pairs
    assert abs(bench.TC_DRAM_BYTES_PER_PAIR * 10905072 - 278.444544e6) < 1.0


def test_form_label_names_what_ran():
    idle = bench.form_label("fp32_surrogate", {"surr_net_pairs": 0, "surr_quad_pairs": 0})
    assert "idle" in idle and "plain FP32 form" in idle
    used = bench.form_label("fp32_surrogate", {"surr_net_pairs": 5, "surr_quad_pairs": 7})
    assert "kernels on (network pairs 5, quadrature pairs 7)" in used
    assert bench.form_label("fp64", {}) == "FP64 throughout"
