"""GPU tests of the learned near-field reaction kernels (the surrogate network).

* the training kernels' loss and gradient against the FP64 oracle of the
  network (oracle/mlp.py);
* the tensor-core inference kernel against the same oracle's forward pass;
* a trained network against the image-series oracle of the Sommerfeld
  kernels, where its error table accepts a pair;
* the FMM with the network in the near field against the direct-sum oracle,
  and what the network gains over the quadrature there.
"""
import time

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1908_10863_gb300 import LayeredFMM, LfmmError, workloads
from paper_1908_10863_gb300.lfmm import OPT_PROFILE, OPT_SURROGATE

pytestmark = pytest.mark.gpu
D3 = [0.0, -1.2]
EPS = [1.0, 5.0, 10.0]
COMP = (1, 1, 1, 1)
COMPS = [(0, 0, 1, 1), (1, 0, 2, 1), (1, 0, 1, 1), (2, 0, 2, 1), (0, 1, 1, 2), (0, 1, 1, 1), (1, 1, 1, 1),
         (1, 1, 2, 1), (1, 1, 1, 2), (1, 1, 2, 2), (2, 1, 2, 2), (2, 1, 2, 1), (0, 2, 1, 2), (1, 2, 2, 2),
         (1, 2, 1, 2), (2, 2, 2, 2)]


def _theta(seed):
    rng = np.random.default_rng(seed)
    th = np.zeros(mlp.NPARAM)
    o = 0
    for name, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        if name.startswith("W"):
            a = np.sqrt(6.0 / (shp[0] + shp[1]))
            th[o:o + n] = rng.uniform(-a, a, n)
        else:
            th[o:o + n] = rng.uniform(-0.1, 0.1, n)
        o += n
    return th.astype(np.float32)


def test_training_gradient_matches_oracle():
    th = _theta(11)
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, (256, 4)).astype(np.float32)
    y = rng.normal(0, 1, (256, 3)).astype(np.float32)
    with LayeredFMM(D3, EPS, 4) as f:
        f.surrogate_set_params(*COMP, th)
        assert np.array_equal(f.surrogate_params(*COMP), th)
        loss, g = f.surrogate_loss_grad(*COMP, x, y)
    rl, rg = mlp.loss_and_grad(th.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    # per parameter block, relative to the block's largest oracle gradient
    o = 0
    for name, shp in mlp.SHAPES:
        n = int(np.prod(shp))
        scale = np.max(np.abs(rg[o:o + n]))
        err = np.max(np.abs(g[o:o + n] - rg[o:o + n])) / scale
        print("grad %s: max rel err %.2e" % (name, err))
        assert err < 1e-4, name
        o += n


def test_inference_kernel_matches_oracle_forward():
    th = _theta(21)
    rng = np.random.default_rng(22)
    x = rng.uniform(-1, 1, (1000, 4)).astype(np.float32)  # not a multiple of 32: ragged last warp
    with LayeredFMM(D3, EPS, 4) as f:
        f.surrogate_set_params(*COMP, th)
        y = f.surrogate_forward(*COMP, x)
    ref, _ = mlp.forward(th.astype(np.float64), x.astype(np.float64), quantize=True)
    err = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    print("inference: max err %.2e (relative to max |out|)" % err)
    # activations carry ~16 bits (bfloat16 high + low parts)
    assert err < 2e-4


def test_surrogate_needs_training():
    with LayeredFMM(D3, EPS, 4) as f:
        with pytest.raises(LfmmError):
            f.set_option(OPT_SURROGATE, 1)
        with pytest.raises(LfmmError):
            f.surrogate_eval(*COMP, [0.1], [0.01], [0.01])
    with LayeredFMM([0.0], [1.0, 3.0], 4) as f:  # two layers: closed form, nothing to learn
        with pytest.raises(LfmmError):
            f.surrogate_train(4096, 1, 1)


@pytest.fixture(scope="module")
def trained():
    f = LayeredFMM(D3, EPS, 10)
    t0 = time.perf_counter()
    f.surrogate_train(1 << 18, 32, 5)
    print("surrogate training: %.2f s" % (time.perf_counter() - t0))
    yield f
    f.close()


def test_trained_network_accuracy(trained):
    f = trained
    rng = np.random.default_rng(31)
    worst_acc = 0.0
    for comp in COMPS:
        info = f.surrogate_info(*comp)
        assert info["trained"] == 1.0
        n = 200
        rho = 10.0 ** rng.uniform(-3, np.log10(3.0), n)
        ht = 10.0 ** rng.uniform(-4, np.log10(1.2), n)
        hs = 10.0 ** rng.uniform(-4, np.log10(1.2), n)
        out = f.surrogate_eval(*comp, rho, ht, hs)
        ref = np.array([[oracle.sommerfeld_K_images(D3, EPS, *comp, N, mu, r, a + b)
                         for N, mu in ((0, 0), (1, 0), (1, 1))] for r, a, b in zip(rho, ht, hs)])
        e0 = np.abs(out[:, 0] - ref[:, 0]) / np.abs(ref[:, 0])
        e1 = np.hypot(out[:, 1] - ref[:, 1], out[:, 2] - ref[:, 2]) / np.hypot(ref[:, 1], ref[:, 2])
        acc = out[:, 3] > 0
        ea = np.maximum(e0, e1)[acc]
        print("%s: loss %.2e, max val err %.2e, cells ok %.2f, val samples ok %.2f; fresh: accepted %d/%d, "
              "max rel err accepted %.2e, all %.2e" % (comp, info["loss"], info["max_err"], info["cells_ok"],
                                                       info["samples_ok"], acc.sum(), n,
                                                       ea.max() if acc.any() else 0.0, np.maximum(e0, e1).max()))
        if acc.any():
            worst_acc = max(worst_acc, ea.max())
    assert worst_acc < 5e-6


def _sampled_err(w, phi, E, targets):
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=targets, mode=oracle.MODE_IMAGES)
    return oracle.err2(ref, phi[targets]), oracle.err2(refE, E[targets])


def test_fmm_with_surrogate_matches_oracle(trained):
    f = trained
    w = workloads.near_interface(12000)
    f.build(w.xyz, w.layer)
    st = f.stats()
    print("near_interface 12k stats:", st)
    assert st["p2p_reaction"] > 0
    phi0, E0 = f.evaluate(w.q)
    f.set_option(OPT_SURROGATE, 1)
    try:
        phi1, E1 = f.evaluate(w.q)
        st1 = f.stats()
    finally:
        f.set_option(OPT_SURROGATE, 0)
    print("pairs by network %d, by quadrature %d" % (st1["surr_net_pairs"], st1["surr_quad_pairs"]))
    assert st1["surr_net_pairs"] > 0
    targets = workloads.subsample(w.n, 300)
    e_off = _sampled_err(w, phi0, E0, targets)
    e_on = _sampled_err(w, phi1, E1, targets)
    d_on_off = oracle.err2(phi0, phi1)
    print("Err2 quadrature (phi, E) = %.2e %.2e; with network %.2e %.2e; network vs quadrature %.2e"
          % (e_off + e_on + (d_on_off,)))
    assert e_off[0] < 5e-6 and e_on[0] < 5e-6
    assert e_on[1] < 5e-5
    assert d_on_off < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_surrogate_gain_in_near_field(trained, precision):
    """Time the reaction near field (P2P stage) with and without the network
    on a workload whose near field is dominated by reaction pairs."""
    f = trained
    w = workloads.near_interface(1 << 18)
    f.set_option(1, precision)
    f.set_option(OPT_PROFILE, 1)
    try:
        f.build(w.xyz, w.layer)
        res = {}
        for use in (0, 1):
            f.set_option(OPT_SURROGATE, use)
            f.evaluate(w.q)  # warm-up
            ts = []
            for _ in range(3):
                phi, _ = f.evaluate(w.q)
                ts.append(f.timings()["p2p"])
            res[use] = (min(ts), phi, f.stats())
    finally:
        f.set_option(OPT_SURROGATE, 0)
        f.set_option(OPT_PROFILE, 0)
        f.set_option(1, 0)
    st = res[1][2]
    frac = st["surr_net_pairs"] / max(1, st["surr_net_pairs"] + st["surr_quad_pairs"])
    print("precision %d: P2P %.3f ms quadrature, %.3f ms network (%.2fx); %.1f%% of reaction pairs by network; "
          "network vs quadrature Err2(phi) %.2e" % (precision, res[0][0], res[1][0], res[0][0] / res[1][0],
                                                    100 * frac, oracle.err2(res[0][1], res[1][1])))
    assert frac > 0.0
    assert oracle.err2(res[0][1], res[1][1]) < (1e-6 if precision == 0 else 1e-5)
    gain = res[0][0] / res[1][0]
    if precision == 0:
        # FP64 form: the network (bfloat16 tensor-core MMAs) replaces the FP64
        # quadrature of about half the reaction pairs; measured 1.6-2.0x
        assert gain > 1.3
    else:
        # float32 form: the float32 quadrature is cheaper than the network
        # (measured 0.44x), so the network is a loss there
        assert gain < 1.0
