"""GPU parity: the CUDA path through the C ABI against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, LfmmError, workloads

pytestmark = pytest.mark.gpu
D3 = [0.0, -1.2]
EPS = [1.0, 5.0, 10.0]


def _cube(n, seed, lo=-0.5, hi=0.5):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, 3)), rng.uniform(-1, 1, n)


@pytest.mark.parametrize("p,tol", [(4, 3e-3), (8, 1e-4), (12, 1e-5), (20, 1e-8)])
def test_free_space_matches_direct_sum(p, tol):
    xyz, q = _cube(3000, 1)
    lay = np.zeros(3000, np.int32)
    with LayeredFMM([], [1.0], p) as f:
        f.build(xyz, lay)
        phi, E = f.evaluate(q)
    ref, refE = oracle.direct([], [1.0], xyz, lay, q, mode=oracle.MODE_FREE_ONLY)
    assert oracle.err2(ref, phi) < tol
    assert oracle.err2(refE, E) < 10 * tol


def test_two_layer_matches_image_charge_oracle():
    rng = np.random.default_rng(2)
    n = 2000
    lay = rng.integers(0, 2, n).astype(np.int32)
    xyz = rng.uniform(-0.5, 0.5, (n, 3))
    xyz[:, 2] = np.where(lay == 0, rng.uniform(0.05, 1.0, n), -rng.uniform(0.05, 1.0, n))
    q = rng.uniform(-1, 1, n)
    with LayeredFMM([0.0], [2.0, 7.0], 12) as f:
        f.build(xyz, lay)
        phi, E = f.evaluate(q)
    ref, refE = oracle.direct([0.0], [2.0, 7.0], xyz, lay, q, mode=oracle.MODE_QUAD)
    assert oracle.err2(ref, phi) < 1e-5
    assert oracle.err2(refE, E) < 1e-4


COMPS = [(0, 0, 1, 1), (1, 0, 2, 1), (1, 0, 1, 1), (2, 0, 2, 1), (0, 1, 1, 2), (0, 1, 1, 1), (1, 1, 1, 1),
         (1, 1, 2, 1), (1, 1, 1, 2), (1, 1, 2, 2), (2, 1, 2, 2), (2, 1, 2, 1), (0, 2, 1, 2), (1, 2, 2, 2),
         (1, 2, 1, 2), (2, 2, 2, 2)]


@pytest.mark.parametrize("eps", [EPS, [1.0, 80.0, 2.0]])
def test_sommerfeld_tables_match_image_series(eps):
    P = 10
    with LayeredFMM(D3, eps, P) as f:
        for comp in COMPS:
            for S, (rh, zh) in [(0.6, (1.0, 2.0)), (0.15, (0.0, 2.0)), (0.15, (2.0 ** 0.5, 3.0)),
                                (0.0375, (3.0, 2.0)), (1.2, (1.0, 1.0))]:
                T = f.sommerfeld_tables(*comp, [rh * S], [zh * S], S, P)[0]
                worst = 0.0
                for N in range(0, 2 * P + 1, 3):
                    row = np.array([S ** (N + 1) * oracle.sommerfeld_K_images(D3, eps, *comp, N, mu, rh * S, zh * S)
                                    for mu in range(N + 1)])
                    sc = np.max(np.abs(row))
                    worst = max(worst, np.max(np.abs(T[N, :N + 1] - row)) / sc)
                assert worst < 1e-11, (comp, S, rh, zh, worst)


@pytest.mark.parametrize("eps", [EPS, [1.0, 80.0, 2.0]])
def test_reaction_near_kernel_matches_image_series(eps):
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.0, 0.6, 40)
    h = rng.uniform(0.15, 2.0, 40)
    with LayeredFMM(D3, eps, 4) as f:
        for comp in COMPS:
            got = f.reaction_kernel(*comp, rho, h)
            ref = np.array([[oracle.sommerfeld_K_images(D3, eps, *comp, 0, 0, r, z),
                             oracle.sommerfeld_K_images(D3, eps, *comp, 1, 0, r, z),
                             oracle.sommerfeld_K_images(D3, eps, *comp, 1, 1, r, z)] for r, z in zip(rho, h)])
            # high contrast (|q| = 0.93): composite Legendre/Laguerre rule, ~3e-13
            tol = 1e-12
            assert np.max(np.abs(got - ref) / (np.abs(ref[:, :1]) + 1e-300)) < tol, comp


# measured: p=6 1.1e-4, p=10 2.6e-6, p=14 9.7e-8 (one-box separation);
# p=20 7.4e-11 (orders >= 18 also need a centre distance of sqrt(6) boxes)
@pytest.mark.parametrize("p,tol", [(6, 3e-4), (10, 5e-6), (14, 2e-7), (20, 1e-9)])
def test_config1_three_layer_full_oracle(p, tol):
    w = workloads.config1(1000)
    with LayeredFMM(w.d, w.eps, p) as f:
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q)
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, mode=oracle.MODE_IMAGES)
    e2 = oracle.err2(ref, phi)
    print("config1 p=%d Err2(phi)=%.3e Err2(E)=%.3e" % (p, e2, oracle.err2(refE, E)))
    assert e2 < tol
    assert oracle.err2(refE, E) < 20 * tol


def test_config2_mixed_layers_sampled():
    w = workloads.config2(20000)
    t = workloads.subsample(w.n, 300)
    with LayeredFMM(w.d, w.eps, 10) as f:
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q)
        st = f.stats()
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES)
    print("config2 N=20000 p=10 stats", st, "Err2", oracle.err2(ref, phi[t]))
    assert oracle.err2(ref, phi[t]) < 1e-5
    assert oracle.err2(refE, E[t]) < 1e-4


def test_fp32_form_config1():
    w = workloads.config1(1000)
    with LayeredFMM(w.d, w.eps, 10, precision=1) as f:
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q)
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, mode=oracle.MODE_IMAGES)
    print("fp32 config1 p=10 Err2", oracle.err2(ref, phi), oracle.err2(refE, E))
    assert oracle.err2(ref, phi) < 3e-5


def test_single_and_tiny_inputs():
    for n in (1, 2, 7):
        w = workloads.config2(n=max(n, 3), seed=5)
        xyz, lay, q = w.xyz[:n], w.layer[:n], w.q[:n]
        with LayeredFMM(w.d, w.eps, 8) as f:
            f.build(xyz, lay)
            phi, E = f.evaluate(q)
        ref, refE = oracle.direct(w.d, w.eps, xyz, lay, q, mode=oracle.MODE_IMAGES)
        assert np.allclose(phi, ref, rtol=1e-9, atol=1e-12), (n, phi, ref)
        assert np.allclose(E, refE, rtol=1e-8, atol=1e-11)


def test_rejects_points_outside_their_layer():
    w = workloads.config1(50)
    bad = w.xyz.copy()
    bad[7, 2] = 0.3  # above the top interface but tagged middle layer
    with LayeredFMM(w.d, w.eps, 6) as f:
        with pytest.raises(LfmmError) as ei:
            f.build(bad, w.layer)
        assert "EINVAL" in str(ei.value)
        with pytest.raises(LfmmError):
            f.evaluate(w.q)  # no successful build yet
        f.build(w.xyz, w.layer)  # context still usable
        phi, _ = f.evaluate(w.q)
        assert np.all(np.isfinite(phi))


# measured Err2 (phi, field): 3.45e-6 4.7e-6 (FP64), 3.46e-6 5.2e-6 (float32)
@pytest.mark.parametrize("precision,tol_phi,tol_fld", [(0, 6e-6, 1.2e-5), (1, 6e-6, 1.5e-5)])
def test_near_interface_forms_match_oracle(precision, tol_phi, tol_fld):
    # every charge within 0.02 of an interface: the near field holds reaction
    # pairs (float32 form: offsets from leaf centres, compensated sums); each
    # form against the oracle's exact image series on sampled targets
    w = workloads.near_interface(16000)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q)
        st = f.stats()
    assert st["p2p_reaction"] > 0
    t = workloads.subsample(w.n, 300)
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES)
    e_phi, e_fld = oracle.err2(ref, phi[t]), oracle.err2(refE, E[t])
    print("near_interface 16k precision %d: Err2 phi %.2e field %.2e" % (precision, e_phi, e_fld))
    assert e_phi < tol_phi
    assert e_fld < tol_fld


@pytest.mark.parametrize("p", [4, 8, 10, 12, 14])
def test_precision_change_after_build_reassembles_reaction_operators(p):
    # the keyed reaction operators are assembled at build time in the build's
    # precision; a later precision change must assemble them again
    w = workloads.config2(20000)
    with LayeredFMM(w.d, w.eps, p) as f:
        f.build(w.xyz, w.layer)
        assert f.stats()["reaction_keys"] > 0
        ref64 = f.evaluate(w.q)
        f.set_option(1, 1)
        got32 = f.evaluate(w.q)
        f.set_option(1, 0)
        again64 = f.evaluate(w.q)
    with LayeredFMM(w.d, w.eps, p, precision=1) as g:
        g.build(w.xyz, w.layer)
        ref32 = g.evaluate(w.q)
    assert oracle.err2(ref64[0], again64[0]) < 1e-13
    assert oracle.err2(ref32[0], got32[0]) < 1e-6
    assert oracle.err2(ref64[0], got32[0]) < 1e-5


def test_rebuild_larger_geometry_grows_the_lists():
    # list arrays keep the capacity of the first build; a much larger
    # geometry overflows them once and is rebuilt with measured capacities
    small = workloads.config2(2000, seed=3)
    big = workloads.config2(150000, seed=4)
    with LayeredFMM(big.d, big.eps, 6) as f:
        f.build(small.xyz, small.layer)
        f.evaluate(small.q)
        f.build(big.xyz, big.layer)
        phi, E = f.evaluate(big.q)
        st = f.stats()
    with LayeredFMM(big.d, big.eps, 6) as g:
        g.build(big.xyz, big.layer)
        phi0, E0 = g.evaluate(big.q)
        st0 = g.stats()
    for k in ("boxes", "m2l_free", "m2l_reaction", "p2p_free", "p2p_reaction"):
        assert st[k] == st0[k], k
    assert oracle.err2(phi0, phi) < 1e-13
    assert oracle.err2(E0, E) < 1e-13


def test_host_inputs_checked_before_device_work():
    w = workloads.config2(300000, seed=5)  # large enough for the threaded checks
    with LayeredFMM(w.d, w.eps, 6) as f:
        for bad_i, what in ((123456, "nan"), (299999, "layer"), (7, "inf")):
            xyz = w.xyz.copy()
            lay = w.layer.copy()
            if what == "nan":
                xyz[bad_i, 0] = np.nan
            elif what == "inf":
                xyz[bad_i, 2] = np.inf
            else:
                lay[bad_i] = 3
            with pytest.raises(LfmmError) as ei:
                f.build(xyz, lay)
            assert "EINVAL" in str(ei.value), what
        f.build(w.xyz, w.layer)
        q = w.q.copy()
        q[200000] = np.nan
        with pytest.raises(LfmmError) as ei:
            f.evaluate(q)
        assert "ENUMERIC" in str(ei.value)
        phi = np.empty(w.n)
        E = np.empty((w.n, 3))
        r = f.evaluate(w.q, out=(phi, E))
        assert r[0] is phi and r[1] is E
        ref_phi, ref_E = f.evaluate(w.q)
        assert np.array_equal(phi, ref_phi) or oracle.err2(ref_phi, phi) < 1e-14


def test_device_inputs_checked_on_the_device():
    # build_device has no host copy to check: the key kernel flags bad points
    # and the build returns EINVAL, leaving the context usable
    torch = pytest.importorskip("torch")
    w = workloads.config2(50000, seed=6)
    dev = torch.device("cuda")
    with LayeredFMM(w.d, w.eps, 6) as f:
        for what in ("nan", "layer"):
            xyz = w.xyz.copy()
            lay = w.layer.copy()
            if what == "nan":
                xyz[4321, 1] = np.nan
            else:
                lay[4321] = -1
            with pytest.raises(LfmmError) as ei:
                f.build_device(torch.from_numpy(xyz).to(dev), torch.from_numpy(lay).to(dev))
            assert "EINVAL" in str(ei.value), what
        f.build_device(torch.from_numpy(w.xyz).to(dev), torch.from_numpy(w.layer).to(dev))
        phi, _ = f.evaluate(w.q)
        assert np.all(np.isfinite(phi))


@pytest.mark.parametrize("precision,tol", [(1, 1e-5), (0, 1e-5)])
def test_full_size_sampled_against_oracle(precision, tol):
    # the benchmark's own workload and call path (device buffers, N = 1M,
    # p = 10), checked on a seeded sample of targets the oracle computes one by one
    torch = pytest.importorskip("torch")
    w = workloads.config2(1 << 20)
    t = workloads.subsample(w.n, 48, seed=11)
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES)
    dev = torch.device("cuda")
    s = torch.cuda.current_stream()
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build_device(torch.from_numpy(w.xyz).to(dev), torch.from_numpy(w.layer).to(dev), s)
        q = torch.from_numpy(w.q).to(dev)
        phi = torch.empty_like(q)
        fld = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
        f.evaluate_device(q, phi, fld, s)
        torch.cuda.synchronize()
        st = f.stats()
    e_phi = oracle.err2(ref, phi.cpu().numpy()[t])
    e_fld = oracle.err2(refE, fld.cpu().numpy()[t])
    print("N=1M precision %d: Err2 phi %.2e field %.2e (48 targets), %d free M2L pairs" % (precision, e_phi, e_fld,
                                                                                        st["m2l_free"]))
    assert st["timeouts"] == 0
    assert e_phi < tol and e_fld < 5 * tol


@pytest.mark.parametrize("p,tol", [(12, 1e-6), (14, 3e-7)])
def test_keyed_reaction_m2l_high_order_against_oracle(p, tol):
    # orders 11 .. 15 stage each key's operator in chunks; FP64 against the
    # exact image series (measured at N = 20,000: p = 12 ~5e-7, p = 14 ~1e-7)
    w = workloads.config2(20000)
    with LayeredFMM(w.d, w.eps, p) as f:
        f.build(w.xyz, w.layer)
        st = f.stats()
        phi, E = f.evaluate(w.q)
    assert st["reaction_keys"] > 0
    t = workloads.subsample(w.n, 300)
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES)
    e = oracle.err2(ref, phi[t])
    print("config2 20k p=%d FP64 keyed reaction M2L: Err2 phi %.2e field %.2e" % (p, e, oracle.err2(refE, E[t])))
    assert e < tol


@pytest.mark.parametrize("half_width", [10.0, 50.0])
@pytest.mark.parametrize("precision,tol_phi,tol_fld", [(0, 2e-5, 5e-6), (1, 5e-5, 1e-4)])
def test_flat_wide_layout_against_oracle(half_width, precision, tol_phi, tol_fld):
    # Reaction pairs up to 100 apart laterally but shallow (rho >> depth) stay
    # in the near field; their remainder splits into images and a quadrature
    # at a deeper depth.  With the Gauss-Laguerre rule alone the potential was
    # off by Err2 2e-4 (half width 10) and 9e-3 (half width 50).
    w = workloads.slab(4000, half_width)
    with LayeredFMM(w.d, w.eps, 10, precision=precision) as f:
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q)
        st = f.stats()
    assert st["p2p_reaction"] > 0 and st["timeouts"] == 0
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, mode=oracle.MODE_IMAGES)
    e, ef = oracle.err2(ref, phi), oracle.err2(refE, E)
    print("slab half width %g precision %d: Err2 phi %.2e field %.2e (p2p_reaction %d)"
          % (half_width, precision, e, ef, st["p2p_reaction"]))
    assert e < tol_phi and ef < tol_fld
