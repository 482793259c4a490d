"""GPU tests of the batched form: many independent, uneven problems evaluated
together, captured once into a CUDA graph and replayed.  Every problem of a
batch must reproduce its own one-at-a-time evaluation, and sampled targets
must match the direct-sum oracle."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, LayeredFMMBatch, LfmmError, workloads
from paper_1908_10863_gb300.lfmm import EINVAL, ESTATE, OPT_PRECISION, OPT_PROFILE

pytestmark = pytest.mark.gpu


def _members(problems, p, precision):
    out = []
    for w in problems:
        f = LayeredFMM(w.d, w.eps, p, precision=precision)
        f.build(w.xyz, w.layer)
        out.append(f)
    return out


def _close(ms):
    for m in ms:
        m.close()


def _charges(problems, seed, nrhs=None):
    rng = np.random.default_rng(seed)
    nr = nrhs or [1] * len(problems)
    return [rng.uniform(-1, 1, (r, w.n)) if r > 1 else rng.uniform(-1, 1, w.n) for w, r in zip(problems, nr)]


def _worst(a_list, b_list):
    return max(oracle.err2(a, b) for a, b in zip(a_list, b_list))


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_graph_matches_single_evaluations(precision, tol):
    probs = workloads.uneven_problems(7, 2000, 30000, seed=5)
    ms = _members(probs, 8, precision)
    try:
        with LayeredFMMBatch(ms) as b:
            for it in range(3):  # direct run + capture, then two graph replays with new charges
                qs = _charges(probs, 100 + it)
                phi, E = b.evaluate(qs)
                singles = [m.evaluate(q) for m, q in zip(ms, qs)]
                ep = _worst(phi, [s[0] for s in singles])
                ef = _worst(E, [s[1] for s in singles])
                print("iteration %d: batch vs single Err2 phi %.2e field %.2e" % (it, ep, ef))
                assert ep < tol and ef < tol
            info = b.info()
    finally:
        _close(ms)
    print(info)
    assert info["direct_runs"] == 1 and info["captures"] == 1 and info["graph_launches"] == 2
    assert info["kernel_nodes"] >= 7 * 5 and info["timeouts"] == 0  # every problem's stages are in the graph


def test_batch_mixed_media_multi_rhs_and_oracle():
    # problems in different media (three layers of two contrasts, two layers),
    # one of them with three charge vectors
    w0 = workloads.config2(6000, seed=1)
    w1 = workloads.config2(15000, seed=2, eps=workloads.EPS_HIGH_CONTRAST)
    w2 = workloads.config1(3000, seed=3)
    rng = np.random.default_rng(4)
    xyz = np.column_stack([rng.uniform(-0.5, 0.5, (5000, 2)), rng.uniform(-1.0, 1.0, 5000)])
    xyz[np.abs(xyz[:, 2]) < 1e-3, 2] = 0.5
    layer = (xyz[:, 2] < 0).astype(np.int32)
    two = workloads.Workload("two_layer", np.array([0.0]), np.array([1.0, 4.0]), xyz, layer,
                             rng.uniform(-1, 1, 5000))
    probs = [w0, w1, w2, two]
    nrhs = [1, 3, 1, 1]
    ms = _members(probs, 10, 0)
    try:
        with LayeredFMMBatch(ms, nrhs=nrhs) as b:
            qs = _charges(probs, 7, nrhs)
            b.evaluate(qs)
            phi, E = b.evaluate(qs)  # graph replay
            assert b.info()["graph_launches"] == 1
            singles = [m.evaluate(q) for m, q in zip(ms, qs)]
            assert _worst(phi, [s[0] for s in singles]) < 1e-12
            assert _worst(E, [s[1] for s in singles]) < 1e-12
        for i, w in enumerate(probs):
            three = len(w.d) == 2  # image series for three layers, adaptive quadrature otherwise
            t = workloads.subsample(w.n, 80 if three else 16)
            q = qs[i][1] if nrhs[i] > 1 else qs[i]
            ph = phi[i][1] if nrhs[i] > 1 else phi[i]
            ref, _ = oracle.direct(w.d, w.eps, w.xyz, w.layer, q, targets=t,
                                   mode=oracle.MODE_IMAGES if three else oracle.MODE_QUAD)
            e = oracle.err2(ref, ph[t])
            print("%s: Err2 vs oracle %.2e" % (w.name, e))
            assert e < 1e-5  # p = 10 truncation on sampled targets, as for single problems
    finally:
        _close(ms)


def test_batch_device_buffers_and_recapture():
    torch = pytest.importorskip("torch")
    probs = workloads.uneven_problems(5, 2000, 20000, seed=8)
    ms = _members(probs, 8, 1)
    dev = torch.device("cuda")
    try:
        with LayeredFMMBatch(ms) as b:
            qs = _charges(probs, 9)
            ref_phi, ref_E = b.evaluate(qs)
            q = torch.from_numpy(b.concat(qs)).to(dev)
            phi = torch.empty_like(q)
            fld = torch.empty(3 * b.total, dtype=torch.float64, device=dev)
            s = torch.cuda.Stream()
            for _ in range(2):
                with torch.cuda.stream(s):
                    phi.zero_()
                    b.evaluate_device(q, phi, fld, s)
                s.synchronize()
                got_phi = b.split(phi.cpu().numpy())
                got_E = b.split(fld.cpu().numpy(), True)
                assert _worst(ref_phi, got_phi) < 1e-6 and _worst(ref_E, got_E) < 1e-6
            info = b.info()
            # host staging buffers first, then the device tensors: two captures, one direct run
            assert info["captures"] == 2 and info["direct_runs"] == 1 and info["graph_launches"] == 2
            # a member changes: one direct run and a new capture, still right
            ms[2].set_option(OPT_PRECISION, 0)
            phi2, _ = b.evaluate(qs)
            single = ms[2].evaluate(qs[2])
            assert oracle.err2(single[0], phi2[2]) < 1e-12
            info = b.info()
            assert info["direct_runs"] == 2 and info["captures"] == 3
    finally:
        _close(ms)


def test_batch_without_graph_matches():
    probs = workloads.uneven_problems(4, 2000, 10000, seed=12)
    ms = _members(probs, 6, 0)
    try:
        qs = _charges(probs, 13)
        with LayeredFMMBatch(ms, graph=False) as b:
            phi0, _ = b.evaluate(qs)
            phi1, _ = b.evaluate(qs)
            assert b.info()["graph_nodes"] == 0 and b.info()["direct_runs"] == 2
        with LayeredFMMBatch(ms) as b:
            b.evaluate(qs)
            phi2, _ = b.evaluate(qs)
        assert _worst(phi0, phi1) < 1e-12 and _worst(phi0, phi2) < 1e-12
    finally:
        _close(ms)


def test_batch_argument_and_state_errors():
    w = workloads.config2(3000)
    a = LayeredFMM(w.d, w.eps, 6)
    c = LayeredFMM(w.d, w.eps, 6)
    try:
        a.build(w.xyz, w.layer)
        with pytest.raises(LfmmError) as ei:
            LayeredFMMBatch([a, a])
        assert ei.value.status == EINVAL
        with pytest.raises(LfmmError) as ei:
            LayeredFMMBatch([a, c])  # c is not built
        assert ei.value.status == ESTATE
        c.build(w.xyz, w.layer)
        with LayeredFMMBatch([a, c]) as b:
            with pytest.raises(ValueError):
                b.evaluate([w.q])
            c.set_option(OPT_PROFILE, 1)
            with pytest.raises(LfmmError) as ei:
                b.evaluate([w.q, w.q])
            assert ei.value.status == ESTATE
            c.set_option(OPT_PROFILE, 0)
            phi, _ = b.evaluate([w.q, w.q])
            assert oracle.err2(phi[0], phi[1]) < 1e-12
    finally:
        a.close()
        c.close()


def test_batch_autotune_times_the_whole_graph():
    # the tuner applies each candidate to every member, times graph replays of
    # the whole batch and leaves the winner set; results stay those of the
    # members evaluated one at a time (float32 form), and against the oracle
    probs = workloads.uneven_problems(8, 2000, 40000, seed=9)
    ms = _members(probs, 8, 1)
    try:
        with LayeredFMMBatch(ms) as b:
            rows = b.autotune(reps=2)
            print("batch tuner:", rows)
            assert len(rows) == 9 and sum(r["chosen"] for r in rows) == 1
            best = [r for r in rows if r["chosen"]][0]
            assert best["ms"] == min(r["ms"] for r in rows) and all(r["ms"] > 0 for r in rows)
            qs = _charges(probs, 7)
            phi, E = b.evaluate(qs)
            singles = [m.evaluate(q) for m, q in zip(ms, qs)]
            assert _worst(phi, [s[0] for s in singles]) < 1e-6
            w = probs[3]
            t = workloads.subsample(w.n, 60)
            ref, _ = oracle.direct(w.d, w.eps, w.xyz, w.layer, qs[3], targets=t, mode=oracle.MODE_IMAGES)
            assert oracle.err2(ref, phi[3][t]) < 1e-5
            assert b.info()["timeouts"] == 0
    finally:
        _close(ms)


def test_batch_autotune_needs_the_graph():
    probs = workloads.uneven_problems(2, 2000, 4000, seed=3)
    ms = _members(probs, 6, 1)
    try:
        with LayeredFMMBatch(ms, graph=False) as b:
            with pytest.raises(LfmmError) as ei:
                b.autotune(reps=1)
            assert ei.value.status == ESTATE
    finally:
        _close(ms)
