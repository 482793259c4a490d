"""GPU tests of the batched evaluation: many charge vectors over one tree
(the GMRES matrix-vector use the paper motivates).  A batch must reproduce
the one-at-a-time evaluation of each vector, and match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, workloads

pytestmark = pytest.mark.gpu


def _charges(nrhs, n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (nrhs, n))


def _batch_vs_single(w, p, precision, Q, surrogate=False):
    with LayeredFMM(w.d, w.eps, p, precision=precision) as f:
        if surrogate:
            f.surrogate_train(1 << 15, 4, 3)
            f.set_option(5, 1)
        f.build(w.xyz, w.layer)
        phi_b, E_b = f.evaluate(Q)
        singles = [f.evaluate(q) for q in Q]
    e_phi = max(oracle.err2(s[0], phi_b[r]) for r, s in enumerate(singles))
    e_fld = max(oracle.err2(s[1], E_b[r]) for r, s in enumerate(singles))
    return phi_b, E_b, e_phi, e_fld


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_matches_single_evaluations(precision, tol):
    w = workloads.config2(20000)
    Q = _charges(5, w.n, 7)
    _, _, e_phi, e_fld = _batch_vs_single(w, 10, precision, Q)
    print("config2 20k, 5 vectors, precision %d: batch vs single Err2 phi %.2e field %.2e" % (precision, e_phi,
                                                                                              e_fld))
    assert e_phi < tol and e_fld < tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_reaction_near_field(precision, tol):
    # reaction pairs in the near field: the quadrature is shared by the batch
    w = workloads.near_interface(12000)
    Q = _charges(3, w.n, 8)
    _, _, e_phi, e_fld = _batch_vs_single(w, 10, precision, Q)
    print("near_interface 12k, 3 vectors, precision %d: Err2 phi %.2e field %.2e" % (precision, e_phi, e_fld))
    assert e_phi < tol and e_fld < tol


def test_batch_longer_than_one_pass_and_oracle():
    # 70 vectors: two passes (64 + 6), ragged near-field batches of 8
    w = workloads.config2(3000)
    Q = _charges(70, w.n, 9)
    phi_b, E_b, e_phi, e_fld = _batch_vs_single(w, 8, 0, Q)
    assert e_phi < 1e-12 and e_fld < 1e-12
    t = workloads.subsample(w.n, 100)
    for r in (0, 41, 69):
        ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, Q[r], targets=t, mode=oracle.MODE_IMAGES)
        assert oracle.err2(ref, phi_b[r][t]) < 1e-4
        assert oracle.err2(refE, E_b[r][t]) < 1e-3


def test_batch_with_network_near_field():
    w = workloads.near_interface(8000)
    Q = _charges(2, w.n, 10)
    _, _, e_phi, e_fld = _batch_vs_single(w, 10, 0, Q, surrogate=True)
    assert e_phi < 1e-12 and e_fld < 1e-12


def test_batch_device_buffers():
    torch = pytest.importorskip("torch")
    w = workloads.config2(10000)
    Q = _charges(4, w.n, 11)
    dev = torch.device("cuda")
    with LayeredFMM(w.d, w.eps, 10, precision=1) as f:
        f.build(w.xyz, w.layer)
        phi_h, E_h = f.evaluate(Q)
        q_d = torch.from_numpy(Q).to(dev)
        phi_d = torch.empty_like(q_d)
        fld_d = torch.empty((4, w.n, 3), dtype=torch.float64, device=dev)
        f.evaluate_device(q_d, phi_d, fld_d, torch.cuda.current_stream())
        torch.cuda.synchronize()
    # float32 form: the far field's float atomics may sum in another order
    assert oracle.err2(phi_h, phi_d.cpu().numpy()) < 1e-6
    assert oracle.err2(E_h, fld_d.cpu().numpy()) < 1e-6
