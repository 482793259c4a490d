"""GPU tests of the tensor-core reaction M2L of the float32 form: each key's
operator formed in shared memory from its Sommerfeld table and lateral phases,
applied with 3xTF32 MMAs (eqs. metoleimage1, coefintable).  Checked against the
FP64 path, the CUDA-core float32 reaction GEMM (tensor cores off) and, through
several charge vectors, against one-at-a-time evaluations."""
import numpy as np
import pytest

import oracle
from paper_1908_10863_gb300 import LayeredFMM, workloads
from paper_1908_10863_gb300.lfmm import OPT_TENSOR_CORES

pytestmark = pytest.mark.gpu

# float32 form against FP64 at the same order: the CUDA-core float32 form
# measures ~1e-6 at p = 10; a wrong operator entry (sign, phase, index) shows
# as 1e-3 or more because the reaction terms are O(1) of the potential
PHI_BOUND = 5e-6
FIELD_BOUND = 5e-6


def _eval(w, p, precision, tc, q=None):
    with LayeredFMM(w.d, w.eps, p, precision=precision) as f:
        f.set_option(OPT_TENSOR_CORES, tc)
        f.build(w.xyz, w.layer)
        phi, E = f.evaluate(w.q if q is None else q)
        st = f.stats()
    return phi, E, st


@pytest.mark.parametrize("p", [4, 7, 10])
@pytest.mark.parametrize("eps", [None, (1.0, 80.0, 2.0)], ids=["config", "high_contrast"])
def test_reaction_tensor_cores_against_fp64(p, eps):
    # p = 4, 7, 10: 2, 4 and 8 K chunks of 16 input coefficients
    w = workloads.config2(30000) if eps is None else workloads.config2(30000, eps=eps)
    phi_t, E_t, st = _eval(w, p, 1, 2)
    phi_c, E_c, _ = _eval(w, p, 1, 0)
    phi_64, E_64, _ = _eval(w, p, 0, 0)
    assert st["m2l_reaction"] > 0 and st["reaction_keys"] > 0
    assert st["timeouts"] == 0
    e_t, e_c = oracle.err2(phi_64, phi_t), oracle.err2(phi_64, phi_c)
    f_t, f_c = oracle.err2(E_64, E_t), oracle.err2(E_64, E_c)
    print("p=%d eps=%s: Err2 vs FP64: tensor cores phi %.2e field %.2e; CUDA cores phi %.2e field %.2e"
          % (p, eps, e_t, f_t, e_c, f_c))
    assert e_t < PHI_BOUND and f_t < FIELD_BOUND


def test_reaction_tensor_cores_several_vectors():
    # the operator stays in shared memory while the vectors take turns
    w = workloads.config2(20000)
    Q = np.random.default_rng(11).uniform(-1.0, 1.0, (3, w.n))
    with LayeredFMM(w.d, w.eps, 10, precision=1) as f:
        f.build(w.xyz, w.layer)
        phi_b, E_b = f.evaluate(Q)
        singles = [f.evaluate(q) for q in Q]
        assert f.stats()["m2l_reaction"] > 0 and f.stats()["timeouts"] == 0
    for r, (phi, E) in enumerate(singles):
        assert oracle.err2(phi, phi_b[r]) < 1e-6
        assert oracle.err2(E, E_b[r]) < 1e-6


@pytest.mark.parametrize("aligned", [True, False])
def test_reaction_tensor_cores_four_layers_against_fp64(aligned):
    # 36 reaction components; keys on grids aligned with the interfaces or not
    d = workloads.D_FOUR if aligned else workloads.D_FOUR_UNALIGNED
    w = workloads.four_layers(6000, d=d)
    phi_t, E_t, st = _eval(w, 10, 1, 2)
    phi_64, E_64, _ = _eval(w, 10, 0, 0)
    assert st["m2l_reaction"] > 0 and st["reaction_keys"] > 0 and st["timeouts"] == 0
    e, ef = oracle.err2(phi_64, phi_t), oracle.err2(E_64, E_t)
    print("four layers 6000 aligned=%s: float32 tensor-core form vs FP64 Err2 phi %.2e field %.2e" % (aligned, e, ef))
    assert e < PHI_BOUND and ef < FIELD_BOUND
