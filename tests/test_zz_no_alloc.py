"""The allocation-free reaction-kernel entry point.

It serves callers that may not allocate device memory during a call (loops
that forbid allocator calls after start-up, hosts whose device memory is
budgeted by another runtime).  It must return what the allocating entry
point returns.  Two calls are made in a row, the second one smaller than the
first, so that reuse of the shared device array is exercised; free device
memory must not change across a call of the largest size it takes.
"""
import numpy as np
import pytest

from paper_1908_10863_gb300 import LayeredFMM, LfmmError
from paper_1908_10863_gb300.lfmm import NOALLOC_MAX_POINTS

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    rng = np.random.default_rng(12)
    cases = [((1, 1, 1, 1), 5000), ((0, 2, 1, 2), 777)]
    inputs = [(comp, rng.uniform(0.0, 0.6, n), rng.uniform(0.05, 2.0, n)) for comp, n in cases]
    with LayeredFMM([0.0, -1.2], [1.0, 5.0, 10.0], 6) as f:
        got = [f.reaction_kernel_noalloc(*comp, rho, h) for comp, rho, h in inputs]
        ref = [f.reaction_kernel(*comp, rho, h) for comp, rho, h in inputs]
    for g, r in zip(got, ref):
        assert g.shape == r.shape
        # same tolerance as the near-kernel parity test (relative to I_00)
        assert np.max(np.abs(g - r) / np.abs(r[:, :1])) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_array():
    n = NOALLOC_MAX_POINTS + 1
    with LayeredFMM([0.0, -1.2], [1.0, 5.0, 10.0], 4) as f:
        with pytest.raises(LfmmError) as ei:
            f.reaction_kernel_noalloc(1, 1, 1, 1, np.zeros(n), np.ones(n))
        assert "LFMM_NOALLOC_MAX_POINTS" in str(ei.value)
        out = f.reaction_kernel_noalloc(1, 1, 1, 1, [0.1], [0.5])  # context still usable
        assert np.all(np.isfinite(out))


def test_noalloc_leaves_free_device_memory_unchanged():
    torch = pytest.importorskip("torch")
    n = NOALLOC_MAX_POINTS
    rng = np.random.default_rng(13)
    rho, h = rng.uniform(0.0, 0.6, n), rng.uniform(0.05, 2.0, n)
    with LayeredFMM([0.0, -1.2], [1.0, 5.0, 10.0], 4) as f:
        # the first call may load the module that holds the static array
        first = f.reaction_kernel_noalloc(1, 1, 1, 1, rho, h)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        second = f.reaction_kernel_noalloc(1, 1, 1, 1, rho, h)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(first, second)
