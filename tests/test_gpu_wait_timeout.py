"""Bounded device waits: the single-launch downward pass (2D, compile-time orders) waits on
flags set by other blocks of the same launch.  The test hook wait_test=1 points the first
dependent wait at a flag that nothing sets; the wait must give up after about a second, the
evaluation must report PDMK_ERR_TIMEOUT, and the CUDA context must stay usable."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

PDMK_ERR_TIMEOUT = -8


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_28608_b300 as P
    return P, torch


def test_expired_wait_reports_timeout_and_context_survives():
    P, torch = _cuda()
    g = W.oblique2d_clusters(20000)
    ref = P.Plan(g["L"], 1e-6, precision="mixed")
    ref.set_sources(g["y"], g["q"])
    p_ref, g_ref = ref.eval()

    bad = P.Plan(g["L"], 1e-6, precision="mixed", wait_test=1)
    bad.set_sources(g["y"], g["q"])
    assert bad.info()["depth"] >= 3
    t0 = time.time()
    with pytest.raises(P.PdmkError) as ei:
        bad.eval()
    assert ei.value.code == PDMK_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    # device evaluation: the timeout surfaces at the next call of the plan
    n = len(g["q"])
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    bad.eval_device(pot, grad)
    torch.cuda.synchronize()
    with pytest.raises(P.PdmkError) as ei2:
        bad.eval_device(pot, grad)
    assert ei2.value.code == PDMK_ERR_TIMEOUT
    torch.cuda.synchronize()
    bad.close()

    # the context still works: a fresh evaluation matches the one before the timeouts
    p2, g2 = ref.eval()
    assert np.array_equal(p2, p_ref) and np.array_equal(g2, g_ref)
    ref.close()
