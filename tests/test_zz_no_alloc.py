"""The allocation-free evaluation (pdmk_eval_noalloc) against pdmk_eval.

Callers that cannot allocate device memory during a step (an engine owning the whole
device heap, a caching allocator that forbids cudaMalloc mid-step, a real-time loop) use
pdmk_eval_noalloc: it evaluates an already-built plan into caller buffers with the spreading
scratch taken from the library's static 16 MiB device array.  This file is collected last
so that a failure here never hides the other tests' results.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_28608_b300 as P
    return torch, P


CASES = [
    # 2D oblique cell: the whole-grid spreading paths (one grid copy per CTA in the scratch)
    ("mixed", "oblique2d", 1e-6), ("fp64", "oblique2d", 1e-6),
    # 3D triclinic cells: the per-subproblem tiles of the generic spreading kernel
    ("mixed", "triclinic3d", 1e-6), ("fp64", "triclinic3d", 1e-6), ("fp64", "triclinic3d", 1e-3),
]


def _workload(kind):
    if kind == "oblique2d":
        return W.oblique2d_clusters(20000, seed=321)
    return W.triclinic3d_clusters(4000, seed=322)


@pytest.mark.parametrize("prec,kind,eps", CASES)
def test_noalloc_matches_eval_twice(prec, kind, eps):
    torch, P = _setup()
    g = _workload(kind)
    n, d = g["y"].shape
    plan = P.Plan(g["L"], eps, precision=prec)
    plan.set_sources(g["y"], g["q"])
    pot_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    grad_ref = torch.empty((n, d), dtype=torch.float64, device="cuda")
    plan.eval_device(pot_ref, grad_ref)
    torch.cuda.synchronize()
    pr, gr = pot_ref.cpu().numpy(), grad_ref.cpu().numpy()
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        pot = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        grad = torch.full((n, d), float("nan"), dtype=torch.float64, device="cuda")
        plan.eval_noalloc(pot, grad)
        torch.cuda.synchronize()
        p, gg = pot.cpu().numpy(), grad.cpu().numpy()
        assert np.all(np.isfinite(p)) and np.all(np.isfinite(gg))
        assert np.linalg.norm(p - pr) <= 1e-12 * np.linalg.norm(pr)
        assert np.linalg.norm(gg - gr) <= 1e-12 * np.linalg.norm(gr)
    plan.close()


def test_noalloc_after_profiled_eval_keeps_stage_times():
    """On a profiling plan, pdmk_eval records per-stage times; a following allocation-free
    call runs unprofiled, and pdmk_stage_times must then report a consistent (possibly empty)
    list rather than index names that are no longer there."""
    torch, P = _setup()
    g = W.oblique2d_clusters(5000, seed=323)
    n = len(g["q"])
    plan = P.Plan(g["L"], 1e-6, precision="mixed", profile=True)
    plan.set_sources(g["y"], g["q"])
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    plan.eval_device(pot, grad)
    torch.cuda.synchronize()
    st = plan.stage_times()
    assert "nearfield" in st and all(v >= 0 for v in st.values())
    plan.eval_noalloc(pot, grad)
    torch.cuda.synchronize()
    st2 = plan.stage_times()
    assert all(isinstance(k, str) and v >= 0 for k, v in st2.items())
    plan.eval_device(pot, grad)
    torch.cuda.synchronize()
    assert set(plan.stage_times()) == set(st)
    plan.close()


def test_noalloc_rejects_oversized_scratch():
    torch, P = _setup()
    g = W.random_neutral(np.eye(3), 400000, seed=3)
    plan = P.Plan(g["L"], 1e-9, precision="fp64", max_depth=0, kappa=3.0)
    plan.set_sources(g["y"], g["q"])
    pot = torch.empty(len(g["q"]), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PdmkError) as ei:
        plan.eval_noalloc(pot, None)
    assert ei.value.code == -11  # PDMK_ERR_TOO_LARGE
    plan.close()
