"""Repeated set-ups on one plan (the buffers of a set-up are handed to the next one).

A plan reuses the device buffers of its previous set-up when the sizes fit, so the arrays a
set-up finds hold the previous problem's data, not zeros.  Every result must depend on the
current sources only: the same sources after a different problem give the same potential and
gradient bit for bit, equal to a fresh plan's, and both match the FP64 Ewald oracle.  A 3D
device set-up also leaves the host tree on the device until a host path asks for it; the
per-call targets after such a set-up are checked here too.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ewald as E

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_28608_b300 as P
    return P


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


CASES = {
    "triclinic3d": (lambda: W.triclinic3d_clusters(12000, nclusters=8, seed=31),
                    lambda: W.triclinic3d_clusters(9000, nclusters=3, seed=32)),
    "oblique2d": (lambda: W.oblique2d_clusters(20000, seed=33), lambda: W.oblique2d_clusters(15000, seed=34)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_same_sources_same_result_after_other_problem(case, precision):
    P = _cuda()
    ga, gb = CASES[case][0](), CASES[case][1]()
    assert np.allclose(ga["L"], gb["L"])
    eps = 1e-6
    plan = P.Plan(ga["L"], eps, precision=precision, n_s=40)
    plan.set_sources(ga["y"], ga["q"])
    p1, g1 = plan.eval()
    plan.set_sources(gb["y"], gb["q"])  # a different problem in between (other sizes and data)
    plan.eval()
    plan.set_sources(ga["y"], ga["q"])
    p3, g3 = plan.eval()
    plan.set_sources(ga["y"], ga["q"])  # the same sizes again: every buffer reused
    p4, g4 = plan.eval()
    plan.close()
    fresh = P.Plan(ga["L"], eps, precision=precision, n_s=40)
    fresh.set_sources(ga["y"], ga["q"])
    p5, g5 = fresh.eval()
    fresh.close()
    for p, g in ((p3, g3), (p4, g4), (p5, g5)):
        assert np.array_equal(p, p1) and np.array_equal(g, g1)
    pref, gref = E.ewald(ga["L"], ga["y"], ga["q"])
    assert rel(p1, pref) <= eps
    assert rel(g1, gref) <= 2 * eps


def test_targets_after_device_setup_without_host_tree():
    """Per-call targets after a 3D device set-up (the host tree is read back on that call),
    then again after a second set-up of the same plan; the bars of the per-call target tests
    (eps for the potential, 10 eps for the gradient at arbitrary points)."""
    P = _cuda()
    g = W.triclinic3d_clusters(10000, nclusters=6, seed=35)
    rng = np.random.default_rng(36)
    x = rng.random((500, 3)) @ g["L"].T
    eps = 1e-6
    pref, gref = E.ewald(g["L"], g["y"], g["q"], x=x)
    plan = P.Plan(g["L"], eps, precision="fp64", n_s=40)
    for _ in range(2):
        plan.set_sources(g["y"], g["q"])
        pot, grad = plan.eval_targets(x)
        assert rel(pot, pref) <= eps
        assert rel(grad, gref) <= 10 * eps
    plan.close()
