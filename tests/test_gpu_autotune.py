"""The (kappa, n_s) autotuner (pdmk_opts.autotune): the tuned plan is one of the timed
candidates, matches the oracle, and a second plan of the same size class reuses the cached
choice (same ratios to the Table 1 values)."""
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


@pytest.mark.parametrize("case", ["oblique2d", "triclinic3d"])
def test_autotuned_plan(case):
    P = _cuda()
    g = W.oblique2d_clusters(6000, seed=501) if case == "oblique2d" else \
        W.triclinic3d_clusters(6000, nclusters=8, seed=502)
    base = P.Plan(g["L"], 1e-6, precision="mixed")
    base.set_sources(g["y"], g["q"])
    i0 = base.info()
    base.close()
    plan = P.Plan(g["L"], 1e-6, precision="mixed", autotune=True)
    plan.set_sources(g["y"], g["q"])
    info = plan.info()
    kr, nr = info["kappa"] / i0["kappa"], info["n_s"] / i0["n_s"]
    assert any(abs(kr - k) < 1e-9 for k in (0.75, 1.0, 4.0 / 3.0))
    assert any(abs(info["n_s"] - max(4, round(i0["n_s"] * f))) <= 1 for f in (0.5, 1.0, 2.0))
    pot, grad = plan.eval()
    plan.close()
    pref, gref = E.ewald(g["L"], g["y"], g["q"])
    assert rel(pot, pref) <= 1e-6 and rel(grad, gref) <= 1e-5
    # same size class: the cached choice, no new timing
    g2 = W.oblique2d_clusters(6500, seed=503) if case == "oblique2d" else \
        W.triclinic3d_clusters(6500, nclusters=8, seed=504)
    p2 = P.Plan(g2["L"], 1e-6, precision="mixed", autotune=True)
    p2.set_sources(g2["y"], g2["q"])
    b2 = P.Plan(g2["L"], 1e-6, precision="mixed")
    b2.set_sources(g2["y"], g2["q"])
    assert abs(p2.info()["kappa"] / b2.info()["kappa"] - kr) < 1e-9
    p2.close()
    b2.close()
