"""Per-call targets (pdmk_eval_targets) against the FP64 Ewald oracle, element by element.

The sources' tree is built once by pdmk_set_sources; every call evaluates the sources' field
at new targets against it: inside the cell, outside it (negative and > 1 fractional
coordinates, shifted by lattice vectors), exactly on the cell's faces, in empty regions of
clustered cells, and exactly at sources (whose self term is then excluded, as the oracle's
self_idx excludes it).  Bar: relative L2 over the targets <= eps for the potential, 10 eps
for the gradient, and no single target off by more than 10 eps of the largest |Phi|.
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
    return P, torch


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


CELLS = {
    "oblique2d": (lambda: W.oblique2d_clusters(3000, seed=901), {}),
    "oblique2d_deep": (lambda: W.oblique2d_clusters(20000, seed=902), {}),
    "triclinic3d": (lambda: W.triclinic3d_clusters(3000, nclusters=8, seed=903), {}),
    "triclinic3d_deep": (lambda: W.triclinic3d_clusters(12000, nclusters=8, seed=904), {"n_s": 60}),
    "cube": (lambda: W.cube_uniform(2000, seed=905), {"n_s": 20}),
}


def _targets(g, rng):
    """(x, self_idx): random interior points, points outside the cell, points on the cell's
    faces and exactly at sources."""
    L, y = g["L"], g["y"]
    d = L.shape[0]
    n = len(y)
    xs, sidx = [], []
    u = rng.random((60, d))
    xs.append(u @ L.T)                                           # inside
    sidx += [-1] * 60
    shift = rng.integers(-3, 4, size=(40, d)).astype(float)
    xs.append((rng.random((40, d)) + shift) @ L.T)               # outside (negative, > 1)
    sidx += [-1] * 40
    uf = rng.random((20, d))
    uf[np.arange(20), rng.integers(0, d, 20)] = 0.0              # on a face of the cell
    xs.append(uf @ L.T)
    sidx += [-1] * 20
    k = rng.choice(n, 30, replace=False)
    xs.append(y[k])                                              # exactly at sources
    sidx += list(k)
    return np.concatenate(xs), np.asarray(sidx, dtype=np.int64)


@pytest.mark.parametrize("case", list(CELLS))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eval_targets_against_oracle(case, prec):
    P, _ = _cuda()
    make, opts = CELLS[case]
    g = make()
    eps = 1e-6
    rng = np.random.default_rng(77)
    x, sidx = _targets(g, rng)
    pref, gref = E.ewald(g["L"], g["y"], g["q"], x=x, self_idx=sidx)
    plan = P.Plan(g["L"], eps, precision=prec, **opts)
    plan.set_sources(g["y"], g["q"])
    pot, grad = plan.eval_targets(x)
    plan.close()
    ep, eg = rel(pot, pref), rel(grad, gref)
    worst = float(np.max(np.abs(pot - pref)) / np.max(np.abs(pref)))
    print(f"{case} {prec}: E_pot={ep:.2e} E_grad={eg:.2e} worst={worst:.2e}")
    assert np.all(np.isfinite(pot)) and np.all(np.isfinite(grad))
    assert ep <= eps
    assert eg <= 10 * eps
    assert worst <= 10 * eps


def test_eval_targets_per_call_and_charges():
    """New targets on every call against one tree; new charges are seen; device buffers."""
    P, torch = _cuda()
    g = W.triclinic3d_clusters(4000, nclusters=8, seed=906)
    plan = P.Plan(g["L"], 1e-6, precision="mixed")
    plan.set_sources(g["y"], g["q"])
    rng = np.random.default_rng(5)
    for call in range(3):
        x = (rng.random((150, 3)) + rng.integers(-1, 2, size=(150, 3))) @ g["L"].T
        q = g["q"] if call < 2 else g["q"] * rng.uniform(0.5, 1.5, len(g["q"]))
        if call == 2:
            plan.set_charges(q)
        pref, gref = E.ewald(g["L"], g["y"], q, x=x)
        xt = torch.tensor(x, device="cuda")
        pot, grad = plan.eval_targets(xt)
        torch.cuda.synchronize()
        assert rel(pot.cpu().numpy(), pref) <= 1e-6
        assert rel(grad.cpu().numpy(), gref) <= 1e-5
    plan.close()


def test_eval_targets_at_the_sources_match_eval():
    """At the sources themselves the per-call path reproduces pdmk_eval to the method's
    accuracy (the plane-wave part may come from a different box of the same tree path)."""
    P, _ = _cuda()
    g = W.oblique2d_clusters(5000, seed=907)
    plan = P.Plan(g["L"], 1e-6, precision="fp64")
    plan.set_sources(g["y"], g["q"])
    p0, g0 = plan.eval()
    p1, g1 = plan.eval_targets(g["y"])
    plan.close()
    assert rel(p1, p0) <= 1e-7
    assert rel(g1, g0) <= 1e-6


def test_eval_targets_rejects_bad_arguments():
    P, _ = _cuda()
    g = W.cube_uniform(500, seed=908)
    plan = P.Plan(g["L"], 1e-3)
    with pytest.raises(P.PdmkError) as ei:
        plan.eval_targets(np.zeros((3, 3)))
    assert ei.value.code == -9  # NOT_READY before set_sources
    plan.set_sources(g["y"], g["q"])
    with pytest.raises(P.PdmkError) as ei:
        plan.eval_targets(np.array([[0.1, np.nan, 0.2]]))
    assert ei.value.code == -5  # NONFINITE
    pot, grad = plan.eval_targets(np.zeros((0, 3)))
    assert pot.shape == (0,) and grad.shape == (0, 3)
    plan.close()
