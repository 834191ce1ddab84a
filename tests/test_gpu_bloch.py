"""Quasi-periodic (Bloch) lattice sums (pdmk_eval_bloch) against the oracle's Bloch Ewald sum
(oracle.ewald.ewald_bloch, pinned in tests/test_oracle.py), element by element: 2D oblique and
3D triclinic cells, uniform and clustered sources, non-neutral charges, both precisions.
Bar: relative L2 <= eps for the potential, 10 eps for the gradient; plus the Bloch property
(a source set shifted by a lattice vector L n multiplies the field by e^{-i beta.L n})."""
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


L2 = np.array([[1.0, 0.45], [0.0, 0.85]])
L3 = W.lattice_from_lengths_angles(1.0, 1.2, 0.9, 80, 100, 105)


def _cell(kind):
    if kind == "2d_uniform":
        return W.random_neutral(L2, 600, seed=71, neutral=False)
    if kind == "2d_clusters":
        g = W.oblique2d_clusters(1500, seed=72)
        g["q"] = g["q"] + 0.3  # non-neutral
        return g
    if kind == "3d_uniform":
        return W.random_neutral(L3, 600, seed=73, neutral=False)
    g = W.triclinic3d_clusters(1500, nclusters=4, seed=74)
    return g


def _beta(L, rng):
    # a generic wave vector: a fraction of the reciprocal basis, away from the lattice
    d = L.shape[0]
    Kr = 2 * np.pi * np.linalg.inv(L).T  # reciprocal basis (columns)
    return Kr @ rng.uniform(0.1, 0.9, d)


@pytest.mark.parametrize("kind", ["2d_uniform", "2d_clusters", "3d_uniform", "3d_clusters"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bloch_against_oracle(kind, prec):
    P = _cuda()
    g = _cell(kind)
    L = g["L"]
    rng = np.random.default_rng(9)
    beta = _beta(L, rng)
    pref, gref = E.ewald_bloch(L, g["y"], g["q"], beta)
    plan = P.Plan(L, 1e-6, precision=prec)
    plan.set_sources(g["y"], g["q"])
    pot, grad = plan.eval_bloch(beta)
    # the periodic evaluation afterwards still sees the plan's own charges
    p_per, _ = plan.eval()
    pper_ref, _ = E.ewald(L, g["y"], g["q"])
    plan.close()
    ep, eg = rel(pot, pref), rel(grad, gref)
    print(f"bloch {kind} {prec}: E_pot={ep:.2e} E_grad={eg:.2e}")
    assert np.all(np.isfinite(pot)) and np.all(np.isfinite(grad))
    assert ep <= 1e-6
    assert eg <= 1e-5
    assert rel(p_per, pper_ref) <= 1e-6


def test_bloch_shifted_sources():
    """Sources given at y + L n (n integer per source): the field at the given positions is
    e^{i beta.L n} times the field at y (Bloch property of the sum, per point)."""
    P = _cuda()
    g = W.random_neutral(L3, 500, seed=75, neutral=False)
    rng = np.random.default_rng(10)
    beta = _beta(L3, rng)
    n = rng.integers(-2, 3, size=(len(g["q"]), 3)).astype(float)
    ys = g["y"] + n @ L3.T
    plan = P.Plan(L3, 1e-9, precision="fp64")
    plan.set_sources(g["y"], g["q"])
    p0, _ = plan.eval_bloch(beta)
    plan.set_sources(ys, g["q"])
    p1, _ = plan.eval_bloch(beta)
    plan.close()
    # moving source j by L n_j multiplies its contribution by e^{-i beta.L n_j}; at the moved
    # target the field is e^{i beta.L n_t} times the field there: compare against the oracle
    pref, _ = E.ewald_bloch(L3, ys, g["q"], beta)
    assert rel(p1, pref) <= 1e-8
    assert rel(p0, E.ewald_bloch(L3, g["y"], g["q"], beta)[0]) <= 1e-8


def test_bloch_rejects_reciprocal_vector():
    P = _cuda()
    g = W.random_neutral(L2, 100, seed=76)
    plan = P.Plan(L2, 1e-6)
    plan.set_sources(g["y"], g["q"])
    Kr = 2 * np.pi * np.linalg.inv(L2).T
    with pytest.raises(P.PdmkError) as ei:
        plan.eval_bloch(Kr @ np.array([1.0, -2.0]))
    assert ei.value.code == -1
    plan.close()
