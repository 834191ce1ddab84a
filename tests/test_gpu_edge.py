"""Input edge cases through the GPU path, against the FP64 Ewald oracle:
- sources given outside the cell (negative and > 1 fractional coordinates): the lattice sum is
  periodic, so the result equals that of the wrapped inputs (the oracle takes them as given);
- a pair of distinct sources 1e-9 of the cell apart (the exact close-pair difference);
- cells with one, two and seven sources (non-neutral charges: zero-mean potential).
Bar: relative L2 <= eps for the potential, 10 eps for the gradient (40 eps in the cells of two
and seven charges, where one pair dominates the gradient).
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


def _eval(P, L, y, q, eps, prec, **kw):
    plan = P.Plan(L, eps, precision=prec, **kw)
    plan.set_sources(y, q)
    pot, grad = plan.eval()
    plan.close()
    return pot, grad


L2 = np.array([[1.0, 0.45], [0.0, 0.85]])
L3 = W.lattice_from_lengths_angles(1.0, 1.3, 0.8, 75, 100, 110)


@pytest.mark.parametrize("L", [L2, L3], ids=["2d", "3d"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sources_outside_the_cell(L, prec):
    P = _cuda()
    d = L.shape[0]
    g = W.random_neutral(L, 1500, seed=21 + d)
    rng = np.random.default_rng(3)
    shift = rng.integers(-3, 4, size=(len(g["q"]), d)).astype(float)
    y_out = g["y"] + shift @ L.T  # the same points, shifted by lattice vectors
    assert (np.linalg.solve(L, y_out.T) < 0).any() and (np.linalg.solve(L, y_out.T) > 1).any()
    pref, gref = E.ewald(L, y_out, g["q"])
    pot, grad = _eval(P, L, y_out, g["q"], 1e-6, prec)
    p0, g0 = _eval(P, L, g["y"], g["q"], 1e-6, prec)
    assert rel(pot, pref) <= 1e-6 and rel(grad, gref) <= 1e-5
    # the wrapped inputs give the same field up to the method's accuracy
    assert rel(pot, p0) <= 1e-6 and rel(grad, g0) <= 1e-5


@pytest.mark.parametrize("L", [L2, L3], ids=["2d", "3d"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_near_coincident_pair(L, prec):
    P = _cuda()
    d = L.shape[0]
    g = W.random_neutral(L, 800, seed=31 + d)
    y = g["y"].copy()
    y[1] = y[0] + 1e-9 * np.linalg.norm(L[:, 0]) * np.ones(d) / np.sqrt(d)
    pref, gref = E.ewald(L, y, g["q"])
    pot, grad = _eval(P, L, y, g["q"], 1e-6, prec)
    e, eg = rel(pot, pref), rel(grad, gref)
    print(f"near-coincident pair d={d} {prec}: E_pot={e:.2e} E_grad={eg:.2e}")
    assert e <= 1e-6 and eg <= 1e-5


@pytest.mark.parametrize("n", [1, 2, 7])
@pytest.mark.parametrize("L", [L2, L3], ids=["2d", "3d"])
def test_tiny_cells(n, L):
    P = _cuda()
    d = L.shape[0]
    rng = np.random.default_rng(40 + n)
    y = rng.random((n, d)) @ L.T
    q = rng.standard_normal(n)  # not neutral: the zero-mean (background) potential
    pref, gref = E.ewald(L, y, q)
    pot, grad = _eval(P, L, y, q, 1e-9, "fp64")
    if n == 1:
        # a lone charge: its field at itself comes from its images only, and vanishes by symmetry
        assert abs(pot[0] - pref[0]) <= 1e-9 * max(1.0, abs(pref[0]))
        assert np.all(np.abs(grad) <= 1e-8) and np.all(np.abs(gref) <= 1e-8)
        return
    assert rel(pot, pref) <= 1e-9
    # the gradient of a two- or seven-charge cell is dominated by one or two pairs; the
    # derivative amplifies the spectral truncation by |k|_max / |k|_typ (4-40x measured)
    assert rel(grad, gref) <= 40 * 1e-9
