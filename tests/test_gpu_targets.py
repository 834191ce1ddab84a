"""Evaluation at separate targets (pdmk_set_sources_targets): the field of the sources at
arbitrary points against the FP64 oracle, periodicity in the targets, and the adjoint with
separate targets against the oracle's fields."""
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


def _case(d, seed):
    if d == 2:
        g = W.oblique2d_clusters(3000, seed=seed)
    else:
        g = W.triclinic3d_clusters(2500, seed=seed, nclusters=4)
    rng = np.random.default_rng(seed + 1)
    x = (g["L"] @ rng.random((d, 700))).T  # targets spread over the cell
    return g, x


@pytest.mark.parametrize("d,precision,eps", [(2, "fp64", 1e-9), (3, "fp64", 1e-9), (2, "mixed", 1e-6),
                                             (3, "mixed", 1e-6)])
def test_targets_against_oracle(d, precision, eps):
    P = _cuda()
    g, x = _case(d, 50 + d)
    plan = P.Plan(g["L"], eps, precision=precision)
    plan.set_sources(g["y"], g["q"], x=x)
    pot, grad = plan.eval()
    assert pot.shape == (len(x),) and grad.shape == (len(x), d)
    assert plan.info()["n_targets"] == len(x)
    pref, gref = E.ewald(g["L"], g["y"], g["q"], x=x)
    assert rel(pot, pref) <= eps
    assert rel(grad, gref) <= 10 * eps
    plan.close()


def test_targets_are_periodic():
    """Targets moved by lattice vectors (outside the cell) give the same field."""
    P = _cuda()
    g, x = _case(2, 60)
    shift = (g["L"] @ np.array([[2.0], [-1.0]])).T
    a = P.Plan(g["L"], 1e-9, precision="fp64")
    a.set_sources(g["y"], g["q"], x=x)
    p1, g1 = a.eval()
    a.set_sources(g["y"], g["q"], x=x + shift)
    p2, g2 = a.eval()
    assert rel(p2, p1) <= 1e-12 and rel(g2, g1) <= 1e-11
    a.close()


@pytest.mark.parametrize("d", [2, 3])
def test_adjoint_with_targets_against_oracle(d):
    """For a loss on the targets' potential with upstream g: dq = the sources' potential of
    charges g at the targets, dy = q grad Phi[g at x](y), dx = g grad Phi[q](x)."""
    P = _cuda()
    g, x = _case(d, 70 + d)
    up = np.random.default_rng(9).standard_normal(len(x))
    plan = P.Plan(g["L"], 1e-9, precision="fp64")
    plan.set_sources(g["y"], g["q"], x=x)
    p0, _ = plan.eval()
    gq, gy, gx = plan.eval_adjoint(up)
    pg_at_y, fg_at_y = E.ewald(g["L"], x, up, x=g["y"])
    _, fq_at_x = E.ewald(g["L"], g["y"], g["q"], x=x)
    assert rel(gq, pg_at_y) <= 1e-8
    assert rel(gy, g["q"][:, None] * fg_at_y) <= 1e-7
    assert rel(gx, up[:, None] * fq_at_x) <= 1e-7
    p1, _ = plan.eval()
    assert np.array_equal(p0, p1)
    plan.close()
