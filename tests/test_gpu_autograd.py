"""Differentiation through the periodic potential (paper_2606_28608_b300.autograd).

Checks: dU/dq = Phi for U = q.Phi/2 (symmetry of the lattice-sum operator), dU/dy = q grad Phi
against the FP64 oracle, and a general loss against central finite differences."""
import numpy as np
import pytest

import workloads as W
from oracle import ewald as E

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_28608_b300.autograd import periodic_potential
    return torch, periodic_potential


@pytest.mark.parametrize("d", [2, 3])
def test_energy_gradients(d):
    torch, pp = _torch()
    g = W.oblique2d_clusters(1500, seed=17) if d == 2 else W.triclinic3d_clusters(1500, seed=18, nclusters=4)
    y = torch.tensor(g["y"], device="cuda", requires_grad=True)
    q = torch.tensor(g["q"], device="cuda", requires_grad=True)
    pot, grad = pp(g["L"], y, q, eps=1e-9, precision="fp64")
    U = 0.5 * (q * pot).sum()
    U.backward()
    pref, gref = E.ewald(g["L"], g["y"], g["q"])
    dq = q.grad.cpu().numpy()
    dy = y.grad.cpu().numpy()
    assert np.linalg.norm(dq - pref) <= 1e-8 * np.linalg.norm(pref)
    want = g["q"][:, None] * gref
    assert np.linalg.norm(dy - want) <= 1e-7 * np.linalg.norm(want)


def test_general_loss_finite_differences():
    torch, pp = _torch()
    g = W.random_neutral(np.array([[1.0, 0.3], [0.0, 0.8]]), 400, seed=4)
    rng = np.random.default_rng(1)
    wgt = torch.tensor(rng.standard_normal(400), device="cuda")
    y = torch.tensor(g["y"], device="cuda", requires_grad=True)
    q = torch.tensor(g["q"], device="cuda", requires_grad=True)
    pot, _ = pp(g["L"], y, q, eps=1e-10, precision="fp64")
    (wgt * pot).sum().backward()

    def loss(yy, qq):
        p, _ = pp(g["L"], torch.tensor(yy, device="cuda"), torch.tensor(qq, device="cuda"), eps=1e-10,
                  precision="fp64")
        return float((wgt * p).sum())

    h = 1e-4
    for k, a in ((3, 0), (177, 1)):
        yp = g["y"].copy(); yp[k, a] += h
        ym = g["y"].copy(); ym[k, a] -= h
        fd = (loss(yp, g["q"]) - loss(ym, g["q"])) / (2 * h)
        assert abs(fd - float(y.grad[k, a])) <= 1e-4 * max(1.0, abs(fd))
    for k in (5, 250):
        qp = g["q"].copy(); qp[k] += 1.0
        fd = loss(g["y"], qp) - loss(g["y"], g["q"])  # linear in q: exact difference
        assert abs(fd - float(q.grad[k])) <= 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("d,precision,tol", [(2, "fp64", 1e-8), (3, "fp64", 1e-8), (2, "mixed", 1e-5)])
def test_eval_adjoint_against_oracle(d, precision, tol):
    """pdmk_eval_adjoint with a random upstream g: dq = A g is the oracle's potential for
    charges g (not neutral), dy = g grad Phi[q] + q grad Phi[g] from the oracle's fields."""
    _torch()
    import paper_2606_28608_b300 as P
    g = W.oblique2d_clusters(1200, seed=31) if d == 2 else W.triclinic3d_clusters(1000, seed=32, nclusters=4)
    n = len(g["q"])
    up = np.random.default_rng(2).standard_normal(n)
    plan = P.Plan(g["L"], 1e-9 if precision == "fp64" else 1e-6, precision=precision)
    plan.set_sources(g["y"], g["q"])
    p0, g0 = plan.eval()
    gq, gy = plan.eval_adjoint(up)
    p_q, f_q = E.ewald(g["L"], g["y"], g["q"])
    p_g, f_g = E.ewald(g["L"], g["y"], up)
    assert np.linalg.norm(gq - p_g) <= tol * np.linalg.norm(p_g)
    want = up[:, None] * f_q + g["q"][:, None] * f_g
    assert np.linalg.norm(gy - want) <= 10 * tol * np.linalg.norm(want)
    # the plan's charges are the caller's again
    p1, g1 = plan.eval()
    assert np.array_equal(p0, p1) and np.array_equal(g0, g1)
    plan.close()


def test_eval_adjoint_device_matches_host_and_rejects_field_gradients():
    torch, _ = _torch()
    import paper_2606_28608_b300 as P
    g = W.oblique2d_clusters(3000, seed=33)
    n = len(g["q"])
    up = np.random.default_rng(3).standard_normal(n)
    plan = P.Plan(g["L"], 1e-6, precision="mixed")
    plan.set_sources(g["y"], g["q"])
    hq, hy = plan.eval_adjoint(up)
    dq, dy = plan.eval_adjoint(torch.tensor(up, device="cuda"))
    assert np.array_equal(hq, dq.cpu().numpy()) and np.array_equal(hy, dy.cpu().numpy())
    only_q, none_y = plan.eval_adjoint(up, want_y=False)
    assert none_y is None and np.array_equal(only_q, hq)
    # an upstream gradient on the returned field is refused (BAD_ARG), nothing is written
    gg = np.zeros((n, 2))
    out = np.zeros(n)
    rc = P.lib().pdmk_eval_adjoint(plan._h, up.ctypes.data, gg.ctypes.data, out.ctypes.data, None, None,
                                   P.PDMK_HOST)
    assert rc == -1 and not out.any()
    plan.close()


def test_plan_reuse_across_steps():
    """A molecular-dynamics-like loop (PeriodicPotential module): positions move every step,
    the plans come from the pool (no new plan once one is free), and every step's energy
    gradient matches a fresh computation with its own plan."""
    torch, pp = _torch()
    from paper_2606_28608_b300.autograd import POOL, PeriodicPotential
    import paper_2606_28608_b300 as P
    g = W.triclinic3d_clusters(3000, seed=19, nclusters=4)
    mod = PeriodicPotential(g["L"], eps=1e-6, precision="mixed")
    rng = np.random.default_rng(2)
    y0 = g["y"].copy()
    for step in range(3):
        y = torch.tensor(y0 + 1e-3 * rng.standard_normal(y0.shape), device="cuda", requires_grad=True)
        q = torch.tensor(g["q"], device="cuda")
        pot, _ = mod(y, q)
        (0.5 * (q * pot).sum()).backward()
        free_after = POOL.size()
        assert free_after >= 1  # the plan went back to the pool after backward
        plan = P.Plan(g["L"], 1e-6, precision="mixed")
        plan.set_sources(y.detach(), q)
        p_ref, g_ref = plan.eval()
        plan.close()
        dy = y.grad.cpu().numpy()
        want = g["q"][:, None] * g_ref
        assert np.linalg.norm(dy - want) <= 1e-6 * np.linalg.norm(want)
    # without a graph the plan returns to the pool at once
    with torch.no_grad():
        before = POOL.size()
        mod(torch.tensor(y0, device="cuda"), torch.tensor(g["q"], device="cuda"))
        assert POOL.size() == before
