"""Parity at full size for the synthetic workloads:
- the 3D triclinic cell (edge ratio ~17) with 4,000,000 clustered sources, at eps 1e-3 and
  1e-6 in both precisions and 1e-9 in FP64;
- the 2D oblique cell with 200,000 clustered sources at eps 1e-3 and 1e-6, both precisions;
- 333,000 three-site water-like molecules (999,000 charges), forward field, the adjoint
  (dU/dq = Phi and dU/dy = q grad Phi for U = q.Phi / 2) and central differences of the
  potential on 64 sites;
- 256 independent triclinic cells of 1e3..2e5 sources each, in one batch (64 sampled
  targets per cell, every cell held to eps).
All are checked on a seeded sample of targets whose FP64 Ewald values are stored under
tests/golden/ (written from the oracle alone by tests/golden/make_fullsize.py). Each stored
file also holds the sampled inputs, compared first against a fresh generation.
Error measure: relative L2 over the sample, potential <= eps, gradient <= 10 eps."""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_28608_b300 as P
    return P, torch


def _golden(name):
    with open(os.path.join(GOLDEN, f"fullsize_{name}.json")) as f:
        return json.load(f)


def _check_inputs(g, cell):
    """The stored sample belongs to these inputs (positions to rounding, charges exactly)."""
    idx = np.asarray(cell["idx"])
    assert len(g["q"]) == cell["n"]
    assert np.allclose(np.asarray(cell["L"]), g["L"], rtol=0, atol=1e-14)
    assert np.allclose(g["y"][idx], np.asarray(cell["y"]), rtol=0, atol=1e-12 * np.abs(g["L"]).max())
    assert np.array_equal(g["q"][idx], np.asarray(cell["q"]))
    return idx, np.asarray(cell["pot"]), np.asarray(cell["grad"])


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def tri4m():
    ref = _golden("triclinic3d_4m")
    g = W.triclinic3d_clusters(4_000_000)
    idx, pref, gref = _check_inputs(g, ref["cells"][0])
    return g, idx, pref, gref


@pytest.mark.parametrize("prec,eps", [("mixed", 1e-3), ("mixed", 1e-6), ("fp64", 1e-3), ("fp64", 1e-6),
                                      ("fp64", 1e-9)])
def test_triclinic3d_4m(tri4m, prec, eps):
    P, torch = _cuda()
    g, idx, pref, gref = tri4m
    n = len(g["q"])
    plan = P.Plan(g["L"], eps, precision=prec)
    plan.set_sources(g["y"], g["q"])
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    plan.eval_device(pot, grad)
    plan.eval_device(pot, grad)  # captured graph
    torch.cuda.synchronize()
    p = pot.cpu().numpy()
    gg = grad.cpu().numpy()
    ep, eg = _rel(p[idx], pref), _rel(gg[idx], gref)
    info = plan.info()
    print(f"triclinic3d 4M {prec} eps={eps:g}: E_pot={ep:.2e} E_grad={eg:.2e} depth={info['depth']} "
          f"images={info['n_images']} near_pairs={info['near_pairs']}")
    assert np.all(np.isfinite(p)) and np.all(np.isfinite(gg))
    assert ep <= eps
    assert eg <= 10 * eps
    plan.close()


@pytest.fixture(scope="module")
def obl200k():
    ref = _golden("oblique2d_200k")
    g = W.oblique2d_clusters(200_000)
    idx, pref, gref = _check_inputs(g, ref["cells"][0])
    return g, idx, pref, gref


@pytest.mark.parametrize("prec,eps", [("mixed", 1e-3), ("mixed", 1e-6), ("fp64", 1e-3), ("fp64", 1e-6)])
def test_oblique2d_200k(obl200k, prec, eps):
    P, torch = _cuda()
    g, idx, pref, gref = obl200k
    n = len(g["q"])
    plan = P.Plan(g["L"], eps, precision=prec)
    plan.set_sources(g["y"], g["q"])
    pot = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    plan.eval_device(pot, grad)
    plan.eval_device(pot, grad)  # captured graph
    torch.cuda.synchronize()
    p, gg = pot.cpu().numpy(), grad.cpu().numpy()
    ep, eg = _rel(p[idx], pref), _rel(gg[idx], gref)
    print(f"oblique2d 200k {prec} eps={eps:g}: E_pot={ep:.2e} E_grad={eg:.2e}")
    assert np.all(np.isfinite(p)) and np.all(np.isfinite(gg))
    assert ep <= eps
    assert eg <= 10 * eps
    plan.close()


@pytest.fixture(scope="module")
def water():
    ref = _golden("water_333k")
    g = W.water_box(333_000)
    idx, pref, gref = _check_inputs(g, ref["cells"][0])
    return g, idx, pref, gref


def test_water_fullsize_forward(water):
    P, torch = _cuda()
    g, idx, pref, gref = water
    plan = P.Plan(g["L"], 1e-6, precision="mixed")
    plan.set_sources(g["y"], g["q"])
    p, gg = plan.eval()
    ep, eg = _rel(p[idx], pref), _rel(gg[idx], gref)
    print(f"water 333k mixed: E_pot={ep:.2e} E_grad={eg:.2e}")
    assert ep <= 1e-6
    assert eg <= 1e-5
    plan.close()


def test_water_fullsize_adjoint(water):
    _, torch = _cuda()
    from paper_2606_28608_b300.autograd import periodic_potential
    g, idx, pref, gref = water
    y = torch.tensor(g["y"], device="cuda", requires_grad=True)
    q = torch.tensor(g["q"], device="cuda", requires_grad=True)
    pot, _ = periodic_potential(g["L"], y, q, eps=1e-6, precision="mixed")
    U = 0.5 * (q * pot).sum()
    U.backward()
    dq = q.grad.cpu().numpy()
    dy = y.grad.cpu().numpy()
    eq = _rel(dq[idx], pref)
    ey = _rel(dy[idx], g["q"][idx, None] * gref)
    print(f"water 333k adjoint: E_dq={eq:.2e} E_dy={ey:.2e}")
    assert eq <= 1e-6
    assert ey <= 1e-5


def test_water_fullsize_finite_differences(water):
    """Forces by central differences on 64 sites of the water box: the mixed plan's gradient
    at a site against (Phi(y_i + h e) - Phi(y_i - h e)) / 2h from an FP64 plan at eps 1e-9,
    both points taken as per-call targets of the same tree (pdmk_eval_targets).  The site's
    own singular term q_i G(+-h e) is even and cancels in the difference; h = 1e-5 r_c keeps
    the truncation (h^2 times the third derivative) and the FP64 rounding (1e-9 |Phi| / h)
    far below the bar."""
    P, _ = _cuda()
    g, _, _, _ = water
    rng = np.random.default_rng(64)
    sites = np.sort(rng.choice(len(g["q"]), 64, replace=False))
    plan = P.Plan(g["L"], 1e-6, precision="mixed")
    plan.set_sources(g["y"], g["q"])
    _, gm = plan.eval()
    rc = plan.info()["rc"]
    plan.close()
    h = 1e-5 * rc
    x = []
    for a in range(3):
        for sgn in (1.0, -1.0):
            xa = g["y"][sites].copy()
            xa[:, a] += sgn * h
            x.append(xa)
    x = np.concatenate(x)
    p64 = P.Plan(g["L"], 1e-9, precision="fp64")
    p64.set_sources(g["y"], g["q"])
    phi, _ = p64.eval_targets(x, grad=False)
    p64.close()
    phi = phi.reshape(3, 2, 64)
    fd = ((phi[:, 0, :] - phi[:, 1, :]) / (2 * h)).T  # (64, 3)
    e = _rel(gm[sites], fd)
    print(f"water 333k finite differences: E_grad(mixed vs FD of FP64)={e:.2e}")
    assert e <= 1e-5


def test_batched_256_fullsize():
    P, _ = _cuda()
    ref = _golden("batched_256")
    cells = W.batched_cells(256)
    assert len(cells) == len(ref["cells"]) == 256
    samples = [_check_inputs(g, c) for g, c in zip(cells, ref["cells"])]
    b = P.Batch([(g["L"], 1e-6) for g in cells], precision="mixed")
    b.set_sources([g["y"] for g in cells], [g["q"] for g in cells])
    pots, grads = b.eval()
    ep, eg = [], []
    for c, (idx, pref, gref) in enumerate(samples):
        assert np.all(np.isfinite(pots[c])) and np.all(np.isfinite(grads[c]))
        ep.append(_rel(pots[c][idx], pref))
        eg.append(_rel(grads[c][idx], gref))
    ep, eg = np.array(ep), np.array(eg)
    # 64 seeded targets per cell: every cell is held to the requested eps on its own
    print(f"256 cells mixed: worst E_pot={ep.max():.2e} (cell {int(ep.argmax())}) E_grad={eg.max():.2e} "
          f"(cell {int(eg.argmax())}), rms E_pot={float(np.sqrt(np.mean(ep ** 2))):.2e}, "
          f"points={sum(len(g['q']) for g in cells)}")
    assert ep.max() <= 1e-6
    assert eg.max() <= 1e-5
    b.close()
