"""The periodic root of cubic (square) cells (Remark 3.3, pdmk_opts.root_mode = 0): no image
sources (n_images = n), neighbours across the faces as virtual copies shifted by L n.  Checked
against the FP64 Ewald oracle and against the multi-cube root with images (root_mode = 1):
uniform and clustered cells with shallow and deep trees, both precisions, and the NaCl and
CsCl Madelung constants."""
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


def _clustered_cube(n, d, a, seed):
    rng = np.random.default_rng(seed)
    L = a * np.eye(d)
    centres = rng.random((6, d))
    u = (centres[np.arange(n) % 6] + 0.02 * rng.standard_normal((n, d))) % 1.0
    q = rng.standard_normal(n)
    q -= q.mean()
    return dict(L=L, y=u @ L.T, q=q)


CASES = {
    "cube_uniform": (lambda: W.cube_uniform(2000), {}),
    "cube_deep": (lambda: _clustered_cube(20000, 3, 2.5, 81), {"n_s": 40}),
    "square_uniform": (lambda: W.random_neutral(1.7 * np.eye(2), 3000, seed=82), {}),
    "square_deep": (lambda: _clustered_cube(30000, 2, 1.0, 83), {}),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,eps", [("fp64", 1e-6), ("fp64", 1e-9), ("mixed", 1e-6)])
def test_periodic_root_against_oracle(case, prec, eps):
    P = _cuda()
    make, opts = CASES[case]
    g = make()
    pref, gref = E.ewald(g["L"], g["y"], g["q"])
    res = {}
    for mode in (0, 1):
        plan = P.Plan(g["L"], eps, precision=prec, root_mode=mode, **opts)
        plan.set_sources(g["y"], g["q"])
        pot, grad = plan.eval()
        info = plan.info()
        plan.close()
        res[mode] = (pot, grad, info)
    p0, g0, i0 = res[0]
    p1, g1, i1 = res[1]
    assert i0["n_images"] == len(g["q"])      # the periodic root makes no images
    assert i1["n_images"] > len(g["q"])
    e0, eg0 = rel(p0, pref), rel(g0, gref)
    print(f"{case} {prec} {eps:g}: periodic root E_pot={e0:.2e} E_grad={eg0:.2e} depth={i0['depth']}, "
          f"images E_pot={rel(p1, pref):.2e}")
    assert e0 <= eps and eg0 <= 10 * eps
    assert rel(p1, pref) <= eps


def test_periodic_root_madelung():
    """NaCl (conventional cubic cell) and CsCl through the periodic root: the Madelung
    constants to 1e-9 (constants cited in tests/golden/madelung.txt)."""
    P = _cuda()
    for g, M, r0 in ((W.nacl_conventional(), 1.7475645946331822, 0.5),
                     (W.cscl_cubic(), 1.7626747730709884, 0.8660254037844386)):
        plan = P.Plan(g["L"], 1e-9, precision="fp64")
        plan.set_sources(g["y"], g["q"])
        pot, _ = plan.eval()
        assert plan.info()["n_images"] == len(g["q"])
        plan.close()
        # Phi_i = -q_i M / (4 pi r0) for unit charges
        want = -g["q"] * M / (4 * np.pi * r0)
        assert np.max(np.abs(pot - want)) <= 1e-9 * np.max(np.abs(want))
