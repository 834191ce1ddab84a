"""The source set-up on the device (pdmk_opts.build_mode) against the host build.

build="compare" runs both builds and compares every array a set-up leaves (the tree's
per-box arrays, the sorted order, the per-point records of the near field, the far field
and the plane-wave passes, the direct lists and their entries, the host copies) byte for
byte; set_sources raises with the first differing array otherwise.  The cases cover 2D and
3D cells, shallow and deep trees, the periodic root of cubic cells, images across every
face, sources given outside the cell, tiny cells, separate targets, a depth limit and both
precisions; then the full-size 4M-point triclinic and 200k-point oblique cells.  The
evaluations after a device set-up are checked against the FP64 Ewald oracle by every other
GPU test, since the device build is the default."""
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


L2 = np.array([[1.0, 0.45], [0.0, 0.85]])
L3 = W.lattice_from_lengths_angles(1.0, 1.3, 0.8, 75, 100, 110)


def _outside(L, n, seed):
    g = W.random_neutral(L, n, seed=seed)
    rng = np.random.default_rng(seed)
    shift = rng.integers(-3, 4, size=(n, L.shape[0])).astype(float)
    return {"L": L, "y": g["y"] + shift @ L.T, "q": g["q"]}


CASES = {
    "oblique2d": (lambda: W.oblique2d_clusters(3000, seed=911), {}),
    "oblique2d_deep": (lambda: W.oblique2d_clusters(20000, seed=912), {}),
    "ring2d_aspect100": (lambda: W.wavy_ring2d(20000, aspect=100.0, seed=913), {}),
    "square_periodic_root": (lambda: W.random_neutral(np.eye(2), 3000, seed=914), {"n_s": 20}),
    "triclinic3d": (lambda: W.triclinic3d_clusters(3000, nclusters=8, seed=915), {}),
    "triclinic3d_deep": (lambda: W.triclinic3d_clusters(12000, nclusters=8, seed=916), {"n_s": 60}),
    "slab3d": (lambda: W.wavy_sphere3d(20000, scale=(1, 1, 0.1), triclinic=True, seed=917), {}),
    "cube_periodic_root": (lambda: W.cube_uniform(2000, seed=918), {"n_s": 20}),
    "cube_images": (lambda: W.cube_uniform(2000, seed=918), {"n_s": 20, "root_mode": 1}),
    "water": (lambda: W.water_box(2000, seed=919), {}),
    "outside2d": (lambda: _outside(L2, 1500, 920), {}),
    "outside3d": (lambda: _outside(L3, 1500, 921), {}),
    "depth_limit3d": (lambda: W.triclinic3d_clusters(12000, nclusters=8, seed=922), {"n_s": 20, "max_depth": 2}),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_build_equals_host_build(case, prec):
    P, _ = _cuda()
    make, opts = CASES[case]
    g = make()
    plan = P.Plan(g["L"], 1e-6, precision=prec, build="compare", **opts)
    plan.set_sources(g["y"], g["q"])  # raises if any array differs
    assert plan.message() == "device and host set-up identical"
    assert "tree_device_images" in plan.setup_times()
    info = plan.info()
    print(f"{case} {prec}: identical; depth={info['depth']} boxes={info['nboxes']} images={info['n_images']}")
    plan.close()


@pytest.mark.parametrize("n", [1, 2, 7])
@pytest.mark.parametrize("L", [L2, L3], ids=["2d", "3d"])
def test_device_build_tiny_cells(n, L):
    P, _ = _cuda()
    rng = np.random.default_rng(60 + n)
    y = rng.random((n, L.shape[0])) @ L.T
    q = rng.standard_normal(n)
    plan = P.Plan(L, 1e-6, precision="fp64", build="compare")
    plan.set_sources(y, q)
    assert plan.message() == "device and host set-up identical"
    plan.close()


def test_device_build_separate_targets():
    P, _ = _cuda()
    g = W.triclinic3d_clusters(4000, nclusters=8, seed=923)
    rng = np.random.default_rng(9)
    x = (rng.random((700, 3)) + rng.integers(-1, 2, size=(700, 3))) @ g["L"].T
    plan = P.Plan(g["L"], 1e-6, precision="mixed", build="compare")
    plan.set_sources(g["y"], g["q"], x=x)
    assert plan.message() == "device and host set-up identical"
    plan.close()


def test_device_build_device_inputs_and_default_mode():
    """Device-resident inputs through the default (device) build, then an evaluation, new
    targets and a Bloch sum (which download the host copies on first use), against the
    oracle."""
    P, torch = _cuda()
    g = W.oblique2d_clusters(5000, seed=924)
    plan = P.Plan(g["L"], 1e-6, precision="mixed")
    y = torch.tensor(g["y"], device="cuda")
    q = torch.tensor(g["q"], device="cuda")
    plan.set_sources(y, q)
    assert "tree_device_images" in plan.setup_times()
    pot, grad = plan.eval()
    rng = np.random.default_rng(3)
    idx = rng.choice(len(g["q"]), 64, replace=False)
    pref, gref = E.ewald(g["L"], g["y"], g["q"], x=g["y"][idx], self_idx=idx)
    assert np.linalg.norm(pot[idx] - pref) / np.linalg.norm(pref) <= 1e-6
    assert np.linalg.norm(grad[idx] - gref) / np.linalg.norm(gref) <= 1e-5
    x = rng.random((50, 2)) @ g["L"].T
    pt, _ = plan.eval_targets(x)
    pxr, _ = E.ewald(g["L"], g["y"], g["q"], x=x)
    assert np.linalg.norm(pt - pxr) / np.linalg.norm(pxr) <= 1e-6
    plan.close()


def test_device_build_rejects_bad_inputs():
    P, _ = _cuda()
    g = W.cube_uniform(500, seed=925)
    plan = P.Plan(g["L"], 1e-3, build="device", neutrality=0)
    y = g["y"].copy()
    y[3, 1] = np.inf
    with pytest.raises(P.PdmkError) as ei:
        plan.set_sources(y, g["q"])
    assert ei.value.code == -5  # NONFINITE
    q = g["q"].copy()
    q[0] += 1.0
    with pytest.raises(P.PdmkError) as ei:
        plan.set_sources(g["y"], q)
    assert ei.value.code == -3  # NON_NEUTRAL
    plan.set_sources(g["y"], g["q"])
    plan.close()


@pytest.mark.parametrize("name", ["triclinic3d_4m", "oblique2d_200k"])
def test_device_build_fullsize(name):
    P, _ = _cuda()
    g = W.triclinic3d_clusters(4_000_000) if name == "triclinic3d_4m" else W.oblique2d_clusters(200_000)
    plan = P.Plan(g["L"], 1e-6, precision="mixed", build="compare")
    plan.set_sources(g["y"], g["q"])
    assert plan.message() == "device and host set-up identical"
    plan.close()
    plan = P.Plan(g["L"], 1e-6, precision="mixed")
    plan.set_sources(g["y"], g["q"])
    t = plan.setup_times()
    print(f"{name}: device set-up {sum(t.values()):.0f} ms: " +
          ", ".join(f"{k} {v:.0f}" for k, v in t.items()))
    plan.close()
