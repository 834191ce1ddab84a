"""Batched cells (pdmk_batch_*): every cell's result equals its own single-cell plan's, bit
for bit (same kernels, same data, deterministic sums), for the eager first evaluation and the
graph replays; and the batch matches the FP64 oracle per cell."""
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


def _cells():
    rng = np.random.default_rng(40)
    cells = []
    for k in range(5):
        if k % 2 == 0:
            L = W.lattice_from_lengths_angles(*rng.uniform(1, 4, 3), *rng.uniform(60, 120, 3))
            g = W.random_neutral(L, int(rng.integers(300, 1500)), seed=100 + k)
        else:
            L = np.array([[1.0, rng.uniform(-0.4, 0.4)], [0.0, rng.uniform(0.6, 1.4)]])
            g = W.random_neutral(L, int(rng.integers(500, 3000)), seed=100 + k)
        cells.append(g)
    return cells


@pytest.mark.parametrize("precision,eps", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_batch_equals_single_cells(precision, eps):
    P, torch = _cuda()
    cells = _cells()
    b = P.Batch([(g["L"], eps) for g in cells], precision=precision)
    b.set_sources([g["y"] for g in cells], [g["q"] for g in cells])
    first = b.eval()
    second = b.eval()   # graph capture
    third = b.eval()    # replay
    for c, g in enumerate(cells):
        pl = P.Plan(g["L"], eps, precision=precision)
        pl.set_sources(g["y"], g["q"])
        p, gr = pl.eval()
        pl.close()
        for pots, grads in (first, second, third):
            assert np.array_equal(pots[c], p) and np.array_equal(grads[c], gr)
    b.close()


def test_batch_against_oracle():
    P, _ = _cuda()
    cells = _cells()[:3]
    b = P.Batch([(g["L"], 1e-6) for g in cells], precision="mixed")
    b.set_sources([g["y"] for g in cells], [g["q"] for g in cells])
    pots, grads = b.eval()
    for c, g in enumerate(cells):
        pref, gref = E.ewald(g["L"], g["y"], g["q"])
        assert np.linalg.norm(pots[c] - pref) <= 1e-6 * np.linalg.norm(pref)
        assert np.linalg.norm(grads[c] - gref) <= 1e-5 * np.linalg.norm(gref)
    b.close()


def test_rank_shares_equal_the_whole_batch():
    """Cells split over two ranks by estimated work (pdmk_partition_cells): each rank's batch of
    its own cells gives, cell for cell, the single-process batch's results bit for bit.  The
    two ranks' batches run one after the other on this GPU (nothing is exchanged between
    ranks, so running them in sequence is the multi-GPU run's arithmetic)."""
    P, torch = _cuda()
    cells = _cells()
    work = [P.cell_work(g["L"], 1e-6, len(g["q"])) for g in cells]
    owner = P.partition_cells(work, 2)
    assert set(owner.tolist()) == {0, 1}
    whole = P.Batch([(g["L"], 1e-6) for g in cells], precision="mixed")
    whole.set_sources([g["y"] for g in cells], [g["q"] for g in cells])
    wp, wg = whole.eval()
    whole.close()
    for r in (0, 1):
        mine = [c for c in range(len(cells)) if owner[c] == r]
        b = P.Batch([(cells[c]["L"], 1e-6) for c in mine], precision="mixed")
        b.set_sources([cells[c]["y"] for c in mine], [cells[c]["q"] for c in mine])
        pp, gg = b.eval()
        b.close()
        for k, c in enumerate(mine):
            assert np.array_equal(pp[k], wp[c]) and np.array_equal(gg[k], wg[c])
