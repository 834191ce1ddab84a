"""The stored full-size oracle values (tests/golden/fullsize_*.json, written by
tests/golden/make_fullsize.py from the oracle alone) belong to the inputs the seeded
generators produce today: sampled positions to rounding, charges exactly, sizes and cells."""
import json
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, f"fullsize_{name}.json")) as f:
        return json.load(f)


def _check(g, cell):
    idx = np.asarray(cell["idx"])
    assert len(g["q"]) == cell["n"]
    assert np.allclose(np.asarray(cell["L"]), g["L"], rtol=0, atol=1e-14)
    assert np.allclose(g["y"][idx], np.asarray(cell["y"]), rtol=0, atol=1e-12 * np.abs(g["L"]).max())
    assert np.array_equal(g["q"][idx], np.asarray(cell["q"]))
    pot, grad = np.asarray(cell["pot"]), np.asarray(cell["grad"])
    assert pot.shape == idx.shape and grad.shape == (len(idx), g["L"].shape[0])
    assert np.all(np.isfinite(pot)) and np.all(np.isfinite(grad))


@pytest.mark.parametrize("name,make", [
    ("triclinic3d_4m", lambda: [W.triclinic3d_clusters(4_000_000)]),
    ("water_333k", lambda: [W.water_box(333_000)]),
    ("batched_256", lambda: W.batched_cells(256)),
])
def test_stored_values_match_generated_inputs(name, make):
    ref = _load(name)
    gens = make()
    assert len(gens) == len(ref["cells"])
    for g, cell in zip(gens, ref["cells"]):
        _check(g, cell)
