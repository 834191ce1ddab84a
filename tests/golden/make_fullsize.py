"""Writes the stored reference values of the full-size parity tests: the FP64 Ewald oracle's
potential and gradient at a seeded sample of targets of each full-size synthetic workload.
It calls only the oracle and the seeded input generators.

    python tests/golden/make_fullsize.py [triclinic3d_4m] [water_333k] [batched_256] [oblique2d_200k]

Each output file holds, besides the values, the sampled indices and the sampled inputs
(positions and charges), which the tests compare against a fresh generation to make sure
the stored values belong to the inputs they evaluate.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ewald as E  # noqa: E402


def sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, k, replace=False))


def one_cell(g, idx):
    pot, grad = E.ewald(g["L"], g["y"], g["q"], x=g["y"][idx], self_idx=idx)
    return dict(name=g["name"], L=g["L"].tolist(), n=int(len(g["q"])), idx=idx.tolist(),
                y=g["y"][idx].tolist(), q=g["q"][idx].tolist(), pot=pot.tolist(), grad=grad.tolist())


def write(name, obj):
    path = os.path.join(HERE, f"fullsize_{name}.json")
    with open(path, "w") as f:
        json.dump(obj, f, indent=None, separators=(",", ":"))
        f.write("\n")
    print("wrote", path, flush=True)


def triclinic3d_4m():
    g = W.triclinic3d_clusters(4_000_000)
    return dict(workload="triclinic3d_clusters(4_000_000)", oracle="ewald, tol 1e-15", cells=[one_cell(g, sample(len(g["q"]), 64, 21))])


def water_333k():
    g = W.water_box(333_000)
    return dict(workload="water_box(333_000)", oracle="ewald, tol 1e-15", cells=[one_cell(g, sample(len(g["q"]), 64, 22))])


def batched_256():
    # 64 seeded targets per cell: enough to hold every cell's relative L2 error to eps
    cells = W.batched_cells(256)
    out = []
    for c, g in enumerate(cells):
        out.append(one_cell(g, sample(len(g["q"]), 64, 1000 + c)))
    return dict(workload="batched_cells(256)", oracle="ewald, tol 1e-15", cells=out)


def oblique2d_200k():
    g = W.oblique2d_clusters(200_000)
    return dict(workload="oblique2d_clusters(200_000)", oracle="ewald, tol 1e-15", cells=[one_cell(g, sample(len(g["q"]), 64, 23))])


MAKERS = {"triclinic3d_4m": triclinic3d_4m, "water_333k": water_333k, "batched_256": batched_256,
          "oblique2d_200k": oblique2d_200k}

if __name__ == "__main__":
    names = sys.argv[1:] or list(MAKERS)
    for nm in names:
        t = time.time()
        write(nm, MAKERS[nm]())
        print(f"{nm}: {time.time() - t:.1f} s", flush=True)
