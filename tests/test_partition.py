"""Partition of independent cells over ranks (pdmk_cell_work, pdmk_partition_cells): host
only.  A multi-GPU run over a batch of cells splits the cells by estimated work and exchanges
nothing on the data path; every rank computes the same partition on its own."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_2606_28608_b300 as P  # noqa: E402
import workloads as W  # noqa: E402


def test_lpt_assignment_small_case():
    # decreasing work 5, 4, 3, 3, 3 over two ranks: 5 -> r0, 4 -> r1, 3 -> r1 (4 < 5),
    # 3 -> r0 (5 < 7), 3 -> r1 (7 < 8)
    assert P.partition_cells([5, 4, 3, 3, 3], 2).tolist() == [0, 1, 1, 0, 1]
    # ties in work keep index order; ties in load go to the lowest rank
    assert P.partition_cells([1, 1, 1, 1], 4).tolist() == [0, 1, 2, 3]
    assert P.partition_cells([2.0], 3).tolist() == [0]
    assert P.partition_cells([], 2).tolist() == []


def test_partition_rejects_bad_arguments():
    with pytest.raises(P.PdmkError):
        P.partition_cells([1.0, -1.0], 2)
    with pytest.raises(P.PdmkError):
        P.partition_cells([1.0, float("nan")], 2)
    with pytest.raises(P.PdmkError):
        P.partition_cells([1.0], 0)


def test_cell_work_estimate():
    L3 = W.lattice_from_lengths_angles(2.0, 3.0, 2.5, 80, 95, 100)
    w1 = P.cell_work(L3, 1e-6, 10000)
    w2 = P.cell_work(L3, 1e-6, 20000)
    assert 0 < w1 < w2 < 2 * w1 + 1  # linear in n plus a transform term
    assert P.cell_work(L3, 1e-3, 10000) < w1 < P.cell_work(L3, 1e-9, 10000)
    with pytest.raises(P.PdmkError):
        P.cell_work(L3, 1e-1, 10)
    with pytest.raises(P.PdmkError):
        P.cell_work(np.full((3, 3), np.nan), 1e-6, 10)


def _balanced(work, owner, nranks):
    load = np.zeros(nranks)
    for w, r in zip(work, owner):
        load[r] += w
    # the LPT bound: no rank exceeds the mean by more than the largest cell
    return load.max() <= load.sum() / nranks + max(work) + 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_2606_28608_b300 as PP
    import workloads as WW
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    cells = WW.batched_cells(32, nmax=5000)
    work = [PP.cell_work(c["L"], 1e-6, len(c["q"])) for c in cells]
    owner = PP.partition_cells(work, ws)
    mine = [i for i, r in enumerate(owner) if r == rank]
    # compare the partitions the ranks computed on their own
    t = torch.tensor(owner.astype(np.int64))
    got = [torch.zeros_like(t) for _ in range(ws)]
    dist.all_gather(got, t)
    q.put((rank, [g.tolist() for g in got], mine, work))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed unavailable")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, parts0, mine0, work), (_, parts1, mine1, _) = out
    assert parts0[0] == parts0[1] == parts1[0] == parts1[1]  # every rank computed the same
    assert sorted(mine0 + mine1) == list(range(32)) and not set(mine0) & set(mine1)
    assert _balanced(work, parts0[0], 2)
