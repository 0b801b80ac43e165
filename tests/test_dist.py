"""The multi-GPU host logic on CPU: two gloo ranks run the helpers that
bench.py's torchrun path uses (barrier, max over ranks, per-rank workloads),
with no GPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import json

    import torch.distributed as tdist

    import bench
    from paper_2108_02997_gb300 import dist, graphgen as gg
    w, r, _ = dist.init("cpu")
    assert (w, r) == (world, rank)
    dist.barrier(w, "cpu")
    mx = dist.max_over_ranks(1.5 * (rank + 1), w, "cpu")
    wl = bench.make_workload("sweep330", gg, rank)
    graphs, specs = wl.graphs, wl.specs
    shapes = [None] * world
    tdist.all_gather_object(shapes, (graphs[0].n, len(specs), int(graphs[0].sources[:64].sum())))
    dist.barrier(w, "cpu")
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": mx, "shapes": shapes}, f)
    dist.finish(w)


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import json

    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in range(world)]
    for r in res:
        assert r["max"] == 3.0                     # max over ranks of 1.5 * (rank + 1)
        (n0, k0, h0), (n1, k1, h1) = r["shapes"]
        assert n0 == n1 == 10000 and k0 == k1 == 330   # same shape on every rank
        assert h0 != h1                                # but each rank its own graph


def test_single_process_defaults(monkeypatch):
    from paper_2108_02997_gb300 import dist
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert dist.env() == (1, 0, 0)
    assert dist.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert dist.rank_seed(22, 0) == 22 and dist.rank_seed(22, 1) != 22
