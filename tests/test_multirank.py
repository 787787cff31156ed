"""The N > 1 path on the CPU: two processes over gloo (127.0.0.1).

* bench.py's rank setup, barrier and max-over-ranks timing, and the
  per-rank workloads (disjoint seeds: weak scaling, no data-path
  collective); the reference arm runs on rank 0 alone;
* the dataset generator: shards dealt round-robin to the ranks, every item
  written exactly once, rank 0 merging after the barrier.
"""

import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(WORLD), LOCAL_RANK=str(rank))


def _bench_rank(rank, port, out):
    _env(rank, port)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup(WORLD)
    try:
        assert (ws, r, local) == (WORLD, rank, rank)
        bench.barrier(ws)
        m = bench.max_over_ranks(ws, 1.5 + rank)
        args = bench.parse_args(["--gpus", str(WORLD)])
        strings, _ = bench.make_workload(args, rank)
        split_args = bench.parse_args(["--gpus", str(WORLD), "--workload", "mixed", "--partition", "lpt",
                                       "--strings", "64", "--seconds", "0.5"])
        split, _ = bench.make_workload(split_args, rank)
        ref = bench.run_reference(bench.parse_args(["--impl", "reference"]), ws, rank) if rank else None
        with open(os.path.join(out, f"bench{rank}.json"), "w") as f:
            json.dump({"max": m, "f0": [d["f0"] for d in strings], "ref": ref,
                       "split": [d["f0"] for d in split], "batch_samples": split_args.batch_samples}, f)
    finally:
        dist.destroy_process_group()


def test_bench_rank_helpers(tmp_path):
    mp.spawn(_bench_rank, args=(free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    got = [json.load(open(tmp_path / f"bench{r}.json")) for r in range(WORLD)]
    assert all(g["max"] == 1.5 + WORLD - 1 for g in got)
    # each rank its own 4096-string batch (weak scaling)
    assert len(got[0]["f0"]) == len(got[1]["f0"]) == 4096
    assert not set(got[0]["f0"]) & set(got[1]["f0"])
    # the reference arm runs on rank 0 alone; the others return without work
    assert got[1]["ref"] == 0
    # --partition lpt: one 64-string batch split between the ranks, every
    # string on exactly one of them
    from paper_2311_18505_gb300 import workloads as W
    whole = W.batch_mixed(64, seconds=0.5, seed=2)
    assert sorted(got[0]["split"] + got[1]["split"]) == sorted(d["f0"] for d in whole)
    assert not set(got[0]["split"]) & set(got[1]["split"])
    assert got[0]["batch_samples"] == got[1]["batch_samples"] == sum(d["n_samples"] for d in whole)


def _dataset_rank(rank, port, out):
    _env(rank, port)
    import torch.distributed as dist
    from paper_2311_18505_gb300 import dataset as D
    from test_dataset import SMALL, fake_renderer
    dist.init_process_group("gloo")
    try:
        mine = D.generate(out, 11, SMALL, seed=12, shard_size=3, rank=rank, world=WORLD, render=fake_renderer())
        assert mine == list(range(rank, 4, WORLD))
        dist.barrier()
        if rank == 0:
            assert D.merge_metadata(out) == 11
    finally:
        dist.destroy_process_group()


def test_dataset_two_ranks(tmp_path):
    out = str(tmp_path / "ds")
    mp.spawn(_dataset_rank, args=(free_port(), out), nprocs=WORLD, join=True)
    from paper_2311_18505_gb300 import dataset as D
    from test_dataset import SMALL
    audio, index, status = D.load(out)
    assert list(index) == list(range(11)) and not status.any()
    for i in range(11):
        assert np.all(audio[i] == np.float32(D.draw(SMALL, 12, i)["f0"]))
    lines = [json.loads(l) for l in open(os.path.join(out, "metadata.jsonl"))]
    assert [m["index"] for m in lines] == list(range(11))
