"""Multi-rank host logic on CPU: world_size-2 gloo ranks shard a batch by
LPT over pair work, compute their shards (CPU oracle standing in for the GPU
kernels) and gather the results in input order; rank 0 compares with the
single-process results."""
import os
import socket

import numpy as np
import pytest

from paper_2002_05200_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = synth.uneven_batch(n_pairs=120, seed=9, max_len=6000)
        idx = shard.shard_indices(b, world, rank)
        res, _ = oracle.run_batch(b.subset(idx), threads=2)
        full = shard.gather_results(res, idx, b.n_pairs)
        ms, cells = shard.reduce_step(10.0 + rank, int(res["cells"].sum()))
        if rank == 0:
            np.save(out_path, full)
            with open(out_path + ".txt", "w") as fh:
                fh.write(f"{ms} {cells}\n")
    finally:
        dist.destroy_process_group()


def test_lpt_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    work = rng.integers(1, 10_000, size=1000)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(work, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(work.size))
        loads = [int(work[p].sum()) for p in parts]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(loads) / world + work.max()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    out = str(tmp_path / "res.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    full = np.load(out)
    b = synth.uneven_batch(n_pairs=120, seed=9, max_len=6000)
    ref, _ = oracle.run_batch(b, threads=2)
    assert np.array_equal(full, ref)
    ms, cells = open(out + ".txt").read().split()
    assert float(ms) == 11.0 and int(cells) == int(ref["cells"].sum())
