"""One batch split across ranks (the paper's multi-GPU balancer, Sec. IV-C):
two gloo ranks, one process each, both on the one GPU here, each extend
their LPT share of the SAME batch through the C ABI; the gathered results
equal the oracle's on every pair.  The ranks never wait on each other inside
a kernel: the only exchange is the host-side gather after each rank's
stream has finished."""
import os
import socket

import numpy as np
import pytest

from paper_2002_05200_gb300 import shard, synth

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    return synth.uneven_batch(n_pairs=300, seed=21, max_len=40_000)


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    from paper_2002_05200_gb300 import logan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _batch()
        idx = shard.shard_indices(b, world, rank)
        sb = shard.shard_batch(b, idx)
        ctx = logan.Context(0)
        try:
            A, B, S, Xs = logan.batch_to_device(sb, packed2bit=False)
            out = ctx.extend(A, B, S, sb.match, sb.mismatch, sb.gap, sb.X, Xs)
            torch.cuda.synchronize()
            res = logan.results_to_numpy(out)
        finally:
            ctx.close()
        full = shard.gather_results(res, idx, b.n_pairs)
        if rank == 0:
            np.save(out_path, full)
            np.save(out_path + ".sizes.npy", np.array([idx.size]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_one_batch_on_gpu(tmp_path):
    import torch
    import torch.multiprocessing as mp

    from tests.gpu_common import assert_same, run_oracle
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    full = np.load(out)
    b = _batch()
    n0 = int(np.load(out + ".sizes.npy")[0])
    assert 0 < n0 < b.n_pairs  # both ranks had work
    assert_same(full, run_oracle(b), "two LPT shards, gathered")
