"""Helpers shared by the GPU parity tests: run a synth.Batch through the C ABI
and through the oracle, and compare field by field (integer results:
bit-exact)."""
import numpy as np

import oracle
from paper_2002_05200_gb300 import logan

FIELDS = ("score", "left", "right", "begA", "begB", "endA", "endB", "cells")


def run_gpu(ctx, b, packed2bit=False, plain=False, graphs=False):
    import torch
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=packed2bit)
    ctx.set_option(logan.OPT_GRAPHS, 1 if graphs else 0)
    out = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, plain=plain)
    torch.cuda.synchronize()
    return logan.results_to_numpy(out)


def run_oracle(b, threads=None):
    res, _ = oracle.run_batch(b, threads)
    return res


def run_oracle_all(b, chunk=8192, threads=None, run=None):
    """The oracle on every pair of a (possibly 2-bit packed) batch, on all
    host cores: pairs ordered longest first so the long extensions start
    early, in chunks of `chunk` pairs (each chunk's sequences decoded to
    ASCII on its own, which bounds host memory); results in input order.
    `run(sub)` replaces the linear oracle (e.g. the affine one)."""
    key = (b.lenA[b.seeds["idxA"]].astype(np.int64) + b.lenB[b.seeds["idxB"]].astype(np.int64))
    order = np.argsort(-key, kind="stable")
    out = np.zeros(b.n_pairs, dtype=oracle.PAIR_DTYPE)
    for c0 in range(0, b.n_pairs, chunk):
        idx = order[c0:c0 + chunk]
        sub = b.subset(idx)
        out[idx] = run_oracle(sub, threads) if run is None else run(sub)
    return out


def assert_same(gpu, ref, label=""):
    assert gpu.shape[0] == ref.shape[0]
    ok_ref = ref["status"] == oracle.OK
    ok_gpu = gpu["status"] == logan.OK
    bad = np.flatnonzero(ok_ref != ok_gpu)
    assert bad.size == 0, f"{label}: status differs at pairs {bad[:10]}: " \
                          f"gpu {gpu['status'][bad[:10]]} oracle {ref['status'][bad[:10]]}"
    for f in FIELDS:
        g = gpu[f][ok_gpu].astype(np.int64)
        r = ref[f][ok_ref].astype(np.int64)
        diff = np.flatnonzero(g != r)
        if diff.size:
            idx = np.flatnonzero(ok_gpu)[diff[:5]]
            raise AssertionError(f"{label}: field {f} differs at {diff.size} pairs, e.g. "
                                 f"pairs {idx}: gpu {g[diff[:5]]} oracle {r[diff[:5]]}")
    for f in FIELDS:
        assert np.all(gpu[f][~ok_gpu] == 0)
