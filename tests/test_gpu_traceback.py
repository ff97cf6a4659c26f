"""Alignment paths on the GPU (logan_traceback_batch) vs the traceback
oracle: every pair's run-length operations exactly; the paths span the
extension's reported coordinates and rescore to its score."""
import numpy as np
import pytest

import oracle
from paper_2002_05200_gb300 import logan, synth

pytestmark = pytest.mark.gpu

OPS = "MID"


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


def rle(ops: str):
    out = []
    for o in ops:
        code = OPS.index(o)
        if out and (out[-1] & 15) == code:
            out[-1] += 16
        else:
            out.append(16 | code)
    return out


def gpu_paths(ctx, b, packed2bit=False):
    import torch
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=packed2bit)
    codes, start, count = ctx.traceback(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
    res = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
    torch.cuda.synchronize()
    c = codes.cpu().numpy().view(np.uint32)
    st, ct = start.cpu().numpy(), count.cpu().numpy()
    return [list(c[st[p]:st[p] + ct[p]]) for p in range(b.n_pairs)], logan.results_to_numpy(res)


def check(b, paths, res, Xs=None):
    for p in range(b.n_pairs):
        s = b.seeds[p]
        if res["status"][p] != 0:
            assert paths[p] == []
            continue
        X = int(b.Xs[p]) if b.Xs is not None else b.X
        want = oracle.pair_traceback(b.seqA(p), b.seqB(p), int(s["posA"]), int(s["posB"]),
                                     int(s["len"]), b.match, b.mismatch, b.gap, X)
        assert [int(x) for x in paths[p]] == rle(want), p
        # the path spans the reported coordinates and rescores to the score
        A, B = b.seqA(p), b.seqB(p)
        i, j, sc = int(res["begA"][p]), int(res["begB"][p]), 0
        for code in paths[p]:
            op, n = int(code) & 15, int(code) >> 4
            for _ in range(n):
                if op == 0:
                    sc += b.match if A[i] == B[j] else b.mismatch
                    i += 1; j += 1
                elif op == 1:
                    sc += b.gap; i += 1
                else:
                    sc += b.gap; j += 1
        assert (i, j, sc) == (int(res["endA"][p]), int(res["endB"][p]), int(res["score"][p]))


def test_uniform_pairs(ctx):
    b = synth.uniform_pairs(n_pairs=200)
    check(b, *gpu_paths(ctx, b))


def test_lognormal_packed(ctx):
    b = synth.lognormal_batch(n_pairs=120)
    check(b, *gpu_paths(ctx, b, packed2bit=True))


def test_uneven_per_pair_x(ctx):
    b = synth.uneven_batch(n_pairs=80, max_len=15_000, seed=81)
    check(b, *gpu_paths(ctx, b, packed2bit=True))


@pytest.mark.parametrize("seed", range(2))
def test_tiny_edge_cases(ctx, seed):
    b = synth.tiny_pairs(2000, 40, seed=seed)
    check(b, *gpu_paths(ctx, b))


@pytest.mark.parametrize("scheme", [(2, -3, -2), (1, -1, 0), (5, -4, -7)])
def test_scoring_schemes(ctx, scheme):
    b = synth.uniform_pairs(n_pairs=60)
    b.match, b.mismatch, b.gap = scheme
    check(b, *gpu_paths(ctx, b))


def test_invalid_pairs_have_no_path(ctx):
    b = synth.uniform_pairs(n_pairs=30)
    pool = b.poolA.copy()
    pool[::97] = ord("N")
    b.poolA = pool
    paths, res = gpu_paths(ctx, b)
    bad = res["status"] != 0
    assert bad.any() and all(paths[p] == [] for p in np.flatnonzero(bad))
    check(b, paths, res)


@pytest.mark.parametrize("median,X,n", [(3000, 300, 12), (10_000, 1500, 4)])
def test_wide_bands_block_and_device_rings(ctx, median, X, n):
    # unrelated pairs: bands past a warp's 512-row ring (the block form),
    # and at X = 1500 on 10 kbp pairs past 2048 rows (the device-memory ring)
    b = synth.lognormal_batch(n_pairs=n, median=median, lo=median - 500, hi=median + 500,
                              related_frac=0.0, X=X, seed=5)
    check(b, *gpu_paths(ctx, b, packed2bit=True))


def test_timing_stats(ctx):
    b = synth.uniform_pairs(n_pairs=50)
    A, B, S, Xs = logan.batch_to_device(b)
    ctx.set_option(logan.OPT_TIMING, 1)
    try:
        ctx.traceback(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
        st = ctx.traceback_stats()
        ext_launches = ctx.last_stats()["launches"]  # the call's own batch pipeline
    finally:
        ctx.set_option(logan.OPT_TIMING, 0)
    assert st["sweep_ms"] > 0 and st["record_ms"] > 0 and st["walk_ms"] > 0
    assert st["total_ms"] >= st["sweep_ms"] + st["record_ms"] + st["walk_ms"] - 1e-3
    assert st["code_words"] > 0
    # the recorded cells: every anti-diagonal up to the best one of each side
    res = logan.results_to_numpy(ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs))
    assert 0 < st["record_cells"] <= int(res["cells"].sum())
    assert st["code_words"] >= st["record_cells"] // 16
    # the pipeline's launches + prepare, the item order's ids, three
    # recording sweeps (blocks for the wide items beside the warps, blocks
    # for the items that outgrew a warp), walk, join
    assert st["launches"] == ext_launches + 7


@pytest.mark.parametrize("opt,val", [("OPT_GRAPHS", 1), ("OPT_CONCURRENT", 0),
                                     ("OPT_MIGRATION_MB", 0), ("OPT_FORCE_LEVEL", 0)])
def test_pipeline_options(ctx, opt, val):
    # the call's first step is the batch pipeline: its options change the
    # schedule, never the paths
    import torch
    b = synth.lognormal_batch(n_pairs=60, median=4000, lo=2000, hi=8000, seed=11)
    key = getattr(logan, opt)
    old = ctx.get_option(key)
    ctx.set_option(key, val)
    try:
        stream = torch.cuda.Stream()  # graphs are captured on a non-default stream
        with torch.cuda.stream(stream):
            A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
            codes, start, count = ctx.traceback(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs,
                                                stream=stream)
            res = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs, stream=stream)
        stream.synchronize()
    finally:
        ctx.set_option(key, old)
    c = codes.cpu().numpy().view(np.uint32)
    st, ct = start.cpu().numpy(), count.cpu().numpy()
    paths = [list(c[st[p]:st[p] + ct[p]]) for p in range(b.n_pairs)]
    check(b, paths, logan.results_to_numpy(res))


def _rle_np(ops: str) -> np.ndarray:
    """Run-length codes (len << 4 | op) of an 'M'/'I'/'D' string, vectorised."""
    if not ops:
        return np.zeros(0, np.uint32)
    a = np.frombuffer(ops.encode(), np.uint8)
    code = np.where(a == ord("M"), 0, np.where(a == ord("I"), 1, 2)).astype(np.uint32)
    heads = np.flatnonzero(np.concatenate([[True], code[1:] != code[:-1]]))
    runs = np.diff(np.concatenate([heads, [a.size]])).astype(np.uint32)
    return (runs << 4) | code[heads]


def test_bench_size_every_pair(ctx):
    """The benchmark's traced batch (the first 10,000 pairs of the
    100,000-pair lognormal batch, 2-bit packed): every pair's run-length
    codes equal the oracle's path (the oracle on all host cores, one pair
    per task), and every path spans its pair's coordinates."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    b = synth.lognormal_batch().subset(np.arange(10_000))
    paths, res = gpu_paths(ctx, b, packed2bit=True)
    assert np.all(res["status"] == 0)
    for p in range(b.n_pairs):
        cc = np.asarray(paths[p], dtype=np.uint32)
        n, op = cc >> 4, cc & 15
        assert np.all(op <= 2) and np.all(n > 0)
        assert int(n[op != 2].sum()) == int(res["endA"][p] - res["begA"][p]), p
        assert int(n[op != 1].sum()) == int(res["endB"][p] - res["begB"][p]), p

    def want(p):
        s = b.seeds[p]
        return _rle_np(oracle.pair_traceback(b.seqA(p), b.seqB(p), int(s["posA"]),
                                             int(s["posB"]), int(s["len"]), b.match,
                                             b.mismatch, b.gap, b.X))

    # ctypes releases the interpreter lock during each oracle call
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        wants = list(ex.map(want, range(b.n_pairs), chunksize=16))
    bad = [p for p in range(b.n_pairs)
           if not np.array_equal(np.asarray(paths[p], dtype=np.uint32), wants[p])]
    assert not bad, f"{len(bad)} paths differ from the oracle's, e.g. pairs {bad[:10]}"
