"""logan_extend_batch_noalloc: the batch call for callers that cannot allocate
device memory (their GPU memory belongs to another allocator, or their loop
must not call cudaMalloc/cudaFree, which can synchronise the device).

The entry point is called through the C ABI with ctypes and must give
exactly the results of logan_extend_batch (integer outputs: bit-exact) on
two calls in a row, which share the library's static scratch array; one
case is also compared with the CPU oracle directly.  This file is collected
last so that a run stopping at the first failure has run every other test
first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2002_05200_gb300 import logan, synth
from tests.gpu_common import assert_same

pytestmark = pytest.mark.gpu


def _noalloc():
    fn = logan.lib().logan_extend_batch_noalloc
    p = ctypes.c_void_p
    fn.argtypes = [p, ctypes.POINTER(logan.SeqsT), ctypes.POINTER(logan.SeqsT), p,
                   ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_int32, p, p, p]
    fn.restype = ctypes.c_int
    return fn


def _call(ctx, A, B, S, b, Xs, out, stream):
    ca, cb = A.c(), B.c()
    return _noalloc()(ctx._h, ctypes.byref(ca), ctypes.byref(cb), S.data_ptr(), S.shape[0],
                      b.match, b.mismatch, b.gap, b.X,
                      Xs.data_ptr() if Xs is not None else None, out.data_ptr(),
                      ctypes.c_void_p(stream.cuda_stream))


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["uniform_ascii", "lognormal_packed", "uneven_per_pair_x"])
def test_noalloc_matches_workspace_call_twice(ctx, name):
    import torch
    if name == "uniform_ascii":
        b, packed = synth.uniform_pairs(n_pairs=400), False
    elif name == "lognormal_packed":
        b, packed = synth.lognormal_batch(n_pairs=300), True
    else:
        b, packed = synth.uneven_batch(n_pairs=150, max_len=30_000), True
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=packed)
    stream = torch.cuda.current_stream()
    ref = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
    torch.cuda.synchronize()
    ref = logan.results_to_numpy(ref)
    assert np.all(ref["status"] == logan.OK)
    for call in range(2):
        out = torch.full((b.n_pairs, 10), -7, dtype=torch.int32, device="cuda")
        rc = _call(ctx, A, B, S, b, Xs, out, stream)
        assert rc == logan.OK, logan.strerror(rc)
        torch.cuda.synchronize()
        got = logan.results_to_numpy(out)
        for f in logan.RESULT_DTYPE.names:
            assert np.array_equal(got[f], ref[f]), (name, call, f)
    if name == "lognormal_packed":
        # and against the oracle itself, every pair
        assert_same(got, oracle.run_batch(b.subset(np.arange(b.n_pairs)))[0], name)


def _wide_band_batch():
    """Two pairs of identical 20 kbp sequences seeded at the midpoint, at
    X = 9000 (band about 2X/3 = 6000 rows: wider than the no-alloc window of
    4096 rows) and at X = 50, plus 30 ordinary pairs at X = 50."""
    rng = np.random.default_rng(5)
    seq = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 20_000)]
    base = synth.uniform_pairs(n_pairs=30, length=1500, seed=6)
    poolA = np.concatenate([seq, seq, base.poolA])
    poolB = np.concatenate([seq, seq, base.poolB])
    offA = np.concatenate([[0, 20_000], base.offA.astype(np.int64) + 40_000]).astype(np.uint64)
    offB = np.concatenate([[0, 20_000], base.offB.astype(np.int64) + 40_000]).astype(np.uint64)
    lenA = np.concatenate([[20_000, 20_000], base.lenA]).astype(np.uint32)
    lenB = np.concatenate([[20_000, 20_000], base.lenB]).astype(np.uint32)
    seeds = np.zeros(32, dtype=base.seeds.dtype)
    seeds[0] = (0, 0, 9_991, 9_991, 17)
    seeds[1] = (1, 1, 9_991, 9_991, 17)
    seeds[2:] = base.seeds
    seeds["idxA"][2:] += 2
    seeds["idxB"][2:] += 2
    Xs = np.full(32, 50, np.int32)
    Xs[0] = 9000
    return synth.Batch("wide_band", poolA, offA, lenA, poolB, offB, lenB, seeds, 50, Xs)


def test_noalloc_wide_band_erange(ctx):
    # the no-alloc fallback window is 4096 rows where the workspace call's is
    # 65,536: the 6000-row band gets LOGAN_ERANGE, every other pair the
    # workspace call's (and the oracle's) result
    import torch
    b = _wide_band_batch()
    A, B, S, Xs = logan.batch_to_device(b)
    ref = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
    torch.cuda.synchronize()
    ref = logan.results_to_numpy(ref)
    assert np.all(ref["status"] == logan.OK)
    assert_same(ref, oracle.run_batch(b)[0], "wide band, workspace call")
    assert int(ref["score"][0]) == 20_000  # identical sequences: length x match
    out = torch.zeros((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    rc = _call(ctx, A, B, S, b, Xs, out, torch.cuda.current_stream())
    assert rc == logan.OK, logan.strerror(rc)
    torch.cuda.synchronize()
    got = logan.results_to_numpy(out)
    assert got["status"][0] == logan.ERANGE
    for f in logan.RESULT_DTYPE.names:
        assert np.array_equal(got[f][1:], ref[f][1:]), f


def test_noalloc_allocates_nothing(ctx):
    # after a first call (which looks up the scratch address), a call and its
    # completion leave the device's free memory and torch's pool unchanged
    import torch
    b = synth.lognormal_batch(n_pairs=200, seed=9)
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
    out = torch.zeros((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    assert _call(ctx, A, B, S, b, Xs, out, stream) == logan.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    assert _call(ctx, A, B, S, b, Xs, out, stream) == logan.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def _set_custom_options(ctx):
    # values other than the no-alloc call's own (and, but for the ring, other
    # than the defaults)
    opts = {logan.OPT_RING_CAP: 16, logan.OPT_GRAPHS: 1, logan.OPT_MIGRATION_MB: 8,
            logan.OPT_CONCURRENT: 0}
    for k, v in opts.items():
        ctx.set_option(k, v)
    return opts


def _restore_defaults(ctx):
    ctx.set_option(logan.OPT_GRAPHS, 0)
    ctx.set_option(logan.OPT_MIGRATION_MB, 64)
    ctx.set_option(logan.OPT_CONCURRENT, 1)


def test_noalloc_rejects_oversized_batch(ctx):
    import torch
    # 200,000 pairs need more scratch than the static array holds
    opts = _set_custom_options(ctx)
    b = synth.tiny_pairs(200_000, 4, seed=3)
    A, B, S, Xs = logan.batch_to_device(b)
    out = torch.zeros((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    rc = _call(ctx, A, B, S, b, Xs, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert rc == logan.ENOMEM
    assert int(out.abs().sum().item()) == 0  # nothing was launched
    # the rejection restores the caller's options too
    for k, v in opts.items():
        assert ctx.get_option(k) == v, k
    _restore_defaults(ctx)


def test_noalloc_restores_context_options(ctx):
    import torch
    opts = _set_custom_options(ctx)
    b = synth.uniform_pairs(n_pairs=32, length=300)
    A, B, S, Xs = logan.batch_to_device(b)
    out = torch.zeros((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    assert _call(ctx, A, B, S, b, Xs, out, torch.cuda.current_stream()) == logan.OK
    torch.cuda.synchronize()
    for k, v in opts.items():
        assert ctx.get_option(k) == v, k
    _restore_defaults(ctx)
