"""logan_extend_batch_noalloc: the batch call for callers that cannot allocate
device memory (their GPU memory belongs to another allocator, or their loop
must not call cudaMalloc/cudaFree, which can synchronise the device).

The entry point is called through the C ABI with ctypes and must give
exactly the results of logan_extend_batch (integer outputs: bit-exact) on
two calls in a row, which share the library's static scratch array.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2002_05200_gb300 import logan, synth

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


def test_noalloc_rejects_oversized_batch(ctx):
    import torch
    # 200,000 pairs need more scratch than the static array holds
    b = synth.tiny_pairs(200_000, 4, seed=3)
    A, B, S, Xs = logan.batch_to_device(b)
    out = torch.zeros((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    rc = _call(ctx, A, B, S, b, Xs, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert rc == logan.ENOMEM
    assert int(out.abs().sum().item()) == 0  # nothing was launched


def test_noalloc_restores_context_options(ctx):
    import torch
    ctx.set_option(logan.OPT_RING_CAP, 16)
    ctx.set_option(logan.OPT_GRAPHS, 1)
    b = synth.uniform_pairs(n_pairs=32, length=300)
    A, B, S, Xs = logan.batch_to_device(b)
    out = torch.zeros((b.n_pairs, 10), dtype=torch.int32, device="cuda")
    assert _call(ctx, A, B, S, b, Xs, out, torch.cuda.current_stream()) == logan.OK
    torch.cuda.synchronize()
    assert ctx.get_option(logan.OPT_RING_CAP) == 16
    assert ctx.get_option(logan.OPT_GRAPHS) == 1
    ctx.set_option(logan.OPT_GRAPHS, 0)
