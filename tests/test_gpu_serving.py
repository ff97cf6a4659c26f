"""Serving loop (logan_server_*): continuous batching over a device-memory
budget.  Each request's results must be the same alone and in the mix."""
import numpy as np
import pytest

from paper_2002_05200_gb300 import logan, synth
from tests.gpu_common import assert_same, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


def _requests(n, seed, max_pairs=300, max_len=20_000):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        size = int(np.exp(rng.uniform(0, np.log(max_pairs))))
        b = synth.uneven_batch(max(1, size), seed=int(rng.integers(1 << 30)), max_len=max_len,
                               X_choices=(50,))
        out.append(b)
    return out


def _alone(ctx, b):
    import torch
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
    out = ctx.extend(A, B, S, b.match, b.mismatch, b.gap, b.X, Xs)
    torch.cuda.synchronize()
    return logan.results_to_numpy(out)


def test_results_identical_alone_and_in_mix(ctx):
    reqs = _requests(16, seed=1)
    alone = [_alone(ctx, b) for b in reqs]
    # spot-check the alone results against the oracle
    for b, a in list(zip(reqs, alone))[:3]:
        assert_same(a, run_oracle(b), "alone")
    hosts = [logan.HostRequest(b) for b in reqs]
    srv = logan.Server(ctx, budget_bytes=1 << 30, max_inflight=4)
    try:
        tickets = [srv.submit(h) for h in hosts]
        for t in tickets:
            st, lat = srv.wait(t, timeout_ms=120_000)
            assert st == logan.OK and lat > 0
        stats = srv.stats()
        assert stats["completed"] == len(reqs) and stats["used_bytes"] == 0
        assert stats["peak_bytes"] > 0
    finally:
        srv.close()
    for h, a in zip(hosts, alone):
        got = h.result_array()
        for f in logan.RESULT_DTYPE.names:
            assert np.array_equal(got[f], a[f]), f


def test_budget_admission_serialises_but_completes(ctx):
    # a budget that fits one request at a time: every request still completes
    reqs = _requests(5, seed=2, max_pairs=200)
    hosts = [logan.HostRequest(b) for b in reqs]
    need = max(ctx.workspace_size(*logan.batch_to_device(b, packed2bit=True)[:2], b.n_pairs)
               for b in reqs)
    srv = logan.Server(ctx, budget_bytes=need + (64 << 20), max_inflight=4)
    try:
        ts = [srv.submit(h) for h in hosts]
        for t in ts:
            assert srv.wait(t, 120_000)[0] == logan.OK
    finally:
        srv.close()
    for h, b in zip(hosts, reqs):
        assert_same(h.result_array(), run_oracle(b), "budget")


def test_oversized_request_rejected(ctx):
    b = synth.uniform_pairs(n_pairs=200, length=2000)
    srv = logan.Server(ctx, budget_bytes=1 << 20, max_inflight=2)
    try:
        with pytest.raises(logan.LoganError) as e:
            srv.submit(logan.HostRequest(b))
        assert e.value.code == logan.ENOMEM
    finally:
        srv.close()


def test_queue_limit_cancel_and_bounded_wait(ctx):
    big = synth.uneven_batch(600, seed=5, max_len=40_000, X_choices=(100,))
    small = synth.uniform_pairs(n_pairs=8, length=500)
    srv = logan.Server(ctx, budget_bytes=2 << 30, max_inflight=1, max_queued=2)
    try:
        t0 = srv.submit(logan.HostRequest(big))
        t1 = srv.submit(logan.HostRequest(small))
        t2 = srv.submit(logan.HostRequest(small))
        # one slot: t1 waits behind the big request, so a zero wait times out
        with pytest.raises(logan.LoganError) as e:
            srv.wait(t1, timeout_ms=0)
        assert e.value.code == logan.ETIMEOUT
        codes = []
        for _ in range(3):
            try:
                srv.submit(logan.HostRequest(small))
                codes.append(logan.OK)
            except logan.LoganError as err:
                codes.append(err.code)
        assert logan.EAGAIN in codes
        srv.cancel(t2)
        assert srv.wait(t2, 120_000)[0] == logan.ECANCELED
        assert srv.wait(t0, 120_000)[0] == logan.OK
        assert srv.wait(t1, 120_000)[0] == logan.OK
        with pytest.raises(logan.LoganError) as e:
            srv.poll(t1)
        assert e.value.code == logan.ENOTFOUND
    finally:
        srv.close()


@pytest.mark.parametrize("pin", [False, True])
def test_pageable_and_pinned_requests(ctx, pin):
    # pageable buffers go through the server's pinned staging arena, pinned
    # ones are copied directly: the results are the same either way, and the
    # context's options come back when the server is destroyed
    reqs = _requests(8, seed=7)
    alone = [_alone(ctx, b) for b in reqs]
    ctx.set_option(logan.OPT_CONCURRENT, 1)
    hosts = [logan.HostRequest(b, pin=pin) for b in reqs]
    srv = logan.Server(ctx, budget_bytes=1 << 30, max_inflight=4)
    try:
        assert ctx.get_option(logan.OPT_CONCURRENT) == 0
        assert ctx.get_option(logan.OPT_LONG_ITEM) in (65536, -1)
        tickets = [srv.submit(h) for h in hosts]
        for t in tickets:
            st, _ = srv.wait(t, timeout_ms=120_000)
            assert st == logan.OK
    finally:
        srv.close()
    assert ctx.get_option(logan.OPT_CONCURRENT) == 1
    assert ctx.get_option(logan.OPT_LONG_ITEM) == -2
    for h, a in zip(hosts, alone):
        np.testing.assert_array_equal(h.result_array(), a)
