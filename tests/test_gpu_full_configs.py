"""Each benchmark configuration at full size, in the launch configuration the
benchmark times (persistent, 2-bit packed except the ASCII 1,000-pair case):
a seeded sample of pairs is compared bit-exactly with the oracle, and every
pair is checked against what holds at any size (status, score = left + seed
+ right, coordinates inside the sequences, persistent == one-launch form)."""
import numpy as np
import pytest

from paper_2002_05200_gb300 import logan, synth
from tests.gpu_common import assert_same, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


def _properties(b, g):
    s = b.seeds
    assert np.all(g["status"] == logan.OK)
    lA = b.lenA[s["idxA"]].astype(np.int64)
    lB = b.lenB[s["idxB"]].astype(np.int64)
    k = s["len"].astype(np.int64)
    posA, posB = s["posA"].astype(np.int64), s["posB"].astype(np.int64)
    # exact seeds score k * match; both extensions score at least 0
    assert np.all(g["left"] >= 0) and np.all(g["right"] >= 0)
    assert np.array_equal(g["score"].astype(np.int64),
                          g["left"].astype(np.int64) + k * b.match + g["right"])
    bA, bB = g["begA"].astype(np.int64), g["begB"].astype(np.int64)
    eA, eB = g["endA"].astype(np.int64), g["endB"].astype(np.int64)
    assert np.all((0 <= bA) & (bA <= posA) & (0 <= bB) & (bB <= posB))
    assert np.all((posA + k <= eA) & (eA <= lA) & (posB + k <= eB) & (eB <= lB))
    # an extension that scores > 0 computed at least that many cells
    assert np.all(g["cells"].astype(np.int64) >= g["left"] + g["right"])


def _sample_check(b, g, idx):
    idx = np.unique(np.asarray(idx))
    ref = run_oracle(b.subset(idx))
    assert_same(g[idx], ref, f"{b.name} sample of {idx.size}")


def test_plain_1000_pairs_ascii(ctx):
    b = synth.uniform_pairs()
    g = run_gpu(ctx, b)
    _properties(b, g)
    assert_same(g, run_oracle(b), "all 1,000 pairs")
    assert np.array_equal(run_gpu(ctx, b, plain=True), g)


def test_lognormal_100k_sampled(ctx):
    b = synth.lognormal_batch()
    g = run_gpu(ctx, b, packed2bit=True)
    _properties(b, g)
    rng = np.random.default_rng(101)
    _sample_check(b, g, rng.choice(b.n_pairs, 400, replace=False))
    assert np.array_equal(run_gpu(ctx, b, packed2bit=True, plain=True), g)


def test_uneven_20k_sampled(ctx):
    b = synth.uneven_batch()
    g = run_gpu(ctx, b, packed2bit=True)
    _properties(b, g)
    rng = np.random.default_rng(102)
    cls = b.meta["length_class"]
    pick = [rng.choice(np.flatnonzero(cls <= 1), 300, replace=False),
            rng.choice(np.flatnonzero(cls == 2), 6, replace=False)]
    # two of the longest class (200 kbp-1 Mbp), at X <= 100 so the oracle
    # finishes in seconds
    longx = np.flatnonzero((cls == 3) & (b.Xs <= 100))
    pick.append(rng.choice(longx, 2, replace=False))
    _sample_check(b, g, np.concatenate(pick))
    assert np.array_equal(run_gpu(ctx, b, packed2bit=True, plain=True), g)


def test_overlap_1m_sampled(ctx):
    b = synth.overlap_batch()
    g = run_gpu(ctx, b, packed2bit=True)
    _properties(b, g)
    rng = np.random.default_rng(103)
    t = np.flatnonzero(b.meta["is_true"])
    f = np.flatnonzero(~b.meta["is_true"])
    _sample_check(b, g, np.concatenate([rng.choice(t, 150, replace=False),
                                        rng.choice(f, 150, replace=False)]))
    # true overlaps extend along the overlap; spurious pairs stop earlier
    assert np.median(g["score"][t]) > 2 * np.median(g["score"][f])


def test_serving_requests_full_mixture(ctx):
    # requests of up to 10,000 pairs with the uneven length mixture, X = 50
    reqs = [b for _, b in synth.serving_requests(6, 100.0, seed=11)]
    hosts = [logan.HostRequest(b) for b in reqs]
    srv = logan.Server(ctx, budget_bytes=8 << 30, max_inflight=4)
    try:
        tickets = [srv.submit(h) for h in hosts]
        for tk in tickets:
            st, _ = srv.wait(tk, timeout_ms=600_000)
            assert st == logan.OK
    finally:
        srv.close()
    rng = np.random.default_rng(104)
    for b, h in zip(reqs, hosts):
        g = h.result_array()
        _properties(b, g)
        cls = b.meta["length_class"]
        short = np.flatnonzero(cls <= 1)
        if short.size:
            _sample_check(b, g, rng.choice(short, min(40, short.size), replace=False))
