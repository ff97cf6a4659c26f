"""Each benchmark configuration at full size, in the launch configuration the
benchmark times (persistent, 2-bit packed except the ASCII 1,000-pair case),
compared with the oracle on EVERY pair, bit-exactly on status, score, left,
right, the four coordinates and cells:
  * 1,000 uniform pairs, the 100,000-pair lognormal batch, the 20,000-pair
    uneven batch and every serving request: the oracle runs here, on all
    host cores;
  * the 1,000,000-candidate overlap workload (about 2.5e12 oracle cell
    updates): per-chunk digests of the oracle's results, stored in
    tests/golden/overlap_batch_1m.sha256 by tests/golden/overlap_digests.py,
    are compared with the same digests of the GPU's results.
Every pair is also checked against what holds at any size (score = left +
seed + right, coordinates inside the sequences, persistent == one-launch
form)."""
import numpy as np
import pytest

from paper_2002_05200_gb300 import logan, synth
from tests.golden import overlap_digests as od
from tests.gpu_common import assert_same, run_gpu, run_oracle, run_oracle_all

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


def test_lognormal_100k_every_pair(ctx):
    b = synth.lognormal_batch()
    g = run_gpu(ctx, b, packed2bit=True)
    _properties(b, g)
    assert np.array_equal(run_gpu(ctx, b, packed2bit=True, plain=True), g)
    assert_same(g, run_oracle_all(b), "lognormal_batch, all 100,000 pairs")


def test_uneven_20k_every_pair(ctx):
    b = synth.uneven_batch()
    g = run_gpu(ctx, b, packed2bit=True)
    _properties(b, g)
    assert np.array_equal(run_gpu(ctx, b, packed2bit=True, plain=True), g)
    # the longest class (200 kbp - 1 Mbp) at every X, X = 500 included
    cls = b.meta["length_class"]
    assert np.any((cls == 3) & (b.Xs == 500))
    assert_same(g, run_oracle_all(b), "uneven_batch, all 20,000 pairs")


def test_overlap_1m_every_pair_digests(ctx):
    b = synth.overlap_batch()
    inp, chunk, want, want_cells = od.read_digest_file()
    assert chunk == od.CHUNK
    assert od.input_digest(b) == inp, \
        "the generator made other inputs than the ones the stored digests were taken from"
    g = run_gpu(ctx, b, packed2bit=True)
    _properties(b, g)
    arr = od.canonical(g, g["status"] == logan.OK)
    got = od.chunk_digests(arr)
    assert len(got) == len(want)
    bad = [k for k in range(len(got)) if got[k] != want[k]]
    if bad:
        # name the pairs: rerun the oracle on the first chunk that differs
        k = bad[0]
        idx = np.arange(k * chunk, min((k + 1) * chunk, b.n_pairs))
        assert_same(g[idx], run_oracle(b.subset(idx)), f"overlap_batch chunk {k}")
        raise AssertionError(f"chunks {bad[:10]} differ from the oracle's digests")
    cells = arr[:, od.FIELDS.index("cells")]
    assert [int(cells[c0:c0 + chunk].sum()) for c0 in range(0, b.n_pairs, chunk)] == want_cells
    # true overlaps extend along the overlap; spurious pairs stop earlier
    t = np.flatnonzero(b.meta["is_true"])
    f = np.flatnonzero(~b.meta["is_true"])
    assert np.median(g["score"][t]) > 2 * np.median(g["score"][f])


def test_serving_requests_full_mixture(ctx):
    # requests of up to 10,000 pairs with the uneven length mixture, X = 50;
    # every pair of every request against the oracle
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
    assert sum(b.n_pairs for b in reqs) > 5000
    for k, (b, h) in enumerate(zip(reqs, hosts)):
        g = h.result_array()
        _properties(b, g)
        assert_same(g, run_oracle_all(b), f"serving request {k} ({b.n_pairs} pairs)")
