"""Affine-gap path (logan_extend_batch_affine) vs the affine CPU oracle,
bit-exact on every integer field."""
import numpy as np
import pytest

import oracle
from paper_2002_05200_gb300 import logan, synth
from tests.gpu_common import assert_same, run_oracle_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


def run_affine(ctx, b, go, ge, packed2bit=False):
    import torch
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=packed2bit)
    out = ctx.extend_affine(A, B, S, b.match, b.mismatch, go, ge, b.X, Xs)
    torch.cuda.synchronize()
    return logan.results_to_numpy(out)


def ref_affine(b, go, ge):
    return oracle.run_batch_affine(b, go, ge)[0]


@pytest.mark.parametrize("go,ge", [(-2, -1), (-5, -2), (0, -1), (-1, 0)])
def test_uniform_pairs(ctx, go, ge):
    b = synth.uniform_pairs(n_pairs=400)
    assert_same(run_affine(ctx, b, go, ge), ref_affine(b, go, ge), f"uniform {go},{ge}")


def test_lognormal_packed(ctx):
    b = synth.lognormal_batch(n_pairs=300)
    assert_same(run_affine(ctx, b, -2, -1, packed2bit=True), ref_affine(b, -2, -1), "lognormal")


def test_uneven_per_pair_x(ctx):
    b = synth.uneven_batch(n_pairs=200, max_len=30_000, seed=71)
    assert_same(run_affine(ctx, b, -3, -1, packed2bit=True), ref_affine(b, -3, -1), "uneven")


@pytest.mark.parametrize("seed", range(3))
def test_tiny_edge_cases(ctx, seed):
    b = synth.tiny_pairs(3000, 40, seed=seed)
    assert_same(run_affine(ctx, b, -2, -1), ref_affine(b, -2, -1), "tiny")
    assert_same(run_affine(ctx, b, -4, 0, packed2bit=True), ref_affine(b, -4, 0), "tiny packed")


@pytest.mark.parametrize("scheme", [(2, -3, -4, -2), (1, -1, -1, -1), (5, -4, -10, -1),
                                    (1000, -1000, -1000, -1000)])
def test_scoring_schemes(ctx, scheme):
    match, mismatch, go, ge = scheme
    b = synth.uniform_pairs(n_pairs=200)
    b.match, b.mismatch = match, mismatch
    assert_same(run_affine(ctx, b, go, ge), ref_affine(b, go, ge), str(scheme))


def test_zero_open_equals_linear_path(ctx):
    import torch
    b = synth.uneven_batch(n_pairs=150, max_len=8_000, seed=72)
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
    lin = ctx.extend(A, B, S, b.match, b.mismatch, -2, b.X, Xs)
    aff = ctx.extend_affine(A, B, S, b.match, b.mismatch, 0, -2, b.X, Xs)
    torch.cuda.synchronize()
    assert np.array_equal(logan.results_to_numpy(lin), logan.results_to_numpy(aff))


def test_wide_bands_continue_in_the_ring(ctx):
    # unpruned: a side's widest anti-diagonal has min(m, n) + 1 cells; bands
    # above the 512-row register window continue in the device-memory ring
    # and every pair is exact
    b = synth.tiny_pairs(60, 1500, seed=8, X_choices=(200_000,))
    g = run_affine(ctx, b, -2, -1)
    s = b.seeds
    lA, lB = b.lenA[s["idxA"]].astype(np.int64), b.lenB[s["idxB"]].astype(np.int64)
    left = np.minimum(s["posA"], s["posB"]).astype(np.int64) + 1
    right = np.minimum(lA - s["posA"] - s["len"], lB - s["posB"] - s["len"]) + 1
    wide = np.maximum(left, right) > 512
    assert wide.any() and (~wide).any()
    assert_same(g, ref_affine(b, -2, -1), "bands up to 1500 rows")


def test_x_beyond_key_range_is_exact(ctx):
    # X too large for the register windows' keys: the ring kernel runs them
    b = synth.uniform_pairs(n_pairs=20)
    b.Xs = np.full(b.n_pairs, (1 << 20), dtype=np.int32)
    b.Xs[::2] = 50
    assert_same(run_affine(ctx, b, -2, -1), ref_affine(b, -2, -1), "X = 2^20 and 50")


def test_uneven_pairs_x500_no_erange(ctx):
    # the uneven length mixture (up to 200 kbp here) at X = 500 with affine
    # gaps: bands beyond 512 rows included, zero LOGAN_ERANGE, every pair
    # exact
    b = synth.uneven_batch(n_pairs=120, max_len=200_000, seed=31, X_choices=(500,))
    g = run_affine(ctx, b, -2, -1, packed2bit=True)
    assert np.all(g["status"] == logan.OK)
    assert_same(g, run_oracle_all(b, run=lambda sub: ref_affine(sub, -2, -1)),
                "uneven, X = 500")


def test_band_of_65535_rows_and_beyond(ctx):
    # identical sequences at X = 2^20 leave the band unpruned: 50,000 letters
    # stay inside the ring's 65,536 rows (closed form: L * match at (L, L)
    # over all (L+1)^2 - 1 cells); 66,000 letters outgrow it -> LOGAN_ERANGE
    # for that pair; the other pairs are exact
    rng = np.random.default_rng(12)
    L0, L1 = 50_000, 66_000
    s0 = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, L0)]
    s1 = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, L1)]
    base = synth.uniform_pairs(n_pairs=8, length=1200, seed=13)
    poolA = np.concatenate([s0, s1, base.poolA])
    poolB = np.concatenate([s0, s1, base.poolB])
    offA = np.concatenate([[0, L0], base.offA.astype(np.int64) + L0 + L1]).astype(np.uint64)
    offB = np.concatenate([[0, L0], base.offB.astype(np.int64) + L0 + L1]).astype(np.uint64)
    lenA = np.concatenate([[L0, L1], base.lenA]).astype(np.uint32)
    lenB = np.concatenate([[L0, L1], base.lenB]).astype(np.uint32)
    seeds = np.zeros(10, dtype=base.seeds.dtype)
    seeds[1] = (1, 1, 0, 0, 0)
    seeds[2:] = base.seeds
    seeds["idxA"][2:] += 2
    seeds["idxB"][2:] += 2
    Xs = np.full(10, 50, np.int32)
    Xs[:2] = 1 << 20
    b = synth.Batch("ring_limit", poolA, offA, lenA, poolB, offB, lenB, seeds, 50, Xs)
    g = run_affine(ctx, b, -2, -1)
    assert g["status"][0] == logan.OK
    assert (g["score"][0], g["left"][0], g["right"][0]) == (L0 * b.match, 0, L0 * b.match)
    assert (g["begA"][0], g["endA"][0], g["begB"][0], g["endB"][0]) == (0, L0, 0, L0)
    assert g["cells"][0] == (L0 + 1) ** 2 - 1
    assert g["status"][1] == logan.ERANGE
    assert_same(g[2:], ref_affine(b.subset(np.arange(2, 10)), -2, -1), "the other pairs")


def test_argument_errors(ctx):
    b = synth.uniform_pairs(n_pairs=4)
    A, B, S, _ = logan.batch_to_device(b)
    for args in ((1, -1, 1, -1, 5), (1, -1, -1, 1, 5), (1, -1, -1001, -1, 5), (1, 2, -1, -1, 5),
                 (1, -1, -1, -1, -1)):
        with pytest.raises(logan.LoganError) as e:
            ctx.extend_affine(A, B, S, *args)
        assert e.value.code == logan.EINVAL


def test_lognormal_100k_every_pair(ctx):
    # the affine bench workload at full size, in its launch configuration,
    # every pair against the affine oracle
    b = synth.lognormal_batch()
    g = run_affine(ctx, b, -2, -1, packed2bit=True)
    ok = g["status"] == logan.OK
    assert np.all(ok)
    assert_same(g, run_oracle_all(b, run=lambda sub: ref_affine(sub, -2, -1)),
                "lognormal 100K, every pair")
    k = b.seeds["len"].astype(np.int64)
    assert np.array_equal(g["score"][ok].astype(np.int64),
                          (g["left"].astype(np.int64) + k * b.match + g["right"])[ok])


@pytest.mark.parametrize("scheme", [(1, -1, -2, -1, 100), (2, -3, -5, -2, 60), (1, -1, 0, -1, 200),
                                    (1, -2, -30, -10, 40)])
def test_packed_levels_equal_32bit_and_oracle(ctx, scheme):
    # the packed 16-bit windows (128, 256, 512 rows) and the 32-bit ones give
    # the oracle's results; a call reports which levels ran packed
    match, mismatch, go, ge, X = scheme
    b = synth.lognormal_batch(n_pairs=300, median=6000, lo=1000, hi=20_000, seed=77, X=X)
    b.match, b.mismatch = match, mismatch
    ref = ref_affine(b, go, ge)
    try:
        ctx.set_option(logan.OPT_PACKED16, 1)
        g16 = run_affine(ctx, b, go, ge, packed2bit=True)
        packed = ctx.get_option(logan.OPT_AFFINE_PACKED)
        ctx.set_option(logan.OPT_PACKED16, 0)
        g32 = run_affine(ctx, b, go, ge, packed2bit=True)
        assert ctx.get_option(logan.OPT_AFFINE_PACKED) == 0
    finally:
        ctx.set_option(logan.OPT_PACKED16, 1)
    assert packed == 0b1110, packed  # levels 1-3 (128, 256, 512 rows)
    assert_same(g16, ref, f"packed {scheme}")
    assert_same(g32, ref, f"32-bit {scheme}")


def test_packed_levels_per_pair_x_and_bounds(ctx):
    # per-pair X up to 500: only the levels whose X classes fit stay packed;
    # scores too large for 16 bits keep every level 32-bit
    b = synth.uneven_batch(n_pairs=150, max_len=20_000, seed=78)
    g = run_affine(ctx, b, -2, -1, packed2bit=True)
    packed = ctx.get_option(logan.OPT_AFFINE_PACKED)
    assert packed & 0b0010 and not packed & 0b1000, packed
    assert_same(g, ref_affine(b, -2, -1), "uneven, per-pair X")
    b2 = synth.lognormal_batch(n_pairs=60, seed=79, X=100)
    b2.match, b2.mismatch = 300, -300
    g2 = run_affine(ctx, b2, -300, -300, packed2bit=True)
    assert ctx.get_option(logan.OPT_AFFINE_PACKED) == 0
    assert_same(g2, ref_affine(b2, -300, -300), "large scores")
