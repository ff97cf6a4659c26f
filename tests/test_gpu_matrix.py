"""Substitution-matrix path (logan_extend_batch_matrix) vs the matrix CPU
oracle, bit-exact on status, score, left, right, the four coordinates and
cells: BLOSUM62 protein pairs, the DNA match / mismatch matrix against the
affine DNA path, linear gaps, per-pair X, edge cases, invalid inputs and
the ring limit."""
import numpy as np
import pytest

import oracle
from paper_2002_05200_gb300 import logan, synth
from tests.gpu_common import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = logan.Context(0)
    yield c
    c.close()


def run_matrix(ctx, b, M, go, ge):
    import torch
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=False)
    out = ctx.extend_matrix(A, B, S, M, go, ge, b.X, Xs)
    torch.cuda.synchronize()
    return logan.results_to_numpy(out)


def ascii_to_codes(b):
    lut = np.zeros(256, np.uint8)
    lut[np.frombuffer(b"ACGT", np.uint8)] = np.arange(4, dtype=np.uint8)
    c = synth.Batch(b.name + "[codes]", lut[b.poolA], b.offA, b.lenA, lut[b.poolB], b.offB,
                    b.lenB, b.seeds, b.X, b.Xs, b.match, b.mismatch, b.gap)
    return c


@pytest.mark.parametrize("go,ge", [(-11, -1), (0, -4), (-5, -2)])
def test_blosum62_protein_pairs(ctx, go, ge):
    b = synth.protein_pairs(600, lo=50, hi=1500, seed=4)
    M = synth.BLOSUM62
    g = run_matrix(ctx, b, M, go, ge)
    assert_same(g, oracle.run_batch_matrix(b, M, go, ge)[0], f"BLOSUM62 {go},{ge}")


def test_per_pair_x_and_tiny_edge_cases(ctx):
    rng = np.random.default_rng(9)
    M = rng.integers(-5, 6, size=(20, 20)).astype(np.int32)
    b = synth.tiny_pairs(2000, 40, seed=10)
    # letters of a 20-letter alphabet in place of ACGT
    b.poolA = rng.integers(0, 20, size=b.poolA.size).astype(np.uint8)
    b.poolB = rng.integers(0, 20, size=b.poolB.size).astype(np.uint8)
    assert_same(run_matrix(ctx, b, M, -3, -1), oracle.run_batch_matrix(b, M, -3, -1)[0],
                "tiny, per-pair X")


@pytest.mark.parametrize("go,ge", [(-2, -1), (0, -1)])
def test_dna_matrix_equals_affine_path(ctx, go, ge):
    b = synth.uneven_batch(n_pairs=100, max_len=20_000, seed=14)
    M = synth.dna_matrix(b.match, b.mismatch)
    g = run_matrix(ctx, ascii_to_codes(b), M, go, ge)
    assert_same(g, oracle.run_batch_affine(b, go, ge)[0], "DNA matrix vs affine oracle")
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=True)
    import torch
    aff = ctx.extend_affine(A, B, S, b.match, b.mismatch, go, ge, b.X, Xs)
    torch.cuda.synchronize()
    assert np.array_equal(logan.results_to_numpy(aff), g)


def test_wide_bands_escalate_through_every_window(ctx):
    # unpruned bands up to 1500 rows: each register window (64, 128, 256, 512
    # rows) hands its overflows to the next, the widest to the ring
    rng = np.random.default_rng(17)
    M = rng.integers(-3, 4, size=(12, 12)).astype(np.int32)
    b = synth.tiny_pairs(40, 1500, seed=18, X_choices=(100_000,))
    b.poolA = rng.integers(0, 12, size=b.poolA.size).astype(np.uint8)
    b.poolB = rng.integers(0, 12, size=b.poolB.size).astype(np.uint8)
    assert_same(run_matrix(ctx, b, M, -2, -1), oracle.run_batch_matrix(b, M, -2, -1)[0],
                "bands up to 1500 rows")


def test_invalid_inputs(ctx):
    import torch
    b = synth.protein_pairs(40, lo=30, hi=200, seed=5)
    M = synth.BLOSUM62
    b.poolB = b.poolB.copy()
    bad_seq = 3
    b.poolB[b.offB[bad_seq]] = 25  # a code outside the 20-letter alphabet
    g = run_matrix(ctx, b, M, -11, -1)
    ref = oracle.run_batch_matrix(b, M, -11, -1)[0]
    assert g["status"][bad_seq] == logan.EINVAL and ref["status"][bad_seq] == oracle.INVALID
    assert_same(g, ref, "one invalid pair")
    A, B, S, Xs = logan.batch_to_device(b, packed2bit=False)
    for args in ((np.zeros((33, 33), np.int32), -1, -1, 10), (M, 1, -1, 10), (M, -1, 1, 10),
                 (np.full((20, 20), 1001, np.int32), -1, -1, 10), (M, -1, -1, -5)):
        with pytest.raises(logan.LoganError) as e:
            ctx.extend_matrix(A, B, S, *args)
        assert e.value.code == logan.EINVAL
    torch.cuda.synchronize()


def test_band_beyond_the_ring_reports_erange(ctx):
    # an identical pair of 20,000 letters at X = 2^20: the unpruned band
    # outgrows the ring's 16,384 rows; the other pairs are exact
    rng = np.random.default_rng(15)
    seq = rng.integers(0, 20, size=20_000).astype(np.uint8)
    base = synth.protein_pairs(6, lo=100, hi=400, seed=16)
    poolA = np.concatenate([seq, base.poolA])
    poolB = np.concatenate([seq, base.poolB])
    offA = np.concatenate([[0], base.offA.astype(np.int64) + 20_000]).astype(np.uint64)
    offB = np.concatenate([[0], base.offB.astype(np.int64) + 20_000]).astype(np.uint64)
    lenA = np.concatenate([[20_000], base.lenA]).astype(np.uint32)
    lenB = np.concatenate([[20_000], base.lenB]).astype(np.uint32)
    seeds = np.zeros(7, dtype=base.seeds.dtype)
    seeds[1:] = base.seeds
    seeds["idxA"][1:] += 1
    seeds["idxB"][1:] += 1
    Xs = np.full(7, 60, np.int32)
    Xs[0] = 1 << 20
    b = synth.Batch("ring_limit", poolA, offA, lenA, poolB, offB, lenB, seeds, 60, Xs)
    M = synth.BLOSUM62
    g = run_matrix(ctx, b, M, -11, -1)
    assert g["status"][0] == logan.ERANGE
    ref = oracle.run_batch_matrix(b.subset(np.arange(1, 7)), M, -11, -1)[0]
    assert_same(g[1:], ref, "the other pairs")


@pytest.mark.parametrize("go,ge,X", [(-11, -1, 60), (-5, -2, 100), (0, -4, 30)])
def test_packed_windows_equal_32bit_and_oracle(ctx, go, ge, X):
    # the packed windows (128, 256, 512 rows: two cells per register, the
    # table as 16-bit entries) and the 32-bit ones give the oracle's results;
    # the call reports which windows ran packed
    b = synth.protein_pairs(500, lo=50, hi=2000, seed=21)
    b.X = X
    M = synth.BLOSUM62
    ref = oracle.run_batch_matrix(b, M, go, ge)[0]
    try:
        ctx.set_option(logan.OPT_PACKED16, 1)
        g16 = run_matrix(ctx, b, M, go, ge)
        packed = ctx.get_option(logan.OPT_MATRIX_PACKED)
        ctx.set_option(logan.OPT_PACKED16, 0)
        g32 = run_matrix(ctx, b, M, go, ge)
        assert ctx.get_option(logan.OPT_MATRIX_PACKED) == 0
    finally:
        ctx.set_option(logan.OPT_PACKED16, 1)
    assert packed == 0b1110, packed
    assert_same(g16, ref, f"packed {go},{ge},{X}")
    assert_same(g32, ref, f"32-bit {go},{ge},{X}")


def test_packed_windows_bounds(ctx):
    # a matrix whose range does not fit 16-bit keys keeps the 32-bit windows
    rng = np.random.default_rng(23)
    M = rng.integers(-900, 901, size=(20, 20)).astype(np.int32)
    b = synth.protein_pairs(60, lo=30, hi=300, seed=24)
    g = run_matrix(ctx, b, M, -50, -10)
    assert ctx.get_option(logan.OPT_MATRIX_PACKED) == 0
    assert_same(g, oracle.run_batch_matrix(b, M, -50, -10)[0], "wide matrix")
