"""Many-to-many overlap seeding on the GPU (logan_overlap_*) vs the numpy
oracle: candidates and their seeds exactly, the reverse-complement pool
base by base, and the extension + adaptive threshold on the candidates."""
import numpy as np
import pytest

import oracle
from oracle import overlap_oracle as ov
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


def read_set(n_reads, genome_len, mean_len, seed):
    """Reads as sequenced (both strands, 12 % errors) from the overlap
    generator: its packed pool holds read r at index 2r."""
    b = synth.overlap_batch(n_pairs=10, n_reads=n_reads, genome_len=genome_len,
                            mean_len=mean_len, seed=seed, min_len=200)
    idx = np.arange(0, 2 * n_reads, 2)
    ascii_reads = [b._seq(b.poolA, b.offA, b.lenA, i) for i in idx]
    return b.poolA, b.offA[idx].copy(), b.lenA[idx].copy(), ascii_reads


def device_reads(words, off, ln):
    return logan.pool_to_device(words, off, ln, True, (words.size - 1) * 16)


@pytest.mark.parametrize("k,fmin,fmax,mshared", [(15, 2, 4, 1), (13, 2, 6, 2), (17, 2, 2, 1),
                                                (11, 3, 8, 3)])
def test_candidates_match_oracle(ctx, k, fmin, fmax, mshared):
    words, off, ln, reads = read_set(150, 100_000, 2000, seed=7)
    A = device_reads(words, off, ln)
    got = ctx.overlap_candidates(A, k, fmin, fmax, mshared).cpu().numpy().view(np.uint32)
    want = ov.candidates(reads, k, fmin, fmax, mshared)
    assert got.shape[0] == want.size and want.size > 50
    for j, f in enumerate(ov.CAND_DTYPE.names):
        assert np.array_equal(got[:, j], want[f]), f


def test_pool_seeds_extension_and_threshold(ctx):
    import torch
    k = 15
    words, off, ln, reads = read_set(200, 120_000, 2500, seed=9)
    A = device_reads(words, off, ln)
    cands = ctx.overlap_candidates(A, k, 2, 4, 2)
    assert cands.shape[0] > 50
    B = ctx.overlap_pool(A)
    # the pool: reads, then their reverse complements
    pw = B.bases.cpu().numpy().view(np.uint32)
    po, pl = B.offsets.cpu().numpy().view(np.uint64), B.lengths.cpu().numpy().view(np.uint32)
    R = len(reads)
    for r in list(range(0, R, 17)) + [R - 1]:
        assert synth.unpack2bit(pw, int(po[r]), int(pl[r])).tobytes() == reads[r]
        assert synth.unpack2bit(pw, int(po[R + r]), int(pl[R + r])).tobytes() == \
            ov.revcomp(reads[r])
    # seeds
    seeds = ctx.overlap_seeds(cands, A, k)
    want = ov.seeds(cands.cpu().numpy().view(np.uint32).view(ov.CAND_DTYPE).reshape(-1),
                    [len(r) for r in reads], k)
    got = seeds.cpu().numpy().view(np.uint32)
    for j, f in enumerate(("idxA", "idxB", "posA", "posB", "len")):
        assert np.array_equal(got[:, j], want[f]), f
    # extension on the candidates against the oracle
    res = ctx.extend(A, B, seeds, 1, -1, -1, 50)
    keep = ctx.overlap_keep(res, seeds, A, B, 1, 4, 20)
    torch.cuda.synchronize()
    poolB = reads + [ov.revcomp(r) for r in reads]
    asc = np.frombuffer(b"".join(reads), np.uint8)
    ascB = np.frombuffer(b"".join(poolB), np.uint8)
    lA = np.array([len(r) for r in reads], np.uint32)
    lB = np.array([len(r) for r in poolB], np.uint32)
    b = synth.Batch("overlap_candidates", asc, synth._offsets(lA), lA, ascB, synth._offsets(lB),
                    lB, want, 50)
    ref = oracle.run_batch(b)[0]
    g = logan.results_to_numpy(res)
    assert_same(g, ref, "extension of the candidates")
    k_ref = ov.keep(ref["score"], lA[want["idxA"]], lB[want["idxB"]], want["posA"],
                    want["posB"], k, 1, 4, 20)
    assert np.array_equal(keep.cpu().numpy().astype(bool), k_ref)
    assert 0 < k_ref.sum() < k_ref.size


def test_full_read_set_properties(ctx):
    # the overlap workload's 50,000 reads (50 Mbp genome): candidates are
    # unique, ordered, above the hit minimum, their seed k-mers agree, and
    # every pair of reads sharing >= 4 kbp of genome on the same strand
    # relation is found
    k, mshared = 17, 4
    b = synth.overlap_batch(n_pairs=1000)
    R = b.meta["n_reads"]
    idx = np.arange(0, 2 * R, 2)
    A = logan.pool_to_device(b.poolA, b.offA[idx].copy(), b.lenA[idx].copy(), True,
                             (b.poolA.size - 1) * 16)
    c = ctx.overlap_candidates(A, k, 2, 4, mshared).cpu().numpy().view(np.uint32)
    a_, b_, o_ = c[:, 0].astype(np.int64), c[:, 1].astype(np.int64), c[:, 2].astype(np.int64)
    key = (a_ << 33) | (b_ << 1) | o_
    assert np.all(a_ < b_) and np.all(np.diff(key) > 0) and np.all(c[:, 5] >= mshared)
    rng = np.random.default_rng(301)
    reads = lambda i: b._seq(b.poolA, b.offA, b.lenA, 2 * int(i))
    for j in rng.choice(c.shape[0], 500, replace=False):
        sa = reads(c[j, 0])[c[j, 3]:c[j, 3] + k]
        sb = reads(c[j, 1])[c[j, 4]:c[j, 4] + k]
        assert sa == (ov.revcomp(sb) if c[j, 2] else sb)
    rs, rl, rv = b.meta["read_start"], b.meta["read_len"], b.meta["read_rev"]
    found = set(zip(a_.tolist(), b_.tolist(), o_.tolist()))
    order = np.argsort(rs, kind="stable")
    missed = checked = 0
    for i in rng.choice(R, 2000, replace=False):
        lo = np.searchsorted(rs[order], rs[i], side="left")
        hi = np.searchsorted(rs[order], rs[i] + rl[i] - 4000, side="left")
        for j in order[lo:hi]:
            if j == i or min(rs[i] + rl[i], rs[j] + rl[j]) - max(rs[i], rs[j]) < 4000:
                continue
            p, q = (i, j) if i < j else (j, i)
            checked += 1
            missed += (p, q, int(rv[i] ^ rv[j])) not in found
    assert checked > 1000 and missed <= checked // 100
