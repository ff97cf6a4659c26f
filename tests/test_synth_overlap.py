"""The many-to-many overlap workload generator (CPU only): seeds are exact,
true overlaps are seeded at the genome 17-mer they share, spurious pairs
carry one planted 17-mer, and the packed pool reads back unchanged."""
import numpy as np
import pytest

from paper_2002_05200_gb300 import synth


@pytest.fixture(scope="module")
def small():
    return synth.overlap_batch(n_pairs=3000, n_reads=300, genome_len=800_000, seed=9)


def test_pack_roundtrip():
    rng = np.random.default_rng(1)
    pool = synth.ASCII[rng.integers(0, 4, size=70_001)]
    w = synth.pack2bit(pool)
    assert w.size == (pool.size + 15) // 16 + 1 and w[-1] == 0
    for off, n in ((0, 1), (5, 40), (69_990, 11), (32, 16), (0, 70_001)):
        assert np.array_equal(synth.unpack2bit(w, off, n), pool[off:off + n])
    # base k sits at bits 2(k % 16) of word k // 16 (A0 C1 G2 T3)
    w2 = synth.pack2bit(np.frombuffer(b"ACGTT", np.uint8))
    assert int(w2[0]) == 0 | (1 << 2) | (2 << 4) | (3 << 6) | (3 << 8)


def test_seeds_exact_and_fractions(small):
    b = small
    assert b.packed and b.shared_pool and b.n_pairs == 3000
    assert abs(b.meta["is_true"].mean() - 0.3) < 1e-9
    for p in range(b.n_pairs):
        s = b.seeds[p]
        A, B = b.seqA(p), b.seqB(p)
        assert s["posA"] + 17 <= len(A) and s["posB"] + 17 <= len(B)
        assert A[s["posA"]:s["posA"] + 17] == B[s["posB"]:s["posB"] + 17]


def test_true_seeds_are_genome_kmers(small):
    b = small
    g = b.meta["genome"]
    rev = b.meta["read_rev"]
    rs, rl = b.meta["read_start"], b.meta["read_len"]
    tsel, tp = b.meta["true_genome_pos"]
    for p, gp in zip(tsel, tp):
        s = b.seeds[p]
        a, bb = s["idxA"] // 2, s["idxB"] // 2
        # the seed lies in both reads' genome intervals
        assert max(rs[a], rs[bb]) <= gp and gp + 17 <= min(rs[a] + rl[a], rs[bb] + rl[bb])
        kmer = np.frombuffer(b.seqA(p), np.uint8)[s["posA"]:s["posA"] + 17]
        want = synth._COMP[g[gp:gp + 17][::-1]] if rev[a] else g[gp:gp + 17]
        assert np.array_equal(kmer, want)
        # B is read b in a's orientation: its reverse complement when strands differ
        assert s["idxA"] % 2 == 0 and s["idxB"] % 2 == int(rev[a] != rev[bb])


def test_spurious_pairs_are_planted_copies(small):
    b = small
    n_reads = b.meta["n_reads"]
    rs, rl = b.meta["read_start"], b.meta["read_len"]
    for p in np.flatnonzero(~b.meta["is_true"])[:400]:
        s = b.seeds[p]
        assert s["idxB"] >= 2 * n_reads  # a copy, never a pooled read
        copy = np.frombuffer(b.seqB(p), np.uint8)
        # the copy's source read: same length, differing only inside the seed
        src = [i for i in range(0, 2 * n_reads, 2) if b.lenA[i] == copy.size]
        ok = False
        for i in src:
            d = np.flatnonzero(np.frombuffer(b._seq(b.poolA, b.offA, b.lenA, i), np.uint8) != copy)
            if d.size == 0 or (d.min() >= s["posB"] and d.max() < s["posB"] + 17):
                a, bb = s["idxA"] // 2, i // 2
                # the two reads' genome intervals are disjoint
                assert min(rs[a] + rl[a], rs[bb] + rl[bb]) <= max(rs[a], rs[bb])
                ok = True
                break
        assert ok


def test_subset_unpacks(small):
    b = small
    idx = np.array([5, 17, 2999, 0])
    sub = b.subset(idx)
    assert not sub.packed and sub.n_pairs == 4
    for k, p in enumerate(idx):
        assert sub.seqA(k) == b.seqA(p) and sub.seqB(k) == b.seqB(p)
        for f in ("posA", "posB", "len"):
            assert sub.seeds[k][f] == b.seeds[p][f]
