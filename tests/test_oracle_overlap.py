"""Pins of the overlap-candidate oracle (CPU only): k-mer codes against a
per-character definition, candidates against a brute-force string
comparison of every pair of reads, seed coordinates against the sequences,
and the threshold's closed form."""
import collections

import numpy as np
import pytest

from oracle import overlap_oracle as ov


def rand_reads(rng, n, lo, hi, genome=None):
    out = []
    for _ in range(n):
        L = int(rng.integers(lo, hi + 1))
        if genome is None:
            out.append(bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, L)]))
        else:
            s = int(rng.integers(0, len(genome) - L + 1))
            r = genome[s:s + L]
            out.append(ov.revcomp(r) if rng.random() < 0.5 else r)
    return out


def test_kmer_codes_per_character():
    rng = np.random.default_rng(1)
    val = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
    for k in (1, 3, 17, 31):
        reads = rand_reads(rng, 4, 0, 60)
        canon, rd, ps, st = ov.kmer_table(reads, k)
        i = 0
        for r, s in enumerate(reads):
            for p in range(len(s) - k + 1):
                w = s[p:p + k]
                f = sum(val[w[t]] << (2 * t) for t in range(k))
                rc = ov.revcomp(w)
                g = sum(val[rc[t]] << (2 * t) for t in range(k))
                assert (canon[i], rd[i], ps[i], st[i]) == (min(f, g), r, p, int(g < f))
                i += 1
        assert i == canon.size


def brute_candidates(reads, k, min_freq, max_freq, min_shared):
    """Every pair of reads compared window by window as strings."""
    def canon(w):
        return min(w, ov.revcomp(w))
    freq = collections.Counter(canon(s[p:p + k]) for s in reads for p in range(len(s) - k + 1))
    out = []
    for a in range(len(reads)):
        for b in range(a + 1, len(reads)):
            for o in (0, 1):
                hits = []
                for pa in range(len(reads[a]) - k + 1):
                    wa = reads[a][pa:pa + k]
                    if not (min_freq <= freq[canon(wa)] <= max_freq):
                        continue
                    for pb in range(len(reads[b]) - k + 1):
                        wb = reads[b][pb:pb + k]
                        same = wa == wb
                        rev = wa == ov.revcomp(wb)
                        # relative strand of the two occurrences (palindromes
                        # count as strand 0 on both sides)
                        sa = int(ov.revcomp(wa) < wa)
                        sb = int(ov.revcomp(wb) < wb)
                        if (same or rev) and (sa ^ sb) == o:
                            hits.append((pa, pb))
                if len(hits) >= min_shared and hits:
                    hits.sort()
                    pa, pb = hits[len(hits) // 2]
                    out.append((a, b, o, pa, pb, len(hits)))
    return out


@pytest.mark.parametrize("seed,k,fmax,mshared", [(0, 5, 4, 1), (1, 6, 3, 1), (2, 4, 6, 2),
                                                (3, 7, 2, 1)])
def test_candidates_brute_force(seed, k, fmax, mshared):
    rng = np.random.default_rng(seed)
    genome = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 300)])
    reads = rand_reads(rng, 9, 20, 60, genome) + rand_reads(rng, 3, 10, 30)
    got = ov.candidates(reads, k, 2, fmax, mshared)
    want = brute_candidates(reads, k, 2, fmax, mshared)
    assert [tuple(int(x) for x in r) for r in got] == want


def test_error_free_reads_find_every_overlap():
    # reads cut from one genome without errors: every two reads whose
    # intervals share >= 40 bases are candidates, seeded on their diagonal
    rng = np.random.default_rng(4)
    genome = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 5000)])
    starts = np.sort(rng.integers(0, 4600, 40))
    lens = rng.integers(200, 400, 40)
    lens = np.minimum(lens, 5000 - starts)
    reads = [genome[s:s + L] for s, L in zip(starts, lens)]
    k = 15
    got = ov.candidates(reads, k, 2, 64, 1)
    found = {(int(r["a"]), int(r["b"])): r for r in got if r["o"] == 0}
    for a in range(40):
        for b in range(a + 1, 40):
            ov_len = min(starts[a] + lens[a], starts[b] + lens[b]) - max(starts[a], starts[b])
            if ov_len >= 40:
                r = found[(a, b)]
                assert int(r["pos_a"]) + starts[a] == int(r["pos_b"]) + starts[b]


def test_seed_coordinates_match_sequences():
    rng = np.random.default_rng(5)
    genome = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 3000)])
    reads = rand_reads(rng, 30, 100, 400, genome)
    k = 13
    c = ov.candidates(reads, k, 2, 8, 1)
    assert c.size > 10 and np.any(c["o"] == 1)
    sd = ov.seeds(c, [len(r) for r in reads], k)
    pool = reads + [ov.revcomp(r) for r in reads]
    for s in sd:
        A, B = pool[s["idxA"]], pool[s["idxB"]]
        assert A[s["posA"]:s["posA"] + k] == B[s["posB"]:s["posB"] + k]


def test_threshold_closed_form():
    # overlap implied by the seed: min(10, 30) + 5 + min(85, 25) = 40 bases
    assert ov.keep([20], [100], [60], [10], [30], 5, 1, 2, 0)[0]      # 20 >= 40 / 2
    assert not ov.keep([19], [100], [60], [10], [30], 5, 1, 2, 0)[0]  # 19 < 20
    assert ov.keep([17], [100], [60], [10], [30], 5, 1, 2, 3)[0]      # 17 >= 20 - 3
    assert not ov.keep([16], [100], [60], [10], [30], 5, 1, 2, 3)[0]
    assert ov.keep([0], [5], [5], [0], [0], 5, 1, 1, 5)[0]            # L = 5, 0 >= 5 - 5
