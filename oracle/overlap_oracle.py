"""Overlap-candidate oracle (many-to-many seeding) -- TEST INFRASTRUCTURE ONLY.

A plain numpy restatement of the seeding step the paper's application runs
before X-drop extension (Sec. V: k-mers as seeds, pruning of k-mers unlikely
to be useful, a seed chosen per overlapping pair from the k-mer locations,
an adaptive threshold separating true alignments from false positives).
The paper describes these steps only in words; the readings below are this
project's (each is in the design notes).  Only tests and the benchmark's CPU
baseline use this module; it shares no code with the CUDA path.

Readings:
  O1 k-mer codes: base codes A0 C1 G2 T3; the forward code of the k-mer at
     position p of a read is sum_t c[p+t] << 2t (t < k, k <= 31), the
     reverse-complement code sum_t (3 - c[p+k-1-t]) << 2t; the canonical
     code is the smaller, strand = 1 when the reverse complement is
     strictly smaller.
  O2 frequency = occurrences of a canonical code over all k-mer positions of
     all reads; a k-mer is reliable when min_freq <= frequency <= max_freq.
  O3 hits: every two occurrences of a reliable k-mer in different reads
     a < b give a hit (a, b, o = strand_a xor strand_b, pos_a, pos_b).
  O4 candidates: the (a, b, o) with at least min_shared hits; the seed is
     the hit at index floor(count / 2) of the pair's hits sorted by
     (pos_a, pos_b) -- the middle of the chain of shared k-mers.
  O5 seed coordinates for extension: A = read a forward at pos_a; B = read
     b forward at pos_b when o = 0, else the reverse complement of read b
     at len_b - pos_b - k.
  O6 adaptive threshold: with left = min(posA, posB),
     right = min(lenA - posA - k, lenB - posB - k) and L = left + k + right
     (the overlap the seed's diagonal implies), a pair is kept when
     score * den >= ratio_num * L - delta * den (integer form of
     score >= (ratio_num / den) * L - delta).
"""
from __future__ import annotations

import numpy as np

CAND_DTYPE = np.dtype([("a", "<u4"), ("b", "<u4"), ("o", "<u4"), ("pos_a", "<u4"),
                       ("pos_b", "<u4"), ("count", "<u4")])

_LUT = np.zeros(256, dtype=np.uint64)
_LUT[ord("C")] = 1
_LUT[ord("G")] = 2
_LUT[ord("T")] = 3


def kmer_table(reads, k: int):
    """All k-mer occurrences (O1): (canonical, read, pos, strand) arrays,
    reads in order, positions ascending."""
    assert 1 <= k <= 31
    canon, rd, ps, st = [], [], [], []
    shifts = (2 * np.arange(k, dtype=np.uint64))
    for r, s in enumerate(reads):
        c = _LUT[np.frombuffer(s, dtype=np.uint8)] if len(s) else np.zeros(0, np.uint64)
        n = c.size - k + 1
        if n <= 0:
            continue
        win = np.lib.stride_tricks.sliding_window_view(c, k)  # [n, k], base p+t at column t
        f = np.bitwise_or.reduce(win << shifts, axis=1)
        rc = np.bitwise_or.reduce((np.uint64(3) - win[:, ::-1]) << shifts, axis=1)
        strand = (rc < f).astype(np.uint32)
        canon.append(np.minimum(f, rc))
        rd.append(np.full(n, r, dtype=np.uint32))
        ps.append(np.arange(n, dtype=np.uint32))
        st.append(strand)
    if not canon:
        z = np.zeros(0, np.uint32)
        return np.zeros(0, np.uint64), z, z.copy(), z.copy()
    return np.concatenate(canon), np.concatenate(rd), np.concatenate(ps), np.concatenate(st)


def candidates(reads, k: int = 17, min_freq: int = 2, max_freq: int = 4, min_shared: int = 1):
    """Overlap candidates (O2-O4), sorted by (a, b, o)."""
    canon, rd, ps, st = kmer_table(reads, k)
    if canon.size == 0:
        return np.zeros(0, CAND_DTYPE)
    order = np.lexsort((ps, rd, canon))  # by code, then read, then position
    canon, rd, ps, st = canon[order], rd[order], ps[order], st[order]
    starts = np.flatnonzero(np.concatenate([[True], canon[1:] != canon[:-1]]))
    ends = np.concatenate([starts[1:], [canon.size]])
    hits = []
    for s0, e0 in zip(starts, ends):
        f = e0 - s0
        if f < min_freq or f > max_freq:
            continue
        for i in range(s0, e0):
            for j in range(s0, e0):
                if rd[i] < rd[j]:
                    hits.append((rd[i], rd[j], st[i] ^ st[j], ps[i], ps[j]))
    if not hits:
        return np.zeros(0, CAND_DTYPE)
    h = np.array(hits, dtype=np.uint64)
    order = np.lexsort((h[:, 4], h[:, 3], h[:, 2], h[:, 1], h[:, 0]))
    h = h[order]
    key = h[:, :3]
    new = np.concatenate([[True], np.any(key[1:] != key[:-1], axis=1)])
    starts = np.flatnonzero(new)
    ends = np.concatenate([starts[1:], [h.shape[0]]])
    out = []
    for s0, e0 in zip(starts, ends):
        cnt = e0 - s0
        if cnt < min_shared:
            continue
        m = s0 + cnt // 2
        out.append((h[m, 0], h[m, 1], h[m, 2], h[m, 3], h[m, 4], cnt))
    return np.array(out, dtype=CAND_DTYPE) if out else np.zeros(0, CAND_DTYPE)


def seeds(cands, lengths, k: int):
    """Extension seeds (O5): (idxA, idxB, posA, posB, len) with reads 0..R-1
    forward and R + r the reverse complement of read r."""
    R = len(lengths)
    lb = np.asarray(lengths, dtype=np.int64)[cands["b"]]
    o = cands["o"].astype(np.int64)
    out = np.zeros(cands.size, dtype=[("idxA", "<u4"), ("idxB", "<u4"), ("posA", "<u4"),
                                      ("posB", "<u4"), ("len", "<u4")])
    out["idxA"] = cands["a"]
    out["idxB"] = cands["b"].astype(np.int64) + R * o
    out["posA"] = cands["pos_a"]
    out["posB"] = np.where(o == 1, lb - cands["pos_b"].astype(np.int64) - k, cands["pos_b"])
    out["len"] = k
    return out


def keep(score, lenA, lenB, posA, posB, k: int, ratio_num: int, den: int, delta: int):
    """Adaptive-threshold decision per pair (O6)."""
    lenA, lenB = np.asarray(lenA, np.int64), np.asarray(lenB, np.int64)
    posA, posB = np.asarray(posA, np.int64), np.asarray(posB, np.int64)
    left = np.minimum(posA, posB)
    right = np.minimum(lenA - posA - k, lenB - posB - k)
    L = left + k + right
    return np.asarray(score, np.int64) * den >= ratio_num * L - delta * den


def revcomp(s: bytes) -> bytes:
    return s[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA"))
