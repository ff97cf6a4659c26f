"""Seeded synthetic workloads for batched X-drop seed extension.

This module only draws inputs: read pools, seed positions, per-pair X. It
holds none of the method's arithmetic (no scoring, no extension, no seed
score), so both the CUDA path and the CPU oracle can consume what it makes
without sharing any step of the computation.

Every stream is numpy's PCG64 (`default_rng(seed)`), which gives the same
bytes on x86_64 and aarch64.

Workloads (sizes are parameters so tests can draw small copies):

* ``uniform_pairs``  -- 1,000 pairs, A uniform ACGT of 2,000 bp, B = A with
  15 % errors (sub/ins/del equally likely), exact 17-mer seed at A's
  midpoint, X = 50.  The paper's own workload is 100K pairs of 2.5-7.5 kbp
  at about 15 % error (Sec. VI, experimental setting); this is its small
  stand-in.
* ``lognormal_batch`` -- 100,000 pairs, lognormal lengths (median 10 kbp,
  sigma 0.5, clipped to 1-30 kbp), 80 % related at 12 % error with a
  midpoint seed, 20 % unrelated with one planted shared 17-mer, X = 100.
* ``uneven_batch``   -- 20,000 pairs, length classes 60/30/9/1 % over
  [1k,5k] / [5k,50k] / [50k,200k] / [200k,1M] (log-uniform inside a class),
  error rate U[5 %, 20 %] per pair, X drawn per pair from {10,50,100,500}.
* ``serving_requests`` -- Poisson arrivals of requests whose pairs follow
  the uneven mixture, X = 50.

Sequences are uint8 ASCII ('A','C','G','T').  ``pack2bit`` converts a pool
to the 2-bit packed input format of the library (A0 C1 G2 T3, 16 bases per
little-endian uint32 word, base k of the pool at word k//16, bits
2*(k%16)..2*(k%16)+1); it is a storage format, not part of the method.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

ASCII = np.frombuffer(b"ACGT", dtype=np.uint8)
SEED_LEN = 17
SEED_DTYPE = np.dtype([("idxA", "<u4"), ("idxB", "<u4"), ("posA", "<u4"),
                       ("posB", "<u4"), ("len", "<u4")])

# rough chunk of bases handled per vectorised mutation step (bounds host memory)
_CHUNK_BASES = 1 << 24


@dataclass
class Batch:
    """A batch of seeded pairs.

    poolA/poolB: uint8 ASCII bases of all sequences, concatenated.
    offA/offB:   uint64 base offset of each sequence in its pool.
    lenA/lenB:   uint32 length of each sequence.
    seeds:       SEED_DTYPE records, one per pair (indices into the pools).
    X:           scalar X for the batch; Xs: optional int32 per-pair X.
    """
    name: str
    poolA: np.ndarray
    offA: np.ndarray
    lenA: np.ndarray
    poolB: np.ndarray
    offB: np.ndarray
    lenB: np.ndarray
    seeds: np.ndarray
    X: int
    Xs: Optional[np.ndarray] = None
    match: int = 1
    mismatch: int = -1
    gap: int = -1
    shared_pool: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def n_pairs(self) -> int:
        return int(self.seeds.shape[0])

    def seqA(self, p: int) -> bytes:
        s = self.seeds[p]
        o, n = int(self.offA[s["idxA"]]), int(self.lenA[s["idxA"]])
        return self.poolA[o:o + n].tobytes()

    def seqB(self, p: int) -> bytes:
        s = self.seeds[p]
        o, n = int(self.offB[s["idxB"]]), int(self.lenB[s["idxB"]])
        return self.poolB[o:o + n].tobytes()

    def subset(self, idx) -> "Batch":
        """Pairs `idx` only (pools are shared, not copied)."""
        idx = np.asarray(idx)
        return Batch(self.name + "[sub]", self.poolA, self.offA, self.lenA,
                     self.poolB, self.offB, self.lenB, self.seeds[idx].copy(),
                     self.X, None if self.Xs is None else self.Xs[idx].copy(),
                     self.match, self.mismatch, self.gap, self.shared_pool,
                     dict(self.meta))

    @property
    def total_bases(self) -> int:
        n = int(self.lenA.sum(dtype=np.uint64))
        if not self.shared_pool:
            n += int(self.lenB.sum(dtype=np.uint64))
        return n


def pack2bit(pool: np.ndarray) -> np.ndarray:
    """ASCII pool -> uint32 words, 16 bases per word, A0 C1 G2 T3.

    The pool is padded with 'A' codes to a whole number of words plus one
    spare word (readers may fetch one word past the last base).
    """
    lut = np.full(256, 0, dtype=np.uint8)
    lut[ord("C")] = 1
    lut[ord("G")] = 2
    lut[ord("T")] = 3
    codes = lut[pool]
    nw = (codes.size + 15) // 16 + 1
    padded = np.zeros(nw * 16, dtype=np.uint32)
    padded[:codes.size] = codes
    padded = padded.reshape(nw, 16)
    shifts = (2 * np.arange(16, dtype=np.uint32))
    return np.bitwise_or.reduce(padded << shifts, axis=1).astype(np.uint32)


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(lengths.size, dtype=np.uint64)
    if lengths.size > 1:
        np.cumsum(lengths[:-1], dtype=np.uint64, out=off[1:])
    return off


_SHIFTS16 = (2 * np.arange(16, dtype=np.uint32))


def _random_bases(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniform ACGT bases (16 per uniform 32-bit draw)."""
    words = rng.integers(0, 1 << 32, size=(n + 15) // 16, dtype=np.uint32)
    codes = ((words[:, None] >> _SHIFTS16) & 3).astype(np.uint8).ravel()[:n]
    return ASCII[codes]


def _error_positions(rng, n: int, err_p) -> np.ndarray:
    """Sorted positions in [0, n) hit by an error: Bernoulli(err_p) per base.
    A scalar rate draws geometric gaps (same law, p*n draws instead of n)."""
    if np.ndim(err_p) == 0:
        p = float(err_p)
        if p <= 0.0 or n == 0:
            return np.zeros(0, dtype=np.int64)
        pos, base = [], -1
        while True:
            k = int(n * p + 6 * np.sqrt(n * p) + 16)
            gaps = rng.geometric(p, size=k)
            cs = base + np.cumsum(gaps)
            pos.append(cs[cs < n])
            if cs[-1] >= n:
                break
            base = int(cs[-1])
        return np.concatenate(pos)
    u = rng.random(n, dtype=np.float32)
    return np.flatnonzero(u < err_p)


def _mutate_chunk(rng, src: np.ndarray, err_p, protect_idx: np.ndarray, type_p: tuple):
    """Edit walk over `src` (ASCII, one chunk).

    Each base outside `protect_idx` suffers an error with probability err_p
    (a scalar, or one value per base); the error is a substitution (uniform
    other base), an insertion (a uniform base placed before it) or a deletion,
    with probabilities type_p.  Returns the output bases and, per source base,
    the number of output bases it made.
    """
    n = src.size
    err = _error_positions(rng, n, err_p)
    keep = np.ones(n, dtype=bool)
    keep[protect_idx] = False
    err = err[keep[err]]
    t = rng.random(err.size, dtype=np.float32)
    c_sub = np.float32(type_p[0])
    c_ins = np.float32(type_p[0] + type_p[1])
    sub = err[t < c_sub]
    ins = err[(t >= c_sub) & (t < c_ins)]
    dele = err[t >= c_ins]
    counts = np.ones(n, dtype=np.int32)
    counts[ins] = 2
    counts[dele] = 0
    csum = np.cumsum(counts, dtype=np.int64)
    out = np.repeat(src, counts)
    # the source base of an inserting position sits after the inserted base
    ins_pos = csum[ins] - 2
    out[ins_pos] = _random_bases(rng, ins_pos.size)
    lut = np.zeros(256, dtype=np.uint8)
    lut[ASCII] = np.arange(4, dtype=np.uint8)
    code = (lut[src[sub]] + rng.integers(1, 4, size=sub.size, dtype=np.uint8)) & 3
    out[csum[sub] - 1] = ASCII[code]
    return out, csum


def _chunks(lengths: np.ndarray, limit: int = _CHUNK_BASES):
    """Split sequence indices into consecutive runs of about `limit` bases
    (depends on the lengths only, so the random streams do not depend on how
    many threads draw them)."""
    cs = np.cumsum(lengths.astype(np.int64))
    cuts = np.searchsorted(cs, np.arange(limit, int(cs[-1]) if cs.size else 0, limit),
                           side="right") if cs.size else np.zeros(0, np.int64)
    edges = np.unique(np.concatenate([[0], cuts, [lengths.size]]))
    return list(zip(edges[:-1].tolist(), edges[1:].tolist()))


def _parallel(fn, jobs):
    if len(jobs) <= 1:
        return [fn(*j) for j in jobs]
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda j: fn(*j), jobs))


def _related_pairs(seed: int, tag: int, lenA: np.ndarray, protect_pos: np.ndarray,
                   err_rate, protect_len: int = SEED_LEN,
                   type_p=(1 / 3, 1 / 3, 1 / 3)):
    """Draw A uniformly and derive B from it by the edit walk, one chunk of
    pairs per random stream (seeded by (seed, tag, chunk)).

    protect_pos[p]/protect_len: a window of A[p] kept exact (the seed);
    posB[p] is where that window lands in B[p].  err_rate: scalar or one
    rate per pair.  Returns (poolA, poolB, lenB, posB).
    """
    rate = np.asarray(err_rate, dtype=np.float32)

    def one(ci, p0, p1):
        rng = np.random.default_rng([seed, tag, ci])
        lens = lenA[p0:p1].astype(np.int64)
        tot = int(lens.sum())
        src = _random_bases(rng, tot)
        starts = _offsets(lens).astype(np.int64)
        prot = (starts + protect_pos[p0:p1].astype(np.int64))[:, None] + np.arange(protect_len)
        ep = np.repeat(rate[p0:p1], lens) if rate.ndim else rate
        out, csum = _mutate_chunk(rng, src, ep, prot.ravel(), type_p)
        csum = np.concatenate([[0], csum])
        lb = (csum[starts + lens] - csum[starts]).astype(np.uint32)
        pb = (csum[starts + protect_pos[p0:p1].astype(np.int64)] - csum[starts]).astype(np.uint32)
        return src, out, lb, pb

    jobs = [(ci, p0, p1) for ci, (p0, p1) in enumerate(_chunks(lenA))]
    res = _parallel(one, jobs)
    if not res:
        z = np.zeros(0, np.uint8)
        return z, z.copy(), np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    poolA = np.concatenate([r[0] for r in res])
    poolB = np.concatenate([r[1] for r in res])
    return poolA, poolB, np.concatenate([r[2] for r in res]), np.concatenate([r[3] for r in res])


def _random_pool(seed: int, tag: int, lens: np.ndarray) -> np.ndarray:
    def one(ci, p0, p1):
        rng = np.random.default_rng([seed, tag, ci])
        return _random_bases(rng, int(lens[p0:p1].astype(np.int64).sum()))
    res = _parallel(one, [(ci, a, b) for ci, (a, b) in enumerate(_chunks(lens))])
    return np.concatenate(res) if res else np.zeros(0, np.uint8)


def uniform_pairs(n_pairs: int = 1000, length: int = 2000, err: float = 0.15,
                  X: int = 50, seed: int = 0) -> Batch:
    """1,000 x 2 kbp pairs, 15 % errors, midpoint 17-mer seed, X = 50."""
    rng = np.random.default_rng(seed)
    del rng
    lenA = np.full(n_pairs, length, dtype=np.uint32)
    offA = _offsets(lenA)
    posA = np.full(n_pairs, (length - SEED_LEN) // 2, dtype=np.uint32)
    poolA, poolB, lenB, posB = _related_pairs(seed, 1, lenA, posA, err)
    offB = _offsets(lenB)
    seeds = np.zeros(n_pairs, dtype=SEED_DTYPE)
    seeds["idxA"] = seeds["idxB"] = np.arange(n_pairs, dtype=np.uint32)
    seeds["posA"], seeds["posB"], seeds["len"] = posA, posB, SEED_LEN
    return Batch("uniform_pairs", poolA, offA, lenA, poolB, offB, lenB, seeds, X,
                 meta=dict(n_pairs=n_pairs, length=length, err=err, seed=seed))


def _lognormal_lengths(rng, n, median, sigma, lo, hi):
    x = rng.lognormal(np.log(median), sigma, size=n)
    return np.clip(np.rint(x), lo, hi).astype(np.uint32)


def lognormal_batch(n_pairs: int = 100_000, median: int = 10_000, sigma: float = 0.5,
                    lo: int = 1_000, hi: int = 30_000, related_frac: float = 0.8,
                    err: float = 0.12, X: int = 100, seed: int = 2) -> Batch:
    """100K pairs, lognormal lengths, 80 % related at 12 % error, X = 100."""
    rng = np.random.default_rng(seed)
    related = rng.random(n_pairs) < related_frac
    lenA = _lognormal_lengths(rng, n_pairs, median, sigma, lo, hi)
    offA = _offsets(lenA)
    posA = ((lenA.astype(np.int64) - SEED_LEN) // 2).astype(np.uint32)
    poolA, poolB, lenB, posB = _related_pairs(seed, 1, lenA, posA, err)
    offB = _offsets(lenB)
    # unrelated pairs: B is replaced by an independent read carrying one planted
    # 17-mer that also gets written into A at a uniform position
    un = np.flatnonzero(~related)
    if un.size:
        lenU = _lognormal_lengths(rng, un.size, median, sigma, lo, hi)
        randB = _random_pool(seed, 2, lenU)
        lenB = lenB.copy()
        lenB[un] = lenU
        newoff = _offsets(lenB)
        offU = _offsets(lenU)
        slot = np.full(n_pairs, -1, dtype=np.int64)
        slot[un] = np.arange(un.size)
        parts = []
        for p in range(n_pairs):
            if slot[p] < 0:
                o = int(offB[p])
                parts.append(poolB[o:o + int(lenB[p])])
            else:
                o = int(offU[slot[p]])
                parts.append(randB[o:o + int(lenU[slot[p]])])
        newpool = np.concatenate(parts)
        poolB, offB = newpool, newoff
        # one planted shared 17-mer at uniform positions in both sequences
        pa = rng.integers(0, lenA[un].astype(np.int64) - SEED_LEN + 1)
        pb = rng.integers(0, lenU.astype(np.int64) - SEED_LEN + 1)
        kmer = _random_bases(rng, un.size * SEED_LEN).reshape(un.size, SEED_LEN)
        ia = offA[un].astype(np.int64)[:, None] + pa[:, None] + np.arange(SEED_LEN)
        ib = offB[un].astype(np.int64)[:, None] + pb[:, None] + np.arange(SEED_LEN)
        poolA[ia] = kmer
        poolB[ib] = kmer
        posA = posA.copy()
        posA[un] = pa.astype(np.uint32)
        posB = posB.copy()
        posB[un] = pb.astype(np.uint32)
    seeds = np.zeros(n_pairs, dtype=SEED_DTYPE)
    seeds["idxA"] = seeds["idxB"] = np.arange(n_pairs, dtype=np.uint32)
    seeds["posA"], seeds["posB"], seeds["len"] = posA, posB, SEED_LEN
    return Batch("lognormal_batch", poolA, offA, lenA, poolB, offB, lenB, seeds, X,
                 meta=dict(n_pairs=n_pairs, median=median, sigma=sigma, err=err,
                           related_frac=related_frac, seed=seed))


UNEVEN_CLASSES = ((0.60, 1_000, 5_000), (0.30, 5_000, 50_000),
                  (0.09, 50_000, 200_000), (0.01, 200_000, 1_000_000))
UNEVEN_X = (10, 50, 100, 500)


def uneven_lengths(rng, n, max_len=None):
    """Heavy-tailed length mixture: class by 60/30/9/1 %, log-uniform inside."""
    probs = np.array([c[0] for c in UNEVEN_CLASSES])
    cls = rng.choice(len(UNEVEN_CLASSES), size=n, p=probs / probs.sum())
    lo = np.array([c[1] for c in UNEVEN_CLASSES], dtype=np.float64)[cls]
    hi = np.array([c[2] for c in UNEVEN_CLASSES], dtype=np.float64)[cls]
    if max_len is not None:
        hi = np.minimum(hi, max_len)
        lo = np.minimum(lo, hi)
    u = rng.random(n)
    L = np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.uint32)
    return L, cls


def uneven_batch(n_pairs: int = 20_000, seed: int = 3, max_len: Optional[int] = None,
                 X_choices=UNEVEN_X) -> Batch:
    """20K pairs, lengths 1 kbp-1 Mbp (60/30/9/1 %), error U[5,20] %, X per pair."""
    rng = np.random.default_rng(seed)
    lenA, cls = uneven_lengths(rng, n_pairs, max_len)
    lenA = np.maximum(lenA, SEED_LEN)
    offA = _offsets(lenA)
    err = rng.uniform(0.05, 0.20, size=n_pairs).astype(np.float32)
    Xs = np.asarray(X_choices, dtype=np.int32)[rng.integers(0, len(X_choices), size=n_pairs)]
    posA = ((lenA.astype(np.int64) - SEED_LEN) // 2).astype(np.uint32)
    poolA, poolB, lenB, posB = _related_pairs(seed, 1, lenA, posA, err)
    offB = _offsets(lenB)
    seeds = np.zeros(n_pairs, dtype=SEED_DTYPE)
    seeds["idxA"] = seeds["idxB"] = np.arange(n_pairs, dtype=np.uint32)
    seeds["posA"], seeds["posB"], seeds["len"] = posA, posB, SEED_LEN
    return Batch("uneven_batch", poolA, offA, lenA, poolB, offB, lenB, seeds,
                 int(max(X_choices)), Xs=Xs,
                 meta=dict(n_pairs=n_pairs, seed=seed, length_class=cls, max_len=max_len))


def serving_requests(n_requests: int, rate: float, seed: int = 4,
                     max_pairs: int = 10_000, max_len: Optional[int] = None,
                     X: int = 50):
    """Poisson arrivals (rate req/s) of requests of round(exp(U[0, ln max_pairs]))
    pairs each, pairs drawn like the uneven mixture.  Returns a list of
    (arrival_time_s, Batch)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.rint(np.exp(rng.uniform(0, np.log(max_pairs), size=n_requests))).astype(int)
    sizes = np.maximum(sizes, 1)
    out = []
    for r in range(n_requests):
        b = uneven_batch(int(sizes[r]), seed=int(rng.integers(1 << 62)), max_len=max_len,
                         X_choices=(X,))
        b.name = f"request{r}"
        out.append((float(t[r]), b))
    return out


def tiny_pairs(n_pairs: int, max_len: int, seed: int, alphabet: bytes = b"ACGT",
               X_choices=(0, 1, 2, 5, 10, 50)) -> Batch:
    """Random short pairs with arbitrary (in-bounds) seeds, for edge-case tests:
    lengths 0..max_len, seed length 0..min(17, room), X per pair."""
    rng = np.random.default_rng(seed)
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    lenA = rng.integers(0, max_len + 1, size=n_pairs).astype(np.uint32)
    lenB = rng.integers(0, max_len + 1, size=n_pairs).astype(np.uint32)
    poolA = alpha[rng.integers(0, alpha.size, size=int(lenA.sum()))]
    poolB = alpha[rng.integers(0, alpha.size, size=int(lenB.sum()))]
    k = np.minimum(rng.integers(0, SEED_LEN + 1, size=n_pairs), np.minimum(lenA, lenB))
    posA = rng.integers(0, lenA.astype(np.int64) - k + 1)
    posB = rng.integers(0, lenB.astype(np.int64) - k + 1)
    seeds = np.zeros(n_pairs, dtype=SEED_DTYPE)
    seeds["idxA"] = seeds["idxB"] = np.arange(n_pairs, dtype=np.uint32)
    seeds["posA"], seeds["posB"], seeds["len"] = posA, posB, k
    Xs = np.asarray(X_choices, dtype=np.int32)[rng.integers(0, len(X_choices), size=n_pairs)]
    return Batch("tiny_pairs", poolA, _offsets(lenA), lenA, poolB, _offsets(lenB), lenB,
                 seeds, int(max(X_choices)), Xs=Xs, meta=dict(seed=seed, max_len=max_len))
