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
* ``overlap_batch``  -- many-to-many overlap candidates: 50,000 reads
  sampled from a random 50 Mbp genome (lognormal lengths, mean 10 kbp,
  sigma 0.5; reverse strand with p = 0.5; 12 % errors as 6 % insertions,
  4 % deletions, 2 % substitutions), 1,000,000 candidate pairs: 30 % true
  overlaps seeded at the shared exact 17-mer nearest the overlap centre,
  70 % spurious pairs carrying one planted shared 17-mer, X = 50.  Its pool
  is built 2-bit packed (about 2 GB) and never exists as ASCII.

Sequences are uint8 ASCII ('A','C','G','T'), except in a batch built
packed (``Batch.packed``).  ``pack2bit`` converts a pool
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

    poolA/poolB: uint8 ASCII bases of all sequences, concatenated; or, when
                 `packed`, the uint32 words of the 2-bit packed pool (see
                 pack2bit), including its spare word.
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
    packed: bool = False

    @property
    def n_pairs(self) -> int:
        return int(self.seeds.shape[0])

    def _seq(self, pool, off, ln, i) -> bytes:
        o, n = int(off[i]), int(ln[i])
        if self.packed:
            return unpack2bit(pool, o, n).tobytes()
        return pool[o:o + n].tobytes()

    def seqA(self, p: int) -> bytes:
        return self._seq(self.poolA, self.offA, self.lenA, self.seeds[p]["idxA"])

    def seqB(self, p: int) -> bytes:
        return self._seq(self.poolB, self.offB, self.lenB, self.seeds[p]["idxB"])

    @property
    def pool_bases(self) -> int:
        """Bases the pools span (packed: whole words, without the spare)."""
        if self.packed:
            n = (self.poolA.size - 1) * 16
            return n if self.shared_pool else n + (self.poolB.size - 1) * 16
        return int(self.poolA.size) + (0 if self.shared_pool else int(self.poolB.size))

    def subset(self, idx) -> "Batch":
        """Pairs `idx` only.  ASCII pools are shared, not copied; a packed
        batch gives an ASCII batch holding just the sequences those pairs
        use (small enough for the CPU oracle)."""
        idx = np.asarray(idx)
        sd = self.seeds[idx].copy()
        Xs = None if self.Xs is None else self.Xs[idx].copy()
        if not self.packed:
            return Batch(self.name + "[sub]", self.poolA, self.offA, self.lenA,
                         self.poolB, self.offB, self.lenB, sd, self.X, Xs,
                         self.match, self.mismatch, self.gap, self.shared_pool,
                         dict(self.meta))

        def gather(pool, off, ln, ids):
            u, inv = np.unique(ids, return_inverse=True)
            lens = ln[u].astype(np.uint32)
            parts = [unpack2bit(pool, int(off[i]), int(ln[i])) for i in u]
            asc = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
            return asc, _offsets(lens), lens, inv.astype(np.uint32)

        if self.shared_pool:
            both = np.concatenate([sd["idxA"], sd["idxB"]])
            pool, off, ln, inv = gather(self.poolA, self.offA, self.lenA, both)
            sd["idxA"], sd["idxB"] = inv[:idx.size], inv[idx.size:]
            return Batch(self.name + "[sub]", pool, off, ln, pool, off, ln, sd, self.X, Xs,
                         self.match, self.mismatch, self.gap, True, dict(self.meta))
        pa, oa, la, ia = gather(self.poolA, self.offA, self.lenA, sd["idxA"])
        pb, ob, lb, ib = gather(self.poolB, self.offB, self.lenB, sd["idxB"])
        sd["idxA"], sd["idxB"] = ia, ib
        return Batch(self.name + "[sub]", pa, oa, la, pb, ob, lb, sd, self.X, Xs,
                     self.match, self.mismatch, self.gap, False, dict(self.meta))

    @property
    def total_bases(self) -> int:
        n = int(self.lenA.sum(dtype=np.uint64))
        if not self.shared_pool:
            n += int(self.lenB.sum(dtype=np.uint64))
        return n


_SHIFTS16 = (2 * np.arange(16, dtype=np.uint32))
_CODE_LUT = np.zeros(256, dtype=np.uint8)
_CODE_LUT[ord("C")] = 1
_CODE_LUT[ord("G")] = 2
_CODE_LUT[ord("T")] = 3


def pack2bit(pool: np.ndarray) -> np.ndarray:
    """ASCII pool -> uint32 words, 16 bases per word, A0 C1 G2 T3.

    The pool is padded with 'A' codes to a whole number of words plus one
    spare word (readers may fetch one word past the last base).  Works in
    chunks, so host memory stays near the pool's own size.
    """
    n = int(pool.size)
    out = np.zeros((n + 15) // 16 + 1, dtype=np.uint32)
    step = 1 << 24  # bases per chunk, a multiple of 16
    for s0 in range(0, n, step):
        m = min(step, n - s0)
        c = np.zeros((m + 15) // 16 * 16, dtype=np.uint8)
        c[:m] = _CODE_LUT[pool[s0:s0 + m]]
        q = c.reshape(-1, 4)
        # byte j holds bases 4j..4j+3; four bytes make one little-endian word
        by = q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)
        w = by.view("<u4")
        out[s0 // 16:s0 // 16 + w.size] = w
    return out


def unpack2bit(words: np.ndarray, off: int, n: int) -> np.ndarray:
    """Bases [off, off + n) of a packed pool, as ASCII."""
    if n <= 0:
        return np.zeros(0, dtype=np.uint8)
    w0, w1 = off // 16, (off + n + 15) // 16
    codes = ((words[w0:w1, None] >> _SHIFTS16) & 3).astype(np.uint8).ravel()
    s0 = off - 16 * w0
    return ASCII[codes[s0:s0 + n]]


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(lengths.size, dtype=np.uint64)
    if lengths.size > 1:
        np.cumsum(lengths[:-1], dtype=np.uint64, out=off[1:])
    return off


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


def _mutate_chunk(rng, src: np.ndarray, err_p, protect_idx: np.ndarray, type_p: tuple,
                  events: bool = False):
    """Edit walk over `src` (ASCII, one chunk).

    Each base outside `protect_idx` suffers an error with probability err_p
    (a scalar, or one value per base); the error is a substitution (uniform
    other base), an insertion (a uniform base placed before it) or a deletion,
    with probabilities type_p.  Returns the output bases and, per source base,
    the cumulative number of output bases up to and including it; with
    `events`, also the sorted source positions of the substitutions,
    insertions (a base inserted before the position) and deletions.
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
    if events:
        return out, csum, (sub, ins, dele)
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


class PairLibrary:
    """A library of seeded pairs from which serving requests are drawn.

    Every sequence is stored 2-bit packed from a 16-base boundary, so a
    request's pools are plain concatenations of word ranges and cost one
    vectorised gather to build.  Pairs are independent, so a pair's result
    is the same in every request that draws it.
    """

    def __init__(self, b: "Batch"):
        assert not b.packed and not b.shared_pool
        self.n_pairs = b.n_pairs
        self.X = b.X
        self.seeds = b.seeds.copy()
        self.sides = []
        for pool, off, ln, col in ((b.poolA, b.offA, b.lenA, "idxA"),
                                   (b.poolB, b.offB, b.lenB, "idxB")):
            ln = ln[b.seeds[col]].astype(np.uint32)          # one sequence per pair
            src = off[b.seeds[col]].astype(np.int64)
            nw = (ln.astype(np.int64) + 15) // 16            # whole words per sequence
            wo = np.concatenate([[0], np.cumsum(nw)[:-1]]).astype(np.int64)
            asc = np.full(int(nw.sum()) * 16, ord("A"), dtype=np.uint8)
            for i in range(ln.size):
                asc[wo[i] * 16:wo[i] * 16 + int(ln[i])] = pool[src[i]:src[i] + int(ln[i])]
            self.sides.append((pack2bit(asc), wo, nw, ln))
        self.meta = dict(b.meta)

    @property
    def total_bases(self) -> int:
        return int(sum(int(s[3].sum(dtype=np.uint64)) for s in self.sides))

    def request(self, idx, name: str = "request") -> "Batch":
        """A packed batch holding library pairs `idx` (in that order)."""
        idx = np.asarray(idx, dtype=np.int64)
        parts = []
        for words, wo, nw, ln in self.sides:
            cnt = nw[idx]
            start = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
            a, c = wo[idx].tolist(), cnt.tolist()
            w = np.concatenate([words[x:x + n] for x, n in zip(a, c)] +
                               [np.zeros(1, np.uint32)])
            parts.append((w, (start * 16).astype(np.uint64), ln[idx].copy()))
        sd = np.zeros(idx.size, dtype=SEED_DTYPE)
        sd["idxA"] = sd["idxB"] = np.arange(idx.size, dtype=np.uint32)
        for f in ("posA", "posB", "len"):
            sd[f] = self.seeds[f][idx]
        (wa, oa, la), (wb, ob, lb) = parts
        return Batch(name, wa, oa, la, wb, ob, lb, sd, self.X, packed=True,
                     meta=dict(library_pairs=idx))


def serving_library(n_pairs: int = 30_000, seed: int = 5, X: int = 50,
                    max_len: Optional[int] = None) -> PairLibrary:
    """Pairs drawn like the uneven-length mixture (1 kbp - 1 Mbp, error
    U[5, 20] %), one X for all, as a PairLibrary."""
    return PairLibrary(uneven_batch(n_pairs, seed=seed, max_len=max_len, X_choices=(X,)))


def request_sizes(rng: np.random.Generator, n: int, max_pairs: int = 10_000) -> np.ndarray:
    """Request sizes round(exp(U[0, ln max_pairs])), at least 1 (log-uniform)."""
    return np.maximum(np.rint(np.exp(rng.uniform(0, np.log(max_pairs), size=n))), 1).astype(int)


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


# ---------------------------------------------------------------------------
# protein pairs (substitution-matrix scoring)

# BLOSUM62 over the 20 standard amino acids, in this letter order (letter
# code = index), typed from the published table (Henikoff & Henikoff 1992).
AMINO = "ARNDCQEGHILKMFPSTWYV"
BLOSUM62 = np.array([
    [4, -1, -2, -2, 0, -1, -1, 0, -2, -1, -1, -1, -1, -2, -1, 1, 0, -3, -2, 0],
    [-1, 5, 0, -2, -3, 1, 0, -2, 0, -3, -2, 2, -1, -3, -2, -1, -1, -3, -2, -3],
    [-2, 0, 6, 1, -3, 0, 0, 0, 1, -3, -3, 0, -2, -3, -2, 1, 0, -4, -2, -3],
    [-2, -2, 1, 6, -3, 0, 2, -1, -1, -3, -4, -1, -3, -3, -1, 0, -1, -4, -3, -3],
    [0, -3, -3, -3, 9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1],
    [-1, 1, 0, 0, -3, 5, 2, -2, 0, -3, -2, 1, 0, -3, -1, 0, -1, -2, -1, -2],
    [-1, 0, 0, 2, -4, 2, 5, -2, 0, -3, -3, 1, -2, -3, -1, 0, -1, -3, -2, -2],
    [0, -2, 0, -1, -3, -2, -2, 6, -2, -4, -4, -2, -3, -3, -2, 0, -2, -2, -3, -3],
    [-2, 0, 1, -1, -3, 0, 0, -2, 8, -3, -3, -1, -2, -1, -2, -1, -2, -2, 2, -3],
    [-1, -3, -3, -3, -1, -3, -3, -4, -3, 4, 2, -3, 1, 0, -3, -2, -1, -3, -1, 3],
    [-1, -2, -3, -4, -1, -2, -3, -4, -3, 2, 4, -2, 2, 0, -3, -2, -1, -2, -1, 1],
    [-1, 2, 0, -1, -3, 1, 1, -2, -1, -3, -2, 5, -1, -3, -1, 0, -1, -3, -2, -2],
    [-1, -1, -2, -3, -1, 0, -2, -3, -2, 1, 2, -1, 5, 0, -2, -1, -1, -1, -1, 1],
    [-2, -3, -3, -3, -2, -3, -3, -3, -1, 0, 0, -3, 0, 6, -4, -2, -2, 1, 3, -1],
    [-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4, 7, -1, -1, -4, -3, -2],
    [1, -1, 1, 0, -1, 0, 0, 0, -1, -2, -2, 0, -1, -2, -1, 4, 1, -3, -2, -2],
    [0, -1, 0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1, 1, 5, -2, -2, 0],
    [-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1, 1, -4, -3, -2, 11, 2, -3],
    [-2, -2, -2, -3, -2, -1, -2, -3, 2, -1, -1, -2, -1, 3, -3, -2, -2, 2, 7, -1],
    [0, -3, -3, -3, -1, -2, -2, -3, -3, 3, 1, -2, 1, -1, -2, -2, 0, -3, -1, 4],
], dtype=np.int32)


def dna_matrix(match: int = 1, mismatch: int = -1) -> np.ndarray:
    """The 4 x 4 match / mismatch matrix over the codes A0 C1 G2 T3."""
    M = np.full((4, 4), mismatch, dtype=np.int32)
    np.fill_diagonal(M, match)
    return M


def protein_pairs(n_pairs: int = 20_000, lo: int = 100, hi: int = 2_000, err: float = 0.25,
                  related_frac: float = 0.8, seed_len: int = 8, X: int = 60,
                  seed: int = 12) -> Batch:
    """Seeded protein pairs as letter codes 0..19 (AMINO order), one byte each.

    A: uniform letters, length log-uniform in [lo, hi].  Related pairs: B is
    A with an edit at each position with probability err (substitution by a
    uniform other letter, insertion of a uniform letter, deletion: equally
    likely), the seed_len letters at A's midpoint protected and mapped into
    B.  Unrelated pairs: an independent B of its own length, A's seed
    k-mer written at a uniform position of B.  Pools hold codes, not ASCII."""
    rng = np.random.default_rng([seed, 7])
    n_rel = int(round(related_frac * n_pairs))
    lenA = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_pairs))).astype(np.int64)
    lenA = np.maximum(lenA, seed_len)
    posA = (lenA - seed_len) // 2
    As, Bs, posB = [], [], np.zeros(n_pairs, np.int64)
    for p in range(n_pairs):
        a = rng.integers(0, 20, size=int(lenA[p])).astype(np.uint8)
        if p < n_rel:
            out, pb = [], 0
            for t in range(a.size):
                if posA[p] <= t < posA[p] + seed_len:
                    if t == posA[p]:
                        pb = len(out)
                    out.append(a[t])
                    continue
                if rng.random() < err:
                    kind = rng.integers(0, 3)
                    if kind == 0:
                        out.append(np.uint8((a[t] + rng.integers(1, 20)) % 20))
                    elif kind == 1:
                        out.append(np.uint8(rng.integers(0, 20)))
                        out.append(a[t])
                    continue  # deletion (kind 2) keeps nothing
                out.append(a[t])
            b = np.array(out, dtype=np.uint8)
        else:
            lb = int(np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
            lb = max(lb, seed_len)
            b = rng.integers(0, 20, size=lb).astype(np.uint8)
            pb = int(rng.integers(0, lb - seed_len + 1))
            b[pb:pb + seed_len] = a[posA[p]:posA[p] + seed_len]
        As.append(a)
        Bs.append(b)
        posB[p] = pb
    order = rng.permutation(n_pairs)  # related and unrelated mixed
    As = [As[i] for i in order]
    Bs = [Bs[i] for i in order]
    lA = np.array([x.size for x in As], np.uint32)
    lB = np.array([x.size for x in Bs], np.uint32)
    seeds = np.zeros(n_pairs, dtype=SEED_DTYPE)
    seeds["idxA"] = seeds["idxB"] = np.arange(n_pairs, dtype=np.uint32)
    seeds["posA"] = posA[order]
    seeds["posB"] = posB[order]
    seeds["len"] = seed_len
    return Batch("protein_pairs", np.concatenate(As), _offsets(lA), lA, np.concatenate(Bs),
                 _offsets(lB), lB, seeds, X,
                 meta=dict(n_pairs=n_pairs, seed=seed, alphabet=AMINO, related=order < n_rel))


# ---------------------------------------------------------------------------
# many-to-many overlap candidates

OVERLAP_TYPES = (2 / 12, 6 / 12, 4 / 12)  # (sub, ins, del) shares of the errors
_COMP = np.zeros(256, dtype=np.uint8)
_COMP[np.frombuffer(b"ACGT", np.uint8)] = np.frombuffer(b"TGCA", np.uint8)
_KEY_SHIFT = 27  # event key = read << 27 | genome position (genome < 2^27 bases)


def _count_in(keys: np.ndarray, r: np.ndarray, g0: np.ndarray, g1: np.ndarray) -> np.ndarray:
    """Events of read r at genome positions [g0, g1] (vectorised)."""
    base = r.astype(np.int64) << _KEY_SHIFT
    return (np.searchsorted(keys, base | g1.astype(np.int64), side="right") -
            np.searchsorted(keys, base | g0.astype(np.int64), side="left"))


def _read_pos(r, g, starts, ins_keys, del_keys):
    """Index in the forward-oriented read r of the kept genome base g: its
    offset, plus the bases inserted at or before it, minus those deleted
    before it."""
    rr = np.asarray(r, np.int64)
    gg = np.asarray(g, np.int64)
    lo = np.zeros_like(gg)
    n_ins = _count_in(ins_keys, rr, starts[rr] + lo, gg)
    n_del = _count_in(del_keys, rr, starts[rr] + lo, gg - 1)
    return gg - starts[rr] + n_ins - n_del


def overlap_batch(n_pairs: int = 1_000_000, n_reads: int = 50_000,
                  genome_len: int = 50_000_000, mean_len: int = 10_000, sigma: float = 0.5,
                  true_frac: float = 0.3, err: float = 0.12, type_p=OVERLAP_TYPES,
                  X: int = 50, seed: int = 1, min_len: int = 1_000) -> Batch:
    """Overlap candidates between reads of one random genome.

    Genome: uniform ACGT of genome_len bases.  Reads: lognormal lengths with
    the given mean (mu = ln(mean) - sigma^2/2), clipped to [min_len,
    genome_len], uniform start, edit walk at rate `err` split by `type_p`
    (sub, ins, del), reverse-complemented with p = 0.5.  The pool holds every
    read as sequenced (index 2r) and its reverse complement (2r + 1), each
    starting on a 16-base boundary, then one copy per spurious pair.

    True overlaps (true_frac of the pairs): read a uniform, read b uniform
    among the reads whose start lies in a's window, kept when the genome
    intervals share at least 17 bases.  B is b in a's orientation; the seed is
    the genome 17-mer that both reads hold exactly (no substitution or
    deletion in it, no insertion inside it) nearest the centre of the
    overlap, ties to the right; a pair without one is drawn again.
    Spurious pairs: reads a, b with disjoint intervals; B is a copy of b with
    the 17-mer of a at a uniform position written over a uniform position.
    """
    assert genome_len < (1 << _KEY_SHIFT)
    rng = np.random.default_rng([seed, 0])
    genome = _random_bases(rng, genome_len)
    mu = np.log(mean_len) - sigma * sigma / 2
    rl = np.clip(np.rint(rng.lognormal(mu, sigma, size=n_reads)), max(min_len, SEED_LEN),
                 genome_len).astype(np.int64)
    rs = rng.integers(0, genome_len - rl + 1).astype(np.int64)
    rev = rng.random(n_reads) < 0.5

    # edit walks, one chunk of reads per random stream
    def walk(ci, r0, r1):
        g = np.random.default_rng([seed, 1, ci])
        lens = rl[r0:r1]
        src = np.concatenate([genome[a:a + n] for a, n in zip(rs[r0:r1], lens)])
        out, csum, ev = _mutate_chunk(g, src, np.float32(err), np.zeros(0, np.int64), type_p,
                                      events=True)
        st = _offsets(lens).astype(np.int64)
        before = np.where(st > 0, csum[np.maximum(st - 1, 0)], 0)
        olen = csum[st + lens - 1] - before
        keys = []
        n = src.size
        kill = np.zeros(n + 1, dtype=np.int32)
        for t, e in enumerate(ev):
            rr = np.searchsorted(st, e, side="right") - 1
            keys.append(((rr + r0).astype(np.int64) << _KEY_SHIFT) | (rs[r0 + rr] + e - st[rr]))
            # window starts this event spoils: [e-16, e] for a substitution or
            # deletion, [e-16, e-1] for an insertion (placed before base e)
            lo = np.maximum(e - (SEED_LEN - 1), st[rr])
            hi = e if t != 1 else e - 1
            ok = hi >= lo
            kill += np.bincount(lo[ok], minlength=n + 1).astype(np.int32)
            kill -= np.bincount(hi[ok] + 1, minlength=n + 1).astype(np.int32)
        clean = np.cumsum(kill[:n], dtype=np.int32) == 0
        return out, olen, keys, clean

    res = _parallel(walk, [(ci, a, b) for ci, (a, b) in enumerate(_chunks(rl))])
    fwd = np.concatenate([x[0] for x in res])
    flen = np.concatenate([x[1] for x in res]).astype(np.int64)
    sub_k, ins_k, del_k = (np.concatenate([x[2][t] for x in res]) for t in range(3))
    clean = np.concatenate([x[3] for x in res])  # per genome base of each read's span
    coff = _offsets(rl).astype(np.int64)
    foff = _offsets(flen).astype(np.int64)
    del res, sub_k

    # true overlaps: draw, then look for a seed; redraw the pairs that have none
    n_true = int(round(true_frac * n_pairs))
    order = np.argsort(rs, kind="stable")
    ss = rs[order]
    Lmax = int(rl.max())
    ta = np.zeros(0, np.int64)
    tb = np.zeros(0, np.int64)
    tp = np.zeros(0, np.int64)
    while ta.size < n_true:
        need = n_true - ta.size
        a = rng.integers(0, n_reads, size=4 * need + 64)
        lo = np.searchsorted(ss, rs[a] - Lmax, side="left")
        hi = np.searchsorted(ss, rs[a] + rl[a], side="left")
        b = order[np.minimum(lo + (rng.random(a.size) * (hi - lo)).astype(np.int64), n_reads - 1)]
        o0 = np.maximum(rs[a], rs[b])
        o1 = np.minimum(rs[a] + rl[a], rs[b] + rl[b])
        ok = (b != a) & (o1 - o0 >= SEED_LEN)
        a, b, o0, o1 = a[ok], b[ok], o0[ok], o1[ok]
        # nearest clean 17-mer to the centre: offsets 0, +1, -1, +2, ... in blocks
        c = (o0 + o1 - SEED_LEN) // 2
        found = np.full(a.size, -1, np.int64)
        todo = np.arange(a.size)
        span = int((o1 - o0).max()) if a.size else 0
        block = 64
        for k0 in range(0, 2 * span + 2, block):
            if todo.size == 0:
                break
            ks = np.arange(k0, k0 + block)
            delta = np.where(ks % 2 == 1, (ks + 1) // 2, -(ks // 2))
            p = c[todo, None] + delta[None, :]
            valid = (p >= o0[todo, None]) & (p <= o1[todo, None] - SEED_LEN)
            both = valid.copy()
            for r in (a[todo], b[todo]):
                idx = coff[r][:, None] + (p - rs[r][:, None])
                both &= clean[np.where(valid, idx, 0)]
            hit = both.any(axis=1)
            first = np.argmax(both, axis=1)
            found[todo[hit]] = p[hit, first[hit]]
            todo = todo[~hit]
        good = found >= 0
        take = np.flatnonzero(good)[:need]
        ta = np.concatenate([ta, a[take]])
        tb = np.concatenate([tb, b[take]])
        tp = np.concatenate([tp, found[take]])

    # seed coordinates in the forward-oriented reads, then in the stored ones
    qa = _read_pos(ta, tp, rs, ins_k, del_k)
    qb = _read_pos(tb, tp, rs, ins_k, del_k)
    ra = rev[ta]
    posA_t = np.where(ra, flen[ta] - qa - SEED_LEN, qa)
    posB_t = np.where(ra, flen[tb] - qb - SEED_LEN, qb)
    # B in a's orientation: b as sequenced when the strands agree
    idxB_t = 2 * tb + (rev[ta] != rev[tb])
    idxA_t = 2 * ta

    # pool of the oriented reads: 2r = as sequenced, 2r + 1 = reverse complement
    slen = np.repeat(flen, 2)
    pad = (slen + 15) // 16 * 16
    soff = _offsets(pad).astype(np.int64)
    asc = np.full(int(pad.sum()), ord("A"), dtype=np.uint8)
    rcpool = _COMP[fwd[::-1]]  # read r's reverse complement ends where r starts
    tot = fwd.size
    for r in range(n_reads):
        f = fwd[foff[r]:foff[r] + flen[r]]
        rc = rcpool[tot - foff[r] - flen[r]:tot - foff[r]]
        s_, o_ = (rc, f) if rev[r] else (f, rc)
        asc[soff[2 * r]:soff[2 * r] + flen[r]] = s_
        asc[soff[2 * r + 1]:soff[2 * r + 1] + flen[r]] = o_
    del fwd, rcpool, clean
    words = pack2bit(asc)
    del asc

    # spurious pairs: disjoint intervals, B = copy of b with a planted 17-mer
    n_sp = n_pairs - n_true
    sa = np.zeros(0, np.int64)
    sb = np.zeros(0, np.int64)
    while sa.size < n_sp:
        need = n_sp - sa.size
        a = rng.integers(0, n_reads, size=need + 64)
        b = rng.integers(0, n_reads, size=need + 64)
        ok = (np.minimum(rs[a] + rl[a], rs[b] + rl[b]) <= np.maximum(rs[a], rs[b]))
        sa = np.concatenate([sa, a[ok][:need]])
        sb = np.concatenate([sb, b[ok][:need]])
    src = 2 * sb
    cw = pad[src] // 16
    coff_w = words.size - 1 + _offsets(cw).astype(np.int64)  # copies start after the spare word's slot
    parts = [words[:-1]]
    w_of = soff // 16
    parts += [words[w_of[i]:w_of[i] + n] for i, n in zip(src, cw)]
    parts.append(np.zeros(1, np.uint32))
    words = np.concatenate(parts)
    del parts
    posA_s = rng.integers(0, slen[2 * sa] - SEED_LEN + 1)
    posB_s = rng.integers(0, slen[src] - SEED_LEN + 1)
    abase = soff[2 * sa] + posA_s
    cbase = coff_w * 16 + posB_s
    for t in range(SEED_LEN):
        pa_ = abase + t
        code = (words[pa_ >> 4] >> ((pa_ & 15) * 2).astype(np.uint32)) & np.uint32(3)
        pc = cbase + t
        sh = ((pc & 15) * 2).astype(np.uint32)
        wi = pc >> 4
        words[wi] = (words[wi] & ~(np.uint32(3) << sh)) | (code << sh)

    off = np.concatenate([soff, coff_w * 16]).astype(np.uint64)
    lens = np.concatenate([slen, slen[src]]).astype(np.uint32)
    idxB_s = 2 * n_reads + np.arange(n_sp)
    seeds = np.zeros(n_pairs, dtype=SEED_DTYPE)
    is_true = np.zeros(n_pairs, dtype=bool)
    perm = rng.permutation(n_pairs)
    tsel, ssel = perm[:n_true], perm[n_true:]
    is_true[tsel] = True
    seeds["idxA"][tsel], seeds["idxB"][tsel] = idxA_t, idxB_t
    seeds["posA"][tsel], seeds["posB"][tsel] = posA_t, posB_t
    seeds["idxA"][ssel], seeds["idxB"][ssel] = 2 * sa, idxB_s
    seeds["posA"][ssel], seeds["posB"][ssel] = posA_s, posB_s
    seeds["len"] = SEED_LEN
    return Batch("overlap_batch", words, off, lens, words, off, lens, seeds, X,
                 shared_pool=True, packed=True,
                 meta=dict(n_pairs=n_pairs, n_reads=n_reads, genome_len=genome_len,
                           mean_len=mean_len, sigma=sigma, err=err, seed=seed,
                           is_true=is_true, true_genome_pos=(tsel, tp),
                           read_start=rs, read_len=rl, read_rev=rev,
                           genome=genome if genome_len <= (1 << 22) else None))
