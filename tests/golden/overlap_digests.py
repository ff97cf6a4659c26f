"""Stored oracle results of the 1,000,000-candidate overlap workload, as
SHA-256 digests per chunk of pairs.

The oracle needs about 2.5e12 cell updates for this workload (tens of minutes
on a host), too long to rerun inside the GPU test, so this script runs it
once and stores a digest of every chunk's results.  The GPU test hashes its
own results the same way and compares chunk by chunk.

Only the seeded generator (paper_2002_05200_gb300.synth) and the oracle are
called here; nothing comes from the CUDA path.  Regenerate with

    python tests/golden/overlap_digests.py

which rewrites tests/golden/overlap_batch_1m.sha256.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
DIGEST_FILE = os.path.join(HERE, "overlap_batch_1m.sha256")
FIELDS = ("score", "left", "right", "begA", "begB", "endA", "endB", "cells")
CHUNK = 20_000


def input_digest(b) -> str:
    """Digest of everything the extension reads: seeds, X, scoring, the pool."""
    h = hashlib.sha256()
    for f in ("idxA", "idxB", "posA", "posB", "len"):
        h.update(np.ascontiguousarray(b.seeds[f], dtype="<u4").tobytes())
    h.update(np.array([b.X, b.match, b.mismatch, b.gap], dtype="<i8").tobytes())
    for a in (b.offA, b.lenA, b.poolA):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def canonical(res, ok) -> np.ndarray:
    """Results as an int64 [n, 9] array: the eight fields, then 0 (valid) or
    1 (not valid); a pair that is not valid has its fields zeroed."""
    arr = np.zeros((ok.size, len(FIELDS) + 1), dtype="<i8")
    for k, f in enumerate(FIELDS):
        arr[:, k] = np.where(ok, res[f].astype(np.int64), 0)
    arr[:, -1] = (~ok).astype(np.int64)
    return arr


def chunk_digests(arr: np.ndarray):
    return [hashlib.sha256(arr[c0:c0 + CHUNK].tobytes()).hexdigest()
            for c0 in range(0, arr.shape[0], CHUNK)]


def read_digest_file(path: str = DIGEST_FILE):
    """-> (input digest, chunk size, [chunk digests], [chunk cells])"""
    inp, chunk, digs, cells = None, None, [], []
    with open(path) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "input":
                inp = t[1]
            elif t[0] == "chunk_pairs":
                chunk = int(t[1])
            elif t[0] == "chunk":
                digs.append(t[2])
                cells.append(int(t[3]))
    return inp, chunk, digs, cells


def main():
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2002_05200_gb300 import synth

    t0 = time.time()
    b = synth.overlap_batch()
    print(f"generated {b.n_pairs} pairs in {time.time() - t0:.0f} s", flush=True)
    inp = input_digest(b)
    lines = ["# Oracle results of the overlap workload: synth.overlap_batch() with its",
             "# defaults (1,000,000 candidates, 50,000 reads of a 50 Mbp genome, X = 50,",
             "# +1/-1/-1), written by tests/golden/overlap_digests.py, which calls only",
             "# the seeded generator and oracle/.  One SHA-256 per chunk of consecutive",
             "# pairs over little-endian int64 rows (score, left, right, begA, begB, endA,",
             "# endB, cells, not-valid flag), then the chunk's cell count.",
             f"input {inp}", f"chunk_pairs {CHUNK}"]
    total = 0
    for k, c0 in enumerate(range(0, b.n_pairs, CHUNK)):
        t1 = time.time()
        idx = np.arange(c0, min(c0 + CHUNK, b.n_pairs))
        res, used = oracle.run_batch(b.subset(idx))
        ok = res["status"] == oracle.OK
        arr = canonical(res, ok)
        cells = int(arr[:, FIELDS.index("cells")].sum())
        total += cells
        lines.append(f"chunk {k} {chunk_digests(arr)[0]} {cells}")
        print(f"chunk {k}: {cells} cells, {time.time() - t1:.0f} s on {used} threads", flush=True)
    lines.append(f"# total cells {total}; oracle time {time.time() - t0:.0f} s")
    with open(DIGEST_FILE + ".tmp", "w") as fh:
        fh.write("\n".join(lines) + "\n")
    os.replace(DIGEST_FILE + ".tmp", DIGEST_FILE)
    print("wrote", DIGEST_FILE)


if __name__ == "__main__":
    main()
