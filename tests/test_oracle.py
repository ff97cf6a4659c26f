"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * a textbook full-matrix DP (row-major fill, free end) when X is so large
    that nothing can be pruned -- best score, its coordinates under the
    first-anti-diagonal / smallest-row tie-break, and the full cell count;
  * closed forms: identical sequences, disjoint alphabets, an empty side,
    X below the gap cost;
  * hand-derived worked examples (tests/golden/worked_examples.txt);
  * invariants on random inputs (bounds, full-DP upper bound, symmetry);
  * the X-monotonicity counterexample of the chosen reading;
  * input validation;
and cross-checked (not pinned) against a second sweep kept as per-anti-
diagonal dictionaries on every tiny input size.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.txt")
SCHEMES = [(1, -1, -1), (2, -3, -2), (5, -4, -7), (1, -1, 0), (3, 1, -2)]


def full_dp(a: bytes, b: bytes, M: int, MM: int, G: int):
    """Textbook DP over the whole (m+1)x(n+1) matrix, filled row by row.

    S(0,0)=0, S(i,0)=i*G, S(0,j)=j*G, S(i,j)=max(S(i-1,j-1)+sub, S(i-1,j)+G,
    S(i,j-1)+G).  Returns (best, bi, bj) where best = max(0, max S) and the
    cell is on the smallest anti-diagonal holding that value, smallest i.
    """
    m, n = len(a), len(b)
    S = np.zeros((m + 1, n + 1), dtype=np.int64)
    for j in range(1, n + 1):
        S[0, j] = j * G
    for i in range(1, m + 1):
        S[i, 0] = i * G
        for j in range(1, n + 1):
            sub = M if a[i - 1] == b[j - 1] else MM
            S[i, j] = max(S[i - 1, j - 1] + sub, S[i - 1, j] + G, S[i, j - 1] + G)
    best = max(0, int(S.max()))
    if best == 0:
        return 0, 0, 0, S
    cand = [(i + j, i, j) for i in range(m + 1) for j in range(n + 1) if S[i, j] == best]
    d, i, j = min(cand)
    return best, i, j, S


def rand_seq(rng, n: int) -> bytes:
    return np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, size=int(n))].tobytes()


def no_prune_X(a, b, M, MM, G):
    return (len(a) + len(b) + 2) * max(abs(M), abs(MM), abs(G)) + 1


def strings(alpha: bytes, max_len: int):
    for L in range(max_len + 1):
        for t in itertools.product(alpha, repeat=L):
            yield bytes(t)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_unpruned_equals_full_dp_exhaustive(scheme):
    M, MM, G = scheme
    seqs = list(strings(b"ACGT", 3))
    for a in seqs:
        for b in seqs:
            X = no_prune_X(a, b, M, MM, G)
            best, bi, bj, cells = oracle.extend(a, b, M, MM, G, X)
            ref = full_dp(a, b, M, MM, G)
            assert (best, bi, bj) == tuple(ref[:3]), (a, b, scheme)
            assert cells == (len(a) + 1) * (len(b) + 1) - 1


def test_unpruned_equals_full_dp_binary_alphabet():
    seqs = list(strings(b"AC", 5))
    for a in seqs[::3]:
        for b in seqs:
            X = no_prune_X(a, b, 1, -1, -1)
            got = oracle.extend(a, b, 1, -1, -1, X)
            ref = full_dp(a, b, 1, -1, -1)
            assert got[:3] == tuple(ref[:3]), (a, b)


@pytest.mark.parametrize("seed", range(4))
def test_unpruned_equals_full_dp_random(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(25):
        m, n = rng.integers(0, 70, size=2)
        a = rand_seq(rng, m)
        b = rand_seq(rng, n)
        M, MM, G = SCHEMES[rng.integers(len(SCHEMES))]
        X = no_prune_X(a, b, M, MM, G)
        best, bi, bj, cells = oracle.extend(a, b, M, MM, G, X)
        ref = full_dp(a, b, M, MM, G)
        assert (best, bi, bj) == tuple(ref[:3])
        assert cells == (m + 1) * (n + 1) - 1


def test_pruned_bounded_by_full_dp_random():
    rng = np.random.default_rng(7)
    for _ in range(300):
        m, n = rng.integers(0, 40, size=2)
        a = rand_seq(rng, m)
        b = rand_seq(rng, n)
        M, MM, G = SCHEMES[rng.integers(len(SCHEMES))]
        X = int(rng.integers(0, 12))
        best, bi, bj, cells = oracle.extend(a, b, M, MM, G, X)
        ref = full_dp(a, b, M, MM, G)
        assert 0 <= best <= ref[0]
        assert 0 <= bi <= m and 0 <= bj <= n
        assert 0 <= cells <= (m + 1) * (n + 1) - 1
        if best > 0:
            # the reported cell holds a path of score `best`; the full DP at
            # that cell is the best over all paths, so it cannot be lower
            assert ref[3][bi, bj] >= best
        # transposing the problem computes the transposed cells
        tb = oracle.extend(b, a, M, MM, G, X)
        assert tb[0] == best and tb[3] == cells


@pytest.mark.parametrize("L", [1, 2, 7, 40, 333])
@pytest.mark.parametrize("X", [1, 3, 50])
def test_identical_sequences(L, X):
    rng = np.random.default_rng(L)
    a = rand_seq(rng, L)
    best, bi, bj, _ = oracle.extend(a, a, 1, -1, -1, X)
    assert (best, bi, bj) == (L, L, L)
    best, bi, bj, _ = oracle.extend(a, a, 3, -2, -2, X + 2)
    assert (best, bi, bj) == (3 * L, L, L)


def test_x_below_gap_cost_stops_at_first_antidiagonal():
    # X < |gap|: both cells of d=1 are gap cells below 0 - X, so the sweep
    # ends after computing them, whatever follows.
    a = b"ACGTACGT"
    for X in (0,):
        assert oracle.extend(a, a, 1, -1, -1, X) == (0, 0, 0, 2)
    assert oracle.extend(a, a, 2, -3, -2, 1) == (0, 0, 0, 2)


@pytest.mark.parametrize("X", [0, 1, 2, 5, 13, 40])
def test_disjoint_alphabets_closed_form(X):
    # a all A, b all C, +1/-1/-1: S(i,j) = -max(i,j), live iff max(i,j) <= X.
    # The live set of d is [d-X, X]; the evaluated range is one wider on top,
    # giving sum_{d=1}^{2X+1} (min(d,X+1) - max(0,d-1-X) + 1) = (X+1)(X+3)-1
    # cells when both sequences have at least X+1 bases.
    L = X + 1 + 5
    best, bi, bj, cells = oracle.extend(b"A" * L, b"C" * L, 1, -1, -1, X)
    assert (best, bi, bj) == (0, 0, 0)
    assert cells == (X + 1) * (X + 3) - 1


@pytest.mark.parametrize("n", [0, 1, 5, 60])
@pytest.mark.parametrize("X,G", [(0, -1), (3, -1), (10, -1), (7, -2), (9, -3)])
def test_empty_side(n, X, G):
    # m = 0: the only cells are (0,d) = d*G, live while d*|G| <= X.
    exp = 0 if n == 0 else min(n, X // abs(G) + 1)
    assert oracle.extend(b"", b"G" * n, 1, -1, G, X) == (0, 0, 0, exp)
    assert oracle.extend(b"T" * n, b"", 1, -1, G, X) == (0, 0, 0, exp)


def test_unrelated_pairs_terminate_early():
    # Sec. III: X-drop stops early when the sequences do not align -- when
    # the scoring makes unrelated DNA drift downwards.  With +1/-2/-2 a
    # random pair dies within a few anti-diagonals.  With +1/-1/-1 random
    # DNA has a positive optimal-alignment drift (about +0.1 per base), so
    # the sweep runs through the matrix with a band that stays narrow
    # compared with the matrix.
    rng = np.random.default_rng(11)
    a = rand_seq(rng, 3000)
    b = rand_seq(rng, 3000)
    for X in (5, 10, 20):
        best, bi, bj, cells = oracle.extend(a, b, 1, -2, -2, X)
        assert best == 0 and cells < 0.001 * 3000 * 3000
    best, bi, bj, cells = oracle.extend(a, b, 1, -1, -1, 10)
    assert best > 0 and cells < 0.05 * 3000 * 3000


def test_x_monotonicity_counterexample():
    # Under this reading the best score is NOT monotone in X: a larger X lets
    # a faster path lift `best` early, which then prunes a slower path that a
    # smaller X keeps.
    a, b = b"ACACCCACCACA", b"CAACACCACAC"
    assert oracle.extend(a, b, 1, -1, -1, 1)[0] == 6
    assert oracle.extend(a, b, 1, -1, -1, 2)[0] == 5
    # beyond the largest possible drop, X-drop equals the full DP
    assert oracle.extend(a, b, 1, -1, -1, 1000)[0] == full_dp(a, b, 1, -1, -1)[0]


def _golden():
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        yield lhs.split(), [int(v) for v in rhs.split()]


def test_worked_examples():
    n = 0
    for lhs, exp in _golden():
        if lhs[0] == "EXT":
            a, b = lhs[1].encode(), lhs[2].encode()
            M, MM, G, X = map(int, lhs[3:7])
            assert list(oracle.extend(a, b, M, MM, G, X)) == exp, lhs
        else:
            A, B = lhs[1].encode(), lhs[2].encode()
            posA, posB, k, M, MM, G, X = map(int, lhs[3:10])
            r = oracle.pair(A, B, posA, posB, k, M, MM, G, X)
            got = [int(r[f]) for f in ("score", "left", "right", "begA", "begB", "endA",
                                       "endB", "cells")]
            assert int(r["status"]) == oracle.OK
            assert got == exp, lhs
        n += 1
    assert n >= 5


def test_pair_left_side_reads_backwards():
    # the left extension of (A,B) at (posA,posB) is the extension of the
    # reversed prefixes; check against a direct call
    rng = np.random.default_rng(5)
    for _ in range(50):
        A = rand_seq(rng, rng.integers(20, 80))
        B = bytearray(A)
        for p in np.flatnonzero(rng.random(len(B)) < 0.1):
            B[p] = ord("ACGT"[int(rng.integers(4))])
        B = bytes(B)
        k = int(rng.integers(0, 10))
        posA = int(rng.integers(0, len(A) - k + 1))
        posB = int(rng.integers(0, len(B) - k + 1))
        X = int(rng.integers(0, 20))
        r = oracle.pair(A, B, posA, posB, k, 1, -1, -1, X)
        L = oracle.extend(A[:posA][::-1], B[:posB][::-1], 1, -1, -1, X)
        R = oracle.extend(A[posA + k:], B[posB + k:], 1, -1, -1, X)
        seed = sum(1 if A[posA + t] == B[posB + t] else -1 for t in range(k))
        assert int(r["left"]) == L[0] and int(r["right"]) == R[0]
        assert int(r["score"]) == L[0] + seed + R[0]
        assert (int(r["begA"]), int(r["begB"])) == (posA - L[1], posB - L[2])
        assert (int(r["endA"]), int(r["endB"])) == (posA + k + R[1], posB + k + R[2])
        assert int(r["cells"]) == L[3] + R[3]


def test_validation():
    assert oracle.pair(b"ACGT", b"ACGT", 0, 0, 4, 1, -1, -1, 5)["status"] == oracle.OK
    assert oracle.pair(b"ACNT", b"ACGT", 0, 0, 2, 1, -1, -1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"acgt", 0, 0, 2, 1, -1, -1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 1, 0, 4, 1, -1, -1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 0, 1, 4, 1, -1, -1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 0, 0, 0, 1, -1, 1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 0, 0, 0, 1, 2, -1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 0, 0, 0, 1, -1, -1, -1)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 0, 0, 0, 1001, -1, -1, 5)["status"] == oracle.INVALID
    assert oracle.pair(b"ACGT", b"ACGT", 0, 0, 0, 1, -1, -1, 1 << 29)["status"] == oracle.INVALID
    assert oracle.params_valid(1, -1, -1, 1 << 29)
    assert not oracle.params_valid(1, -1, -1, (1 << 29) + 1)


def test_batch_matches_single_pairs():
    from paper_2002_05200_gb300 import synth
    b = synth.tiny_pairs(400, 30, seed=9)
    res, used = oracle.run_batch(b, threads=4)
    assert used >= 1
    for p in range(b.n_pairs):
        s = b.seeds[p]
        r = oracle.pair(b.seqA(p), b.seqB(p), int(s["posA"]), int(s["posB"]), int(s["len"]),
                        b.match, b.mismatch, b.gap, int(b.Xs[p]))
        assert tuple(r) == tuple(res[p])


def _sweep_dicts(a: bytes, b: bytes, M: int, MM: int, G: int, X: int):
    """X-drop sweep kept as one dict {i: score} of live cells per
    anti-diagonal (readings R1-R10), written apart from the C oracle's
    arrays: a cross-check of its bookkeeping, not a pin."""
    m, n = len(a), len(b)
    live = {0: {0: 0}}     # d -> {i: score} of live cells
    rng = {0: (0, 0)}      # d -> stored (trimmed) range
    best, bi, bj, cells = 0, 0, 0, 0
    for d in range(1, m + n + 1):
        lo1, hi1 = rng[d - 1]
        lo, hi = max(lo1, d - n), min(hi1 + 1, m)
        if lo > hi:
            break
        cur = {}
        for i in range(lo, hi + 1):
            j = d - i
            terms = []
            if i > 0 and j > 0 and d >= 2 and (i - 1) in live[d - 2]:
                terms.append(live[d - 2][i - 1] + (M if a[i - 1] == b[j - 1] else MM))
            if i > 0 and (i - 1) in live[d - 1]:
                terms.append(live[d - 1][i - 1] + G)
            if j > 0 and i in live[d - 1]:
                terms.append(live[d - 1][i] + G)
            if terms and max(terms) >= best - X:
                cur[i] = max(terms)
        cells += hi - lo + 1
        if not cur:
            break
        top = max(cur.values())
        if top > best:
            best = top
            bi = min(i for i, v in cur.items() if v == top)
            bj = d - bi
        live[d] = cur
        rng[d] = (min(cur), max(cur))
    return best, bi, bj, cells


@pytest.mark.parametrize("scheme", [(1, -1, -1), (2, -3, -2), (1, -1, 0)])
def test_finite_x_matches_dict_sweep(scheme):
    M, MM, G = scheme
    rng = np.random.default_rng(31)
    for _ in range(4000):
        m, n = (int(v) for v in rng.integers(0, 13, size=2))
        alpha = np.frombuffer(b"AC", np.uint8)
        a = alpha[rng.integers(0, 2, m)].tobytes()
        b = alpha[rng.integers(0, 2, n)].tobytes()
        X = int(rng.integers(0, 9))
        assert tuple(oracle.extend(a, b, M, MM, G, X)) == _sweep_dicts(a, b, M, MM, G, X), \
            (a, b, X)
