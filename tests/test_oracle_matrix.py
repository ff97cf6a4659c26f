"""Pins of the substitution-matrix oracle (oracle/xdrop_matrix_oracle.c)
against what the mathematics fixes, independently of the oracle's own code:

* the 4 x 4 match / mismatch matrix over A C G T gives exactly the affine
  DNA oracle's results (and the linear oracle's at gap_open = 0), every
  field, with finite X -- this pins the pruning, trimming and existence
  rules through two independently written files;
* at unbounded X the extension is a textbook full-matrix Gotoh DP written
  out here (row-major, every cell): best score, its cell under the tie rule
  (first anti-diagonal, then smallest row), and (m+1)(n+1)-1 cells;
* closed forms: identical sequences under a matrix whose off-diagonal
  entries never beat the diagonal ones (BLOSUM62 is one) score the sum of
  their diagonal entries at (L, L); an empty side scores 0;
* invariants of random protein pairs; the BLOSUM62 table's symmetry and
  its published diagonal.
"""
import numpy as np
import pytest

import oracle
from paper_2002_05200_gb300 import synth

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
BIG = 1 << 29


def codes(s: bytes) -> bytes:
    return bytes(CODE[c] for c in s)


def gotoh_full(a: bytes, b: bytes, M, o: int, e: int):
    """Textbook Gotoh over the whole (m+1) x (n+1) matrix, row by row.
    Returns (best, bi, bj) with best >= 0 starting at (0,0) and the tie rule
    of the extension: the smallest anti-diagonal i+j, then the smallest i."""
    NEG = -(1 << 60)
    m, n = len(a), len(b)
    H = [[NEG] * (n + 1) for _ in range(m + 1)]
    E = [[NEG] * (n + 1) for _ in range(m + 1)]
    F = [[NEG] * (n + 1) for _ in range(m + 1)]
    H[0][0] = 0
    for i in range(m + 1):
        for j in range(n + 1):
            if i == 0 and j == 0:
                continue
            if j > 0:
                E[i][j] = max(E[i][j - 1] + e, H[i][j - 1] + o + e)
            if i > 0:
                F[i][j] = max(F[i - 1][j] + e, H[i - 1][j] + o + e)
            h = max(E[i][j], F[i][j])
            if i > 0 and j > 0:
                h = max(h, H[i - 1][j - 1] + int(M[a[i - 1]][b[j - 1]]))
            H[i][j] = h
    best, bi, bj = 0, 0, 0
    for d in range(m + n + 1):
        for i in range(max(0, d - n), min(d, m) + 1):
            if H[i][d - i] > best:
                best, bi, bj = H[i][d - i], i, d - i
    return best, bi, bj


def test_blosum62_table():
    M = synth.BLOSUM62
    assert M.shape == (20, 20) and np.array_equal(M, M.T)
    # the published diagonal, A R N D C Q E G H I L K M F P S T W Y V
    assert list(np.diag(M)) == [4, 5, 6, 6, 9, 5, 5, 6, 8, 4, 4, 5, 5, 6, 7, 4, 5, 11, 7, 4]
    assert M.max() == 11 and M.min() == -4


@pytest.mark.parametrize("match,mismatch,go,ge", [(1, -1, -2, -1), (2, -3, -5, -2),
                                                  (1, -1, 0, -1), (5, -4, -10, -1)])
def test_dna_matrix_equals_affine_oracle(match, mismatch, go, ge):
    M = synth.dna_matrix(match, mismatch)
    b = synth.tiny_pairs(800, 60, seed=41, X_choices=(0, 1, 3, 8, 20, 100))
    for p in range(b.n_pairs):
        s = b.seeds[p]
        A, B = b.seqA(p), b.seqB(p)
        X = int(b.Xs[p])
        args = (int(s["posA"]), int(s["posB"]), int(s["len"]))
        got = oracle.matrix_pair(codes(A), codes(B), *args, M, go, ge, X)
        want = oracle.affine_pair(A, B, *args, match, mismatch, go, ge, X)
        assert tuple(got) == tuple(want), (p, got, want)
        if go == 0:
            assert tuple(got) == tuple(oracle.pair(A, B, *args, match, mismatch, ge, X)), p


@pytest.mark.parametrize("seed", range(3))
def test_unbounded_x_is_full_gotoh(seed):
    rng = np.random.default_rng(seed)
    for t in range(60):
        K = int(rng.integers(2, 21))
        M = rng.integers(-6, 7, size=(K, K)).astype(np.int32)
        m, n = int(rng.integers(0, 14)), int(rng.integers(0, 14))
        a = bytes(rng.integers(0, K, size=m).astype(np.uint8))
        b = bytes(rng.integers(0, K, size=n).astype(np.uint8))
        o, e = int(rng.integers(-6, 1)), int(rng.integers(-3, 1))
        best, bi, bj, cells = oracle.matrix_extend(a, b, M, o, e, BIG)
        assert (best, bi, bj) == gotoh_full(a, b, M, o, e), (t, K, m, n, o, e)
        assert cells == (m + 1) * (n + 1) - 1


def test_identical_sequences_and_empty_side():
    M = synth.BLOSUM62
    # the identity alignment is optimal when no pair beats the mean of its
    # two diagonal entries
    K = M.shape[0]
    assert all(2 * M[x][y] <= M[x][x] + M[y][y] for x in range(K) for y in range(K))
    rng = np.random.default_rng(5)
    for L in (1, 7, 40, 300):
        a = bytes(rng.integers(0, 20, size=L).astype(np.uint8))
        want = int(sum(M[c][c] for c in a))
        assert oracle.matrix_extend(a, a, M, -11, -1, 60)[:3] == (want, L, L)
    b = bytes(rng.integers(0, 20, size=30).astype(np.uint8))
    best, bi, bj, cells = oracle.matrix_extend(b"", b, M, -11, -1, 20)
    assert (best, bi, bj) == (0, 0, 0)
    # only cells (0, j): -11 - j after j steps survives while >= -20
    assert cells == 10


def test_protein_pair_invariants():
    b = synth.protein_pairs(200, lo=30, hi=400, seed=3)
    M = synth.BLOSUM62
    r, _ = oracle.run_batch_matrix(b, M, -11, -1)
    assert np.all(r["status"] == oracle.OK)
    k = b.seeds["len"].astype(np.int64)
    seed_score = np.array([sum(int(M[b.poolA[b.offA[s["idxA"]] + s["posA"] + t]]
                                   [b.poolB[b.offB[s["idxB"]] + s["posB"] + t]])
                               for t in range(int(s["len"]))) for s in b.seeds])
    assert np.array_equal(r["score"], r["left"] + seed_score + r["right"])
    assert np.all(r["left"] >= 0) and np.all(r["right"] >= 0)
    lA = b.lenA[b.seeds["idxA"]].astype(np.int64)
    lB = b.lenB[b.seeds["idxB"]].astype(np.int64)
    assert np.all((r["begA"] >= 0) & (r["endA"] <= lA) & (r["begB"] >= 0) & (r["endB"] <= lB))
    assert np.all(r["endA"] >= b.seeds["posA"].astype(np.int64) + k)
    # related pairs extend well past their seeds
    rel = b.meta["related"]
    assert np.median(r["score"][rel]) > 3 * np.median(r["score"][~rel])


def test_validation():
    M = synth.BLOSUM62
    assert oracle.matrix_params_valid(M, -11, -1, 50)
    assert not oracle.matrix_params_valid(M, 1, -1, 50)
    assert not oracle.matrix_params_valid(M, -11, -1, -1)
    assert not oracle.matrix_params_valid(np.full((2, 2), 1001, np.int32), 0, -1, 5)
    # a letter code outside the alphabet makes the pair invalid
    r = oracle.matrix_pair(bytes([0, 1, 20]), bytes([0, 1, 2]), 0, 0, 1, M, -11, -1, 10)
    assert r["status"] == oracle.INVALID
