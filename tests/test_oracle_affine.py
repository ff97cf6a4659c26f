"""Pins of the affine-gap oracle (CPU only).

The affine extension restates the paper's X-drop sweep (Sec. III-A,
Algorithms 1-2) with Gotoh's three-state recurrence.  It is pinned by:
  * gap_open = 0: the recurrence reduces to the linear one, so every field
    equals the (separately pinned) linear oracle's;
  * X beyond any drop: a textbook row-major Gotoh DP over the whole matrix
    (written here, free end): best, the cell (first anti-diagonal, then
    smallest i) and (m+1)(n+1)-1 cells;
  * closed forms: identical sequences, an empty side;
  * invariants: best <= full DP, monotone in the gap penalties at X = inf.
"""
import itertools

import numpy as np
import pytest

import oracle

INF_X = 1 << 29


def gotoh_full(a: bytes, b: bytes, match, mismatch, go, ge):
    """Row-major full-matrix Gotoh DP; returns (best, bi, bj) with the
    best cell chosen by anti-diagonal, then row."""
    m, n = len(a), len(b)
    NEG = None
    H = [[NEG] * (n + 1) for _ in range(m + 1)]
    E = [[NEG] * (n + 1) for _ in range(m + 1)]
    F = [[NEG] * (n + 1) for _ in range(m + 1)]

    def mx(*v):
        v = [x for x in v if x is not None]
        return max(v) if v else None

    def add(x, y):
        return None if x is None else x + y

    H[0][0] = 0
    for i in range(m + 1):
        for j in range(n + 1):
            if i == 0 and j == 0:
                continue
            E[i][j] = mx(add(E[i][j - 1], ge), add(H[i][j - 1], go + ge)) if j > 0 else None
            F[i][j] = mx(add(F[i - 1][j], ge), add(H[i - 1][j], go + ge)) if i > 0 else None
            diag = add(H[i - 1][j - 1], match if a[i - 1] == b[j - 1] else mismatch) \
                if i > 0 and j > 0 else None
            H[i][j] = mx(diag, E[i][j], F[i][j])
    best, bi, bj = 0, 0, 0
    for d in range(1, m + n + 1):
        for i in range(max(0, d - n), min(m, d) + 1):
            v = H[i][d - i]
            if v is not None and v > best:
                best, bi, bj = v, i, d - i
    return best, bi, bj


SCHEMES = [(1, -1, -2, -1), (2, -3, -5, -2), (1, -1, 0, -1), (3, 1, -4, 0), (5, -4, -10, -1)]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_unbounded_x_equals_full_gotoh_exhaustive(scheme):
    match, mismatch, go, ge = scheme
    words = [b""] + [bytes(w) for L in range(1, 4) for w in itertools.product(b"ACGT", repeat=L)]
    rng = np.random.default_rng(7)
    for a in words[::3]:
        for b in words[::5]:
            best, bi, bj, cells = oracle.affine_extend(a, b, match, mismatch, go, ge, INF_X)
            assert (best, bi, bj) == gotoh_full(a, b, match, mismatch, go, ge), (a, b)
            assert cells == (len(a) + 1) * (len(b) + 1) - 1
    del rng


@pytest.mark.parametrize("scheme", SCHEMES)
def test_unbounded_x_equals_full_gotoh_random(scheme):
    match, mismatch, go, ge = scheme
    rng = np.random.default_rng(11)
    for _ in range(60):
        m, n = rng.integers(0, 25, size=2)
        alpha = np.frombuffer(b"ACGT" if rng.random() < 0.5 else b"AC", np.uint8)
        a = bytes(alpha[rng.integers(0, alpha.size, m)])
        b = bytes(alpha[rng.integers(0, alpha.size, n)])
        best, bi, bj, cells = oracle.affine_extend(a, b, match, mismatch, go, ge, INF_X)
        assert (best, bi, bj) == gotoh_full(a, b, match, mismatch, go, ge), (a, b)
        assert cells == (m + 1) * (n + 1) - 1


def test_zero_open_equals_linear_extension():
    rng = np.random.default_rng(3)
    for _ in range(400):
        m, n = rng.integers(0, 60, size=2)
        alpha = np.frombuffer(b"ACGT" if rng.random() < 0.6 else b"AC", np.uint8)
        a = bytes(alpha[rng.integers(0, alpha.size, m)])
        b = bytes(alpha[rng.integers(0, alpha.size, n)])
        match = int(rng.integers(1, 4))
        mismatch = int(rng.integers(-4, match + 1))
        gap = int(rng.integers(-4, 1))
        X = int(rng.choice([0, 1, 2, 3, 5, 8, 20, 100]))
        assert oracle.affine_extend(a, b, match, mismatch, 0, gap, X) == \
            oracle.extend(a, b, match, mismatch, gap, X), (a, b, match, mismatch, gap, X)


def test_zero_open_pair_equals_linear_pair():
    rng = np.random.default_rng(5)
    for _ in range(200):
        lA, lB = rng.integers(0, 80, size=2)
        A = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, lA)])
        B = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, lB)])
        k = int(rng.integers(0, min(lA, lB) + 1)) if min(lA, lB) else 0
        pA = int(rng.integers(0, lA - k + 1))
        pB = int(rng.integers(0, lB - k + 1))
        X = int(rng.choice([0, 3, 10, 50]))
        r1 = oracle.affine_pair(A, B, pA, pB, k, 1, -1, 0, -2, X)
        r2 = oracle.pair(A, B, pA, pB, k, 1, -1, -2, X)
        assert r1.tobytes() == r2.tobytes()


@pytest.mark.parametrize("L", [1, 7, 40])
def test_identical_sequences(L):
    rng = np.random.default_rng(L)
    a = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, L)])
    for go, ge in ((-3, -1), (0, 0), (-10, -2)):
        best, bi, bj, _ = oracle.affine_extend(a, a, 2, -3, go, ge, 25)
        assert (best, bi, bj) == (2 * L, L, L)


@pytest.mark.parametrize("go,ge,X,n", [(-2, -1, 5, 10), (-2, -1, 1, 10), (-6, -1, 5, 10),
                                        (0, 0, 3, 9), (-3, 0, 5, 4), (-3, -2, 100, 7)])
def test_empty_side_closed_form(go, ge, X, n):
    # m = 0: only cells (0, j), H = go + j*ge; the first pruned one is counted
    b = b"ACGTACGTACGT"[:n]
    best, bi, bj, cells = oracle.affine_extend(b"", b, 1, -1, go, ge, X)
    assert (best, bi, bj) == (0, 0, 0)
    live = [j for j in range(1, n + 1) if go + j * ge >= -X]
    # live cells are a prefix 1..J (scores only fall with j)
    J = len(live)
    assert live == list(range(1, J + 1))
    assert cells == min(n, J + 1)


def test_invariants_random():
    rng = np.random.default_rng(9)
    for _ in range(80):
        m, n = rng.integers(0, 20, size=2)
        a = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, m)])
        b = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)])
        go, ge = int(rng.integers(-6, 1)), int(rng.integers(-3, 1))
        X = int(rng.choice([0, 2, 5, 12]))
        best, bi, bj, cells = oracle.affine_extend(a, b, 1, -1, go, ge, X)
        full = gotoh_full(a, b, 1, -1, go, ge)[0]
        assert 0 <= best <= full
        assert 0 <= bi <= m and 0 <= bj <= n
        assert 0 <= cells <= (m + 1) * (n + 1) - 1
        # harsher gaps never raise the unpruned best
        assert gotoh_full(a, b, 1, -1, go - 2, ge)[0] <= full
        assert gotoh_full(a, b, 1, -1, go, ge - 1)[0] <= full


def test_validation():
    assert oracle.affine_params_valid(1, -1, -2, -1, 50)
    assert oracle.affine_params_valid(1, -1, 0, 0, 0)
    assert not oracle.affine_params_valid(1, -1, 1, -1, 50)      # open > 0
    assert not oracle.affine_params_valid(1, -1, -2, 1, 50)      # extend > 0
    assert not oracle.affine_params_valid(1, 2, -2, -1, 50)      # mismatch > match
    assert not oracle.affine_params_valid(1, -1, -1001, -1, 50)  # |open| > 1000
    assert not oracle.affine_params_valid(1, -1, -2, -1, -1)     # X < 0
    r = oracle.affine_pair(b"ACGN", b"ACGT", 0, 0, 0, 1, -1, -2, -1, 10)
    assert r["status"] == oracle.INVALID


def _affine_sweep_dicts(a, b, M, MM, go, ge, X):
    """The affine X-drop sweep with one dict {i: (H, E, F)} of live cells per
    anti-diagonal (None = -infinity), written apart from the C oracle's
    arrays and existence flags: a cross-check, not a pin."""
    m, n = len(a), len(b)

    def mx(*v):
        v = [x for x in v if x is not None]
        return max(v) if v else None

    live = {0: {0: (0, None, None)}}
    rng = {0: (0, 0)}
    best, bi, bj, cells = 0, 0, 0, 0
    for d in range(1, m + n + 1):
        lo1, hi1 = rng[d - 1]
        lo, hi = max(lo1, d - n), min(hi1 + 1, m)
        if lo > hi:
            break
        cur = {}
        for i in range(lo, hi + 1):
            j = d - i
            left = live[d - 1].get(i) if j > 0 else None     # (i, j-1)
            up = live[d - 1].get(i - 1) if i > 0 else None   # (i-1, j)
            diag = live[d - 2].get(i - 1) if (i > 0 and j > 0 and d >= 2) else None
            E = mx(left[1] + ge if left and left[1] is not None else None,
                   left[0] + go + ge if left else None)
            F = mx(up[2] + ge if up and up[2] is not None else None,
                   up[0] + go + ge if up else None)
            H = mx(diag[0] + (M if a[i - 1] == b[j - 1] else MM) if diag else None, E, F)
            if H is not None and H >= best - X:
                cur[i] = (H, E, F)
        cells += hi - lo + 1
        if not cur:
            break
        top = max(v[0] for v in cur.values())
        if top > best:
            best = top
            bi = min(i for i, v in cur.items() if v[0] == top)
            bj = d - bi
        live[d] = cur
        rng[d] = (min(cur), max(cur))
    return best, bi, bj, cells


@pytest.mark.parametrize("M,MM,go,ge", [(1, -1, -2, -1), (2, -3, -3, -1), (1, -1, 0, -1),
                                        (1, 0, -1, 0)])
def test_finite_x_matches_dict_sweep(M, MM, go, ge):
    rng = np.random.default_rng(41)
    alpha = np.frombuffer(b"AC", np.uint8)
    for _ in range(3000):
        m, n = (int(v) for v in rng.integers(0, 12, size=2))
        a = alpha[rng.integers(0, 2, m)].tobytes()
        b = alpha[rng.integers(0, 2, n)].tobytes()
        X = int(rng.integers(0, 9))
        assert tuple(oracle.affine_extend(a, b, M, MM, go, ge, X)) == \
            _affine_sweep_dicts(a, b, M, MM, go, ge, X), (a, b, X)
