"""Pins of the traceback oracle (CPU only): at unbounded X its path equals
a textbook full-matrix DP traceback with the same tie rule; at any X the
path consumes exactly the best cell's bases and rescores to the best score;
its extension fields equal the (separately pinned) extension oracle's; a
pair's path spans the pair's reported coordinates and rescores to its
score."""
import numpy as np
import pytest

import oracle

INF_X = 1 << 29


def full_dp_path(a, b, match, mismatch, gap):
    m, n = len(a), len(b)
    H = np.full((m + 1, n + 1), 0, dtype=np.int64)
    for i in range(m + 1):
        for j in range(n + 1):
            if i == 0 and j == 0:
                continue
            c = []
            if i and j:
                c.append(H[i - 1, j - 1] + (match if a[i - 1] == b[j - 1] else mismatch))
            if i:
                c.append(H[i - 1, j] + gap)
            if j:
                c.append(H[i, j - 1] + gap)
            H[i, j] = max(c)
    best, bi, bj = 0, 0, 0
    for d in range(1, m + n + 1):
        for i in range(max(0, d - n), min(m, d) + 1):
            if H[i, d - i] > best:
                best, bi, bj = int(H[i, d - i]), i, d - i
    ops, i, j = [], bi, bj
    while i + j:
        if i and j and H[i - 1, j - 1] + (match if a[i - 1] == b[j - 1] else mismatch) == H[i, j]:
            ops.append("M"); i -= 1; j -= 1
        elif i and H[i - 1, j] + gap == H[i, j]:
            ops.append("I"); i -= 1
        else:
            ops.append("D"); j -= 1
    return best, bi, bj, "".join(reversed(ops))


def rescore(a, b, ops, match, mismatch, gap):
    i = j = s = 0
    for o in ops:
        if o == "M":
            s += match if a[i] == b[j] else mismatch
            i += 1; j += 1
        elif o == "I":
            s += gap; i += 1
        else:
            s += gap; j += 1
    return s, i, j


def rand(rng, n, alpha=b"ACGT"):
    return bytes(np.frombuffer(alpha, np.uint8)[rng.integers(0, len(alpha), n)])


@pytest.mark.parametrize("scheme", [(1, -1, -1), (2, -3, -2), (1, -1, 0), (3, 1, -2)])
def test_unbounded_x_equals_full_dp_traceback(scheme):
    match, mismatch, gap = scheme
    rng = np.random.default_rng(21)
    for _ in range(150):
        m, n = rng.integers(0, 22, size=2)
        alpha = b"ACGT" if rng.random() < 0.5 else b"AC"
        a, b = rand(rng, m, alpha), rand(rng, n, alpha)
        best, bi, bj, cells, ops = oracle.traceback(a, b, match, mismatch, gap, INF_X)
        assert (best, bi, bj, ops) == full_dp_path(a, b, match, mismatch, gap), (a, b)
        assert cells == (m + 1) * (n + 1) - 1


def test_finite_x_paths_rescore_to_best():
    rng = np.random.default_rng(22)
    for _ in range(300):
        m, n = rng.integers(0, 120, size=2)
        a = rand(rng, m)
        b = bytearray(a[:n]) if rng.random() < 0.6 else bytearray(rand(rng, n))
        for t in rng.integers(0, max(len(b), 1), size=len(b) // 8):  # a few edits
            if len(b):
                b[int(t)] = ord("ACGT"[int(rng.integers(0, 4))])
        b = bytes(b)
        match, mismatch, gap = 1, int(rng.integers(-3, 0)), int(rng.integers(-3, 1))
        X = int(rng.choice([0, 1, 3, 8, 20, 60]))
        best, bi, bj, cells, ops = oracle.traceback(a, b, match, mismatch, gap, X)
        assert (best, bi, bj, cells) == oracle.extend(a, b, match, mismatch, gap, X)
        assert rescore(a, b, ops, match, mismatch, gap) == (best, bi, bj)


def test_pair_paths_span_the_reported_coordinates():
    rng = np.random.default_rng(23)
    for _ in range(120):
        L = int(rng.integers(20, 300))
        A = rand(rng, L)
        B = bytearray(A)
        for t in rng.integers(0, L, size=L // 10):
            B[int(t)] = ord("ACGT"[int(rng.integers(0, 4))])
        B = bytes(B)
        k = int(rng.integers(0, 12))
        p = int(rng.integers(0, L - k + 1))
        X = int(rng.choice([5, 20, 100]))
        r = oracle.pair(A, B, p, p, k, 1, -1, -1, X)
        ops = oracle.pair_traceback(A, B, p, p, k, 1, -1, -1, X)
        s, di, dj = rescore(A[r["begA"]:], B[r["begB"]:], ops, 1, -1, -1)
        assert (s, di, dj) == (r["score"], r["endA"] - r["begA"], r["endB"] - r["begB"])


def _path_dicts(a, b, match, mismatch, gap, X):
    """The X-drop sweep with one dict {i: (score, how)} of live cells per
    anti-diagonal (how: 'M' diagonal, 'I' vertical, 'D' horizontal, the
    first in that order among the terms giving the score), and the walk
    back from the best cell: a cross-check of the oracle's tie rule and
    walk at finite X, not a pin."""
    m, n = len(a), len(b)
    live = {0: {0: (0, None)}}
    rng = {0: (0, 0)}
    best, bi, bj = 0, 0, 0
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
                terms.append((live[d - 2][i - 1][0] + (match if a[i - 1] == b[j - 1] else mismatch),
                              "M"))
            if i > 0 and (i - 1) in live[d - 1]:
                terms.append((live[d - 1][i - 1][0] + gap, "I"))
            if j > 0 and i in live[d - 1]:
                terms.append((live[d - 1][i][0] + gap, "D"))
            if terms:
                s = max(t[0] for t in terms)
                if s >= best - X:
                    cur[i] = (s, next(h for v, h in terms if v == s))
        if not cur:
            break
        top = max(v[0] for v in cur.values())
        if top > best:
            best = top
            bi = min(i for i, v in cur.items() if v[0] == top)
            bj = d - bi
        live[d] = cur
        rng[d] = (min(cur), max(cur))
    ops, i, j = [], bi, bj
    while i + j:
        h = live[i + j][i][1]
        ops.append(h)
        if h == "M":
            i, j = i - 1, j - 1
        elif h == "I":
            i -= 1
        else:
            j -= 1
    return best, bi, bj, "".join(reversed(ops))


@pytest.mark.parametrize("scheme", [(1, -1, -1), (2, -3, -2), (1, -1, 0)])
def test_finite_x_paths_match_dict_sweep(scheme):
    match, mismatch, gap = scheme
    rng = np.random.default_rng(51)
    for _ in range(3000):
        m, n = (int(v) for v in rng.integers(0, 13, size=2))
        a, b = rand(rng, m, b"AC"), rand(rng, n, b"AC")
        X = int(rng.integers(0, 9))
        best, bi, bj, _, ops = oracle.traceback(a, b, match, mismatch, gap, X)
        assert (best, bi, bj, ops) == _path_dicts(a, b, match, mismatch, gap, X), (a, b, X)
