"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics.

Nothing here compares the oracle with itself: every expected value is either
printed in the paper (fixtures under tests/golden), a closed form, an
invariant, or a brute-force enumeration written independently below.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import inputs

NEG = oracle.NEG_INF
INF = oracle.INF


# ---------------------------------------------------------------- brute force
def is_subsequence(s, t):
    it = iter(t)
    return all(ch in it for ch in s)


def brute_lcs_len(x, y):
    """Longest subsequence of the shorter string that is a subsequence of the
    other, by enumerating every subset (strings of length <= 12)."""
    x, y = bytes(x), bytes(y)
    if len(x) > len(y):
        x, y = y, x
    best = 0
    for mask in range(1 << len(x)):
        pc = bin(mask).count("1")
        if pc <= best:
            continue
        s = bytes(x[i] for i in range(len(x)) if mask >> i & 1)
        if is_subsequence(s, y):
            best = pc
    return best


def brute_dist(a, b):
    n = len(b)
    D = np.full((n + 1, n + 1), NEG, dtype=np.int64)
    for i in range(n + 1):
        for j in range(i, n + 1):
            D[i, j] = brute_lcs_len(a, b[i:j])
    return D


def optimal_paths(a, b):
    """Every heaviest source->sink path of the grid graph (Fig. 1 rules: right
    and down edges weigh 0, a diagonal exists only on a match and weighs 1),
    as the list of entry columns per row (the cross vertices v[0..m])."""
    m, n = len(a), len(b)
    best = {}

    def longest(r, c):                     # heaviest weight from (r, c) to (m, n)
        if (r, c) in best:
            return best[(r, c)]
        w = -1
        if r == m and c == n:
            w = 0
        if c < n:
            w = max(w, longest(r, c + 1))
        if r < m:
            w = max(w, longest(r + 1, c))
        if r < m and c < n and a[r] == b[c]:
            w = max(w, 1 + longest(r + 1, c + 1))
        best[(r, c)] = w
        return w

    total = longest(0, 0)
    paths = []

    def walk(r, c, acc, entries):
        if r == m and c == n:
            paths.append(tuple(entries))
            return
        rem = best[(r, c)]
        if c < n and longest(r, c + 1) == rem:
            walk(r, c + 1, acc, entries)
        if r < m and longest(r + 1, c) == rem:
            walk(r + 1, c, acc, entries + [c])
        if r < m and c < n and a[r] == b[c] and 1 + longest(r + 1, c + 1) == rem:
            walk(r + 1, c + 1, acc + 1, entries + [c + 1])

    walk(0, 0, 0, [0])
    return total, paths


def small_pairs(seed, count, lo=0, hi=9, alphabet=b"ACGT"):
    rng = np.random.default_rng(seed)
    alph = np.frombuffer(alphabet, dtype=np.uint8)
    for _ in range(count):
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        yield bytes(inputs.uniform(rng, m, alph)), bytes(inputs.uniform(rng, n, alph))


# ---------------------------------------------------------------- the paper
def test_intro_example(golden):
    """Sec. I: the LCS of abccb, abba and acbb is abb (so each pair has an LCS
    of length >= 3, and brute force shows exactly 3)."""
    g = golden("intro_example.txt")
    strings = g["strings"].split()
    lcs_all = g["lcs_of_all"].encode()
    for s in strings:
        assert is_subsequence(lcs_all, s.encode())
    for x, y in itertools.combinations(strings, 2):
        assert oracle.lcs_length(x, y) == brute_lcs_len(x.encode(), y.encode()) == 3
        s, _ = oracle.traceback(x, y)
        assert len(s) == 3 and is_subsequence(s, x.encode()) and is_subsequence(s, y.encode())


def test_fig1_breakouts(golden):
    """Sec. II-B-1: the breakouts of top vertex (1,1) are the bottom vertices
    (9,2),(9,3),(9,4),(9,5),(9,13); top vertex (1,8) has no 5th breakout."""
    g = golden("fig1_breakouts.txt")
    a, b = g["rows"], g["cols"]
    D = oracle.dist(a, b)
    F = oracle.dform(D, len(a))
    cols_1based = [int(x) for x in g["breakouts_of_1_1"].split()]
    assert [int(F[0, w]) + 1 for w in range(1, 6)] == cols_1based
    assert F[0, 6] == INF                    # the LCS of the pair is 5
    w_missing = int(g["no_breakout_of_1_8"])
    assert F[7, w_missing] == INF and F[7, w_missing - 1] != INF
    # DIST(0, .) in the DIST form follows from the breakouts alone.
    expect = [max(w for w in range(6) if F[0, w] <= j) for j in range(len(b) + 1)]
    assert D[0].tolist() == expect
    assert oracle.lcs_length(a, b) == 5


def test_leaf_worked_example(golden):
    """Sec. II-B-3: D_{G_1} for a_1 = t over gatttatgcagg."""
    g = golden("leaf_dg1.txt")
    b = g["cols"].encode()
    ah = ord(g["letter"])
    D, gaps = oracle.leaf_dform(ah, b)
    parse = lambda s: [None if t == "x" else (INF if t == "inf" else int(t)) for t in s.split()]
    want_gaps = parse(g["after_gaps"])
    assert [int(x) if x else None for x in gaps] == want_gaps
    assert D.tolist() == parse(g["final"])
    matches = [j + 1 for j in range(len(b)) if b[j] == ah]
    assert matches == [int(x) for x in g["match_positions"].split()]


@pytest.mark.parametrize("seed", range(6))
def test_leaf_construction_equals_definition(seed):
    """The paper's leaf construction (Sec. II-B-3) equals the breakout
    definition applied to the one-row DIST (1-based vertex shift)."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 40))
    b = inputs.uniform(rng, n, inputs.ACGT)
    ah = int(inputs.ACGT[rng.integers(0, 4)])
    D, _ = oracle.leaf_dform(ah, b)
    F = oracle.dform(oracle.dist(bytes([ah]), b), 1)
    want = [INF if F[i, 1] == INF else int(F[i, 1]) + 1 for i in range(n)]
    assert D.tolist() == want


# ---------------------------------------------------------------- length / DIST
@pytest.mark.parametrize("seed", range(4))
def test_length_exhaustive(seed):
    """LCS length against exhaustive subsequence enumeration (<= 12 letters)."""
    for a, b in small_pairs(seed, 40, 0, 12, b"ACG"):
        want = brute_lcs_len(a, b)
        assert oracle.lcs_length(a, b) == want
        if len(b):
            assert oracle.dist(a, b)[0, len(b)] == want


@pytest.mark.parametrize("seed", range(3))
def test_dist_bruteforce(seed):
    """DIST(i, j) = LCS(a, b[i:j]) by enumeration on tiny strings."""
    for a, b in small_pairs(seed + 10, 12, 0, 8, b"AC"):
        assert np.array_equal(oracle.dist(a, b).astype(np.int64), brute_dist(a, b))


def test_dist_rows_match_full():
    rng = np.random.default_rng(7)
    a, b = inputs.random_pair(rng, 37, 53)
    D = oracle.dist(a, b)
    rows = np.array([0, 5, 53, 17], dtype=np.int64)
    assert np.array_equal(oracle.dist_rows(a, b, rows), D[rows])


@pytest.mark.parametrize("seed", range(4))
def test_dist_invariants(seed):
    """Unit steps along rows and columns, bounds 0 <= DIST <= min(m, j-i),
    sentinel below the diagonal, and the Monge inequality
    DIST(i,j) + DIST(i',j') >= DIST(i,j') + DIST(i',j) for i < i' <= j < j'."""
    rng = np.random.default_rng(20 + seed)
    m, n = int(rng.integers(1, 30)), int(rng.integers(1, 30))
    a, b = inputs.random_pair(rng, m, n)
    D = oracle.dist(a, b).astype(np.int64)
    for i in range(n + 1):
        assert D[i, i] == 0
        assert np.all(D[i, :i] == NEG)
        row = D[i, i:]
        assert np.all(np.diff(row) >= 0) and np.all(np.diff(row) <= 1)
        for j in range(i, n + 1):
            assert 0 <= D[i, j] <= min(m, j - i)
    for j in range(n + 1):
        col = D[: j + 1, j]
        assert np.all(-np.diff(col) >= 0) and np.all(-np.diff(col) <= 1)
    for i in range(n + 1):
        for i2 in range(i + 1, n + 1):
            for j in range(i2, n + 1):
                for j2 in range(j + 1, n + 1):
                    assert D[i, j] + D[i2, j2] >= D[i, j2] + D[i2, j]


def test_dist_special_cases():
    rng = np.random.default_rng(3)
    a = inputs.uniform(rng, 25, inputs.ACGT)
    assert oracle.lcs_length(a, a) == 25
    assert oracle.dist(a, a)[0, 25] == 25
    other = np.frombuffer(b"XYZW" * 7, dtype=np.uint8)
    assert oracle.lcs_length(a, other) == 0
    assert np.all(oracle.dist(a, other)[np.triu_indices(29)] == 0)
    assert oracle.lcs_length(b"", b"ACGT") == 0
    D = oracle.dist(b"", b"ACG")
    assert np.all(D[np.triu_indices(4)] == 0)
    assert oracle.dist(b"ACG", b"").tolist() == [[0]]


# ---------------------------------------------------------------- merge
@pytest.mark.parametrize("seed", range(5))
def test_merge_associativity(seed):
    """Sec. II-A: the heaviest path through the boundary row is the best split
    vertex: merge(DIST(a[:s], b), DIST(a[s:], b)) = DIST(a, b) for any s."""
    rng = np.random.default_rng(40 + seed)
    m, n = int(rng.integers(2, 24)), int(rng.integers(0, 24))
    a, b = inputs.random_pair(rng, m, n)
    s = int(rng.integers(0, m + 1))
    D, K = oracle.merge(oracle.dist(a[:s], b), oracle.dist(a[s:], b))
    assert np.array_equal(D, oracle.dist(a, b))


@pytest.mark.parametrize("seed", range(4))
def test_merge_leftmost_argmax_and_knuth_window(seed):
    """K is the smallest maximiser (Algorithm 2 breaks ties to the lower
    index), and the monotonicity that licenses the windowed merge holds:
    K(i, j-1) <= K(i, j) <= K(i+1, j)."""
    rng = np.random.default_rng(60 + seed)
    m, n = int(rng.integers(2, 20)), int(rng.integers(1, 26))
    a, b = inputs.random_pair(rng, m, n, np.frombuffer(b"AB", dtype=np.uint8))
    s = int(rng.integers(1, m))
    U, L = oracle.dist(a[:s], b), oracle.dist(a[s:], b)
    D, K = oracle.merge(U, L)
    for i in range(n + 1):
        for j in range(i, n + 1):
            vals = [int(U[i, k]) + int(L[k, j]) for k in range(i, j + 1)]
            assert D[i, j] == max(vals)
            assert K[i, j] == i + vals.index(max(vals))
            if j > i:
                assert K[i, j - 1] <= K[i, j] <= K[i + 1, j]
        assert np.all(K[i, :i] == -1)


def test_merge_random_monge_matrices():
    """The merge is plain (max,+): check it on random integer matrices too."""
    rng = np.random.default_rng(5)
    n = 9
    U = rng.integers(-5, 6, size=(n + 1, n + 1)).astype(np.int32)
    L = rng.integers(-5, 6, size=(n + 1, n + 1)).astype(np.int32)
    D, K = oracle.merge(U, L)
    for i in range(n + 1):
        for j in range(i, n + 1):
            vals = [int(U[i, k]) + int(L[k, j]) for k in range(i, j + 1)]
            assert D[i, j] == max(vals) and K[i, j] == i + vals.index(max(vals))


# ---------------------------------------------------------------- traceback
@pytest.mark.parametrize("seed", range(5))
def test_traceback_is_leftmost_optimal_path(seed):
    """Sec. II-C..II-E: the cross vertices are those of the leftmost heaviest
    path, i.e. the pointwise minimum over all heaviest paths (itself a heaviest
    path); the letters emitted are a common subsequence of length LCS."""
    for a, b in small_pairs(200 + seed, 25, 0, 7, b"ACG"):
        total, paths = optimal_paths(a, b)
        s, v = oracle.traceback(a, b)
        assert len(s) == total == brute_lcs_len(a, b)
        assert is_subsequence(s, a) and is_subsequence(s, b)
        pointwise = tuple(min(p[r] for p in paths) for r in range(len(a) + 1))
        assert pointwise in set(paths)
        assert tuple(int(x) for x in v) == pointwise


def _tree_traceback(a, b, split):
    """Leftmost argmax down a tree of single-row leaves (Sec. II-D), with DIST
    from brute force and the split row chosen by ``split`` -- a different
    route to the same cross vertices.  v[m] here is the sink column n (the
    bottom boundary of the last leaf), not the cross vertex of row m."""
    m, n = len(a), len(b)
    v = [None] * (m + 1)
    v[0], v[m] = 0, n

    def rec(r0, r1, i, j):
        if r1 - r0 <= 1:
            return
        s = split(r0, r1)
        U = brute_dist(a[r0:s], b)
        L = brute_dist(a[s:r1], b)
        vals = [U[i, k] + L[k, j] for k in range(i, j + 1)]
        c = i + vals.index(max(vals))
        v[s] = c
        rec(r0, s, i, c)
        rec(s, r1, c, j)

    rec(0, m, 0, n)
    out = bytes(a[r - 1] for r in range(1, m + 1)
                if brute_lcs_len(a[r - 1:r], b[v[r - 1]:v[r]]) == 1)
    return v, out


def heaviest_vertex_paths(a, b):
    """Every heaviest source->sink path as its full vertex list, by
    exhaustive depth-first enumeration of all lattice paths (tiny inputs)."""
    m, n = len(a), len(b)
    found = []

    def walk(r, c, w, verts):
        if r == m and c == n:
            found.append((w, tuple(verts)))
            return
        if c < n:
            walk(r, c + 1, w, verts + [(r, c + 1)])
        if r < m:
            walk(r + 1, c, w, verts + [(r + 1, c)])
        if r < m and c < n and a[r] == b[c]:
            walk(r + 1, c + 1, w + 1, verts + [(r + 1, c + 1)])

    walk(0, 0, 0, [(0, 0)])
    top = max(w for w, _ in found)
    return top, [p for w, p in found if w == top]


@pytest.mark.parametrize("seed", range(4))
def test_path_listing_is_leftmost_heaviest_path(seed):
    """Sec. II-D: the listed vertices form the heaviest path whose run in
    every row starts and ends at the smallest columns any heaviest path uses
    there (found by enumerating every lattice path of tiny grids)."""
    for a, b in small_pairs(700 + seed, 20, 0, 6, b"ACG"):
        m, n = len(a), len(b)
        total, paths = heaviest_vertex_paths(a, b)

        def runs(p):
            first, last = {}, {}
            for r, c in p:
                first.setdefault(r, c)
                last[r] = c
            return tuple((first[r], last[r]) for r in range(m + 1))

        lo = tuple((min(runs(p)[r][0] for p in paths), min(runs(p)[r][1] for p in paths)) for r in range(m + 1))
        leftmost = [p for p in paths if runs(p) == lo]
        assert len(leftmost) == 1
        got = oracle.path(a, b)
        assert [tuple(int(x) for x in v) for v in got] == list(leftmost[0])
        assert len(got) == m + n + 1 - total


@pytest.mark.parametrize("seed", range(3))
def test_path_listing_invariants(seed):
    """Larger pairs: the path starts at (0, 0), ends at (m, n), every step is
    right, down or a match diagonal, the diagonals spell the oracle's LCS and
    their number is the exact length."""
    rng = np.random.default_rng(800 + seed)
    for m, n in [(1, 40), (40, 1), (90, 120), (150, 70)]:
        a, b = inputs.random_pair(rng, m, n, np.frombuffer(b"AC" if seed % 2 else b"ACGT", np.uint8))
        P = oracle.path(a, b)
        s, v = oracle.traceback(a, b)
        L = brute_lcs_len(a, b) if min(m, n) <= 12 else oracle.lcs_length(a, b)
        assert tuple(P[0]) == (0, 0) and tuple(P[-1]) == (m, n)
        assert len(P) == m + n + 1 - L
        d = np.diff(P, axis=0)
        steps = {tuple(x) for x in d}
        assert steps <= {(0, 1), (1, 0), (1, 1)}
        diag = np.flatnonzero((d[:, 0] == 1) & (d[:, 1] == 1))
        assert all(a[P[k + 1][0] - 1] == b[P[k + 1][1] - 1] for k in diag)
        assert bytes(a[P[k + 1][0] - 1] for k in diag) == s
        # the first vertex of each row is its cross vertex
        first = {}
        for r, c in P:
            first.setdefault(int(r), int(c))
        assert [first[r] for r in range(m + 1)] == [int(x) for x in v]


@pytest.mark.parametrize("rule", ["mid", "first", "last"])
def test_traceback_tree_independent(rule):
    split = {"mid": lambda r0, r1: (r0 + r1) // 2,
             "first": lambda r0, r1: r0 + 1,
             "last": lambda r0, r1: r1 - 1}[rule]
    for a, b in small_pairs(300, 12, 1, 7, b"AC"):
        v_tree, s_tree = _tree_traceback(a, b, split)
        s, v = oracle.traceback(a, b)
        assert v_tree[:-1] == [int(x) for x in v[:-1]]
        assert s_tree == s


# ---------------------------------------------------------------- D-form
@pytest.mark.parametrize("seed", range(4))
def test_dform_combine_equals_dist_merge(seed):
    """The paper's breakout-matrix combination (Sec. II-B-1) and the DIST
    (max,+) merge describe the same matrix."""
    rng = np.random.default_rng(80 + seed)
    m, n = int(rng.integers(2, 12)), int(rng.integers(1, 20))
    a, b = inputs.random_pair(rng, m, n)
    s = int(rng.integers(1, m))
    U, L = oracle.dist(a[:s], b), oracle.dist(a[s:], b)
    DU, DL = oracle.dform(U, s), oracle.dform(L, m - s)
    D, _ = oracle.merge(U, L)
    assert np.array_equal(oracle.dform_combine(DU, DL), oracle.dform(D, m))


@pytest.mark.parametrize("seed", range(3))
def test_dform_combine_argmin_monotone(seed):
    """Sec. II-B-1: for each top vertex the terms D_L(D_U(i, k), w - k) form a
    monotone matrix -- the leftmost minimising k never decreases as w grows
    -- which is what Algorithm 1's column-minima recursion (and the GPU's
    two-level version of it) relies on.  Checked by brute force over every
    column of random strips."""
    rng = np.random.default_rng(900 + seed)
    for _ in range(6):
        hu, hl, n = int(rng.integers(1, 24)), int(rng.integers(1, 24)), int(rng.integers(0, 60))
        alph = np.frombuffer([b"AC", b"ACGT", bytes(range(20))][int(rng.integers(0, 3))], np.uint8)
        a1, a2, b = inputs.uniform(rng, hu, alph), inputs.uniform(rng, hl, alph), inputs.uniform(rng, n, alph)
        DU, DL = oracle.dform(oracle.dist(a1, b), hu), oracle.dform(oracle.dist(a2, b), hl)
        comb = oracle.dform_combine(DU, DL)
        for i in range(n + 1):
            prev = -1
            for w in range(hu + hl + 1):
                terms = [(int(DL[DU[i, k], w - k]), k) for k in range(min(w, hu) + 1)
                         if w - k <= hl and DU[i, k] != INF]
                best = min(terms)[0] if terms else INF
                assert best == comb[i, w]
                if best == INF:
                    continue
                k = min(k for v, k in terms if v == best)
                assert k >= prev
                prev = k


def test_dform_roundtrip():
    rng = np.random.default_rng(9)
    a, b = inputs.random_pair(rng, 6, 15)
    D = oracle.dist(a, b)
    F = oracle.dform(D, 6)
    for i in range(16):
        assert F[i, 0] == i
        for j in range(i, 16):
            assert D[i, j] == max(w for w in range(7) if F[i, w] <= j)
