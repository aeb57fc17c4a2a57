"""The rules the merge and traceback kernels rest on, checked against the
oracle on small inputs (no GPU).

For a merge D(i, j) = max_k U(i, k) + L(k, j) of two strips' DIST matrices
(Sec. II-A, Sec. II-B-1) with K the smallest maximiser (Algorithm 2's tie
rule), the Monge property makes K monotone in both coordinates and D is
non-increasing in i and non-decreasing in j.  The kernels cut their work with
three consequences, each checked here by brute force over k on tiles of a
grid with a small tile side T (the rules do not depend on T = 64):

* tile band: with kh = K at the tile's far grid corner (clipped to the tile's
  last column) and x the largest maximiser of the near corner that is <= kh,
  every entry (i, j) of the tile keeps a maximiser in [max(x, i), min(kh, j)]
  and its smallest maximiser lies between the corners' K;
* constant tiles: off the diagonal, D(far row, near column) = D(near row, far
  column) makes D constant on the tile;
* traceback window: K at the grid corners around (i, j) bounds K(i, j).

The leaf traceback (Sec. II-C, II-E) takes a strip's part of the path, from
(0, i) to (h, j), without a DP table of pointers: with F(r, c) =
LCS(a[0:r], b[i:c]) and B(r, c) = LCS(a[r:h], b[c:j]) the vertices on
heaviest paths are those with F + B = L = F(h, j), the leftmost heaviest path
enters row r at v[r] = min{c : F(r, c) + B(r, c) = L}, and letter a_r is on
the LCS exactly when v[r] > v[r-1] and a_r = b_{v[r]}.  That is checked
against the oracle's leftmost traceback of the same strip and segment.

The strip builder holds F_j(r) = LCS(a[0:r], b[i:j]) for one source i as an
h-bit vector whose zero bits mark the rows where F steps up, advanced by the
bit-vector step u = V & M, V' = (V + u) | (V & ~M) (Allison-Dix / Hyyro) with
the carry out of the top row the increment of DIST(i, j).  It skips the low
words once they are zero: the first r rows have all stepped exactly when
a[0:r] is a subsequence of b[i:j], zero words stay zero, and a step started
at the first live word with no carry in gives the same vector and carry.
"""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import inputs


def _merge_case(seed):
    rng = np.random.default_rng(900 + seed)
    kind = seed % 4
    n = int(rng.integers(24, 72))
    m = int(rng.integers(4, 40))
    if kind == 0:
        a, b = inputs.random_pair(rng, m, n)
    elif kind == 1:
        a, b = inputs.random_pair(rng, m, n, np.frombuffer(b"AB", dtype=np.uint8))
    elif kind == 2:
        a, b = inputs.zipf20(rng, m), inputs.zipf20(rng, n)
    else:
        # correlated: b is a with substitutions and indels, so long diagonals
        # and wide bands appear
        a = inputs.uniform(rng, m, inputs.ACGT)
        b = inputs.mutate(rng, a, 0.10, 0.05, inputs.ACGT, out_len=n)
    s = int(rng.integers(1, m))
    U = oracle.dist(a[:s], b).astype(np.int64)
    L = oracle.dist(a[s:], b).astype(np.int64)
    D, K = oracle.merge(U, L)
    return n, U, L, D.astype(np.int64), K.astype(np.int64)


def _grid(T, n):
    P = -(-n // T)
    return P, [min(p * T, n) for p in range(P + 1)]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("T", [3, 4, 8])
def test_tile_band_keeps_a_maximiser(seed, T):
    n, U, L, D, K = _merge_case(seed)
    P, g = _grid(T, n)
    for I in range(P):
        for J in range(I, P):
            ia, ja = g[I], g[J]
            rows = range(ia, min(ia + T, n + 1))
            cols = range(ja, min(ja + T, n + 1))
            k_near, k_far = K[g[I], g[J]], K[g[I + 1], g[J + 1]]
            kh = min(k_far, ja + T - 1)
            near = [k for k in range(ia, ja + 1) if k <= kh and U[ia, k] + L[k, ja] == D[ia, ja]]
            assert near, "the near corner's maximisers reach below the far corner's"
            x = max(near)
            for i in rows:
                for j in cols:
                    if i > j:
                        continue
                    assert k_near <= K[i, j] <= k_far
                    lo, hi = max(x, i), min(kh, j)
                    assert lo <= hi
                    best = max(U[i, k] + L[k, j] for k in range(lo, hi + 1))
                    assert best == D[i, j], (I, J, i, j)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("T", [2, 4, 8])
def test_constant_tiles(seed, T):
    n, U, L, D, K = _merge_case(seed)
    P, g = _grid(T, n)
    constant = 0
    for I in range(P):
        for J in range(I + 1, P):
            vmin, vmax = D[g[I + 1], g[J]], D[g[I], g[J + 1]]
            tile = D[g[I]:min(g[I] + T, n + 1), g[J]:min(g[J] + T, n + 1)]
            assert tile.min() >= vmin and tile.max() <= vmax
            if vmin == vmax:
                constant += 1
                assert np.all(tile == vmax)
    # the rule is exercised, not vacuous, on the cases with long b
    if n >= 48 and T == 2:
        assert constant > 0


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("T", [4, 8])
def test_traceback_window_from_grid_corners(seed, T):
    n, U, L, D, K = _merge_case(seed)
    P, g = _grid(T, n)
    for i in range(n + 1):
        for j in range(i, n + 1):
            I0, J0 = min(i // T, P), min(j // T, P)
            I1, J1 = min(I0 + 1, P), min(J0 + 1, P)
            lo = max(i, K[g[I0], g[J0]])
            hi = min(j, K[g[I1], g[J1]])
            assert lo <= K[i, j] <= hi


@pytest.mark.parametrize("seed", range(6))
def test_leaf_rule_matches_leftmost_traceback(seed):
    rng = np.random.default_rng(950 + seed)
    alph = [inputs.ACGT, np.frombuffer(b"AB", dtype=np.uint8), inputs.AA20][seed % 3]
    for _ in range(30):
        h = int(rng.integers(1, 12))
        n = int(rng.integers(0, 16))
        a, b = inputs.random_pair(rng, h, n, alph)
        i = int(rng.integers(0, n + 1))
        j = int(rng.integers(i, n + 1))
        F = np.array([[oracle.lcs_length(a[:r], b[i:c]) for c in range(i, j + 1)] for r in range(h + 1)])
        B = np.array([[oracle.lcs_length(a[r:], b[c:j]) for c in range(i, j + 1)] for r in range(h + 1)])
        L = F[h, j - i]
        assert B[0, 0] == L
        v = [int(np.flatnonzero(F[r] + B[r] == L)[0]) for r in range(h + 1)]
        marked = bytes(int(a[r - 1]) for r in range(1, h + 1)
                       if v[r] > v[r - 1] and a[r - 1] == b[i + v[r] - 1])
        s_ref, v_ref = oracle.traceback(a, b[i:j])
        assert [int(x) for x in v_ref] == v
        assert marked == s_ref


def _is_subsequence(s, t):
    it = iter(bytes(t))
    return all(ch in it for ch in bytes(s))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("word", [4, 8, 32])
def test_strip_vector_and_settled_words(seed, word):
    rng = np.random.default_rng(970 + seed)
    alph = [inputs.ACGT, np.frombuffer(b"AB", dtype=np.uint8), inputs.AA20][seed % 3]
    h = int(rng.integers(1, 41))
    n = int(rng.integers(0, 60))
    a, b = inputs.random_pair(rng, h, n, alph)
    if seed % 2:
        b = inputs.mutate(rng, np.tile(a, 3), 0.1, 0.05, alph, out_len=n)
    D = oracle.dist(a, b).astype(np.int64)
    full = (1 << h) - 1
    M = {int(c): sum(1 << r for r in range(h) if a[r] == c) for c in set(a.tolist()) | set(b.tolist())}
    words = -(-h // word)
    wmask = (1 << word) - 1
    for i in range(n + 1):
        V, d, settled = full, 0, 0
        for j in range(i + 1, n + 1):
            m = M[int(b[j - 1])]
            u = V & m
            tot = V + u
            carry = tot >> h
            Vn = (tot | (V & ~m)) & full
            # the same step from the first live word S on, no carry in
            S = settled
            lo = S * word
            tot_s = (V >> lo) + (u >> lo)
            assert (tot_s >> (h - lo)) == carry
            assert ((tot_s | ((V & ~m) >> lo)) & (full >> lo)) << lo == Vn
            V = Vn
            d += carry
            assert d == D[i, j]
            zeros = [r for r in range(h) if not (V >> r) & 1]
            # F_j(r) = number of zero bits among rows 0..r-1
            for r in range(h + 1):
                assert sum(1 for z in zeros if z < r) == oracle.lcs_length(a[:r], b[i:j])
            # low words zero <=> that prefix of a is a subsequence of b[i:j]
            now = 0
            while now < words and ((V >> (now * word)) & wmask) == 0:
                now += 1
            for w in range(words):
                rows = min((w + 1) * word, h)
                low_zero = (V & ((1 << rows) - 1)) == 0
                assert low_zero == _is_subsequence(a[:rows], b[i:j])
            assert now >= settled          # zero words stay zero
            settled = now
