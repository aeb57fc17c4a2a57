"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is exact: DIST values, lengths, argmax vertices and the LCS
string are integers, so the bar is bit-exact equality element by element.
"""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPH2 = np.frombuffer(b"AB", dtype=np.uint8)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    yield c
    B.lcs_destroy(c)


def dev(x):
    return torch.from_numpy(np.array(x, dtype=np.uint8, copy=True)).cuda()


def dist_buffer(n, dtype=torch.int32, pad=0):
    elem = 4 if dtype == torch.int32 else 2
    ld = n + 1 + pad
    ld = (ld * elem + 15) // 16 * 16 // elem
    buf = torch.full((n + 1, ld), 77, dtype=dtype, device="cuda")
    return buf


def gpu_dist(ctx, a, b, dtype=torch.int32, h=0):
    B.lcs_set_strip_height(ctx, h)
    d = dist_buffer(len(b), dtype)
    B.lcs_dist(ctx, dev(a), dev(b), d)
    B.lcs_sync(ctx)
    return d[:, : len(b) + 1].cpu().numpy().astype(np.int64)


def oracle_dist(a, b, dtype=torch.int32):
    D = oracle.dist(a, b).astype(np.int64)
    if dtype == torch.int16:
        D[D == np.iinfo(np.int32).min] = np.iinfo(np.int16).min
    return D


def gpu_solve(ctx, a, b, h=0, with_dist=False):
    B.lcs_set_strip_height(ctx, h)
    m, n = len(a), len(b)
    out = torch.zeros(max(1, min(m, n)), dtype=torch.uint8, device="cuda")
    cross = torch.full((m + 1,), -7, dtype=torch.int32, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")
    d = dist_buffer(n) if with_dist else None
    B.lcs_solve(ctx, dev(a), dev(b), dist=d, out_lcs=out, cross=cross, out_len=ln)
    B.lcs_sync(ctx)
    L = int(ln.item())
    res = (bytes(out[:L].cpu().numpy()), cross.cpu().numpy().astype(np.int64), L)
    if with_dist:
        res = res + (d[:, : n + 1].cpu().numpy().astype(np.int64),)
    return res


# ------------------------------------------------------------------ strip builder
@pytest.mark.parametrize("h", [1, 5, 31, 32, 33, 64, 100, 128, 200, 256])
@pytest.mark.parametrize("n", [0, 1, 63, 64, 65, 130])
def test_strip_dist(ctx, h, n):
    rng = np.random.default_rng(1000 * h + n)
    a, b = inputs.random_pair(rng, h, n)
    for dtype in (torch.int32, torch.int16):
        d = dist_buffer(n, dtype)
        B.lcs_strip_dist(ctx, dev(a), dev(b), d)
        B.lcs_sync(ctx)
        got = d[:, : n + 1].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, oracle_dist(a, b, dtype))


def test_strip_dist_large_and_single_letter(ctx):
    rng = np.random.default_rng(5)
    a = inputs.uniform(rng, 77, inputs.ACGT)
    b = inputs.uniform(rng, 700, inputs.ACGT)
    d = dist_buffer(700)
    B.lcs_strip_dist(ctx, dev(a), dev(b), d)
    B.lcs_sync(ctx)
    assert np.array_equal(d[:, :701].cpu().numpy(), oracle.dist(a, b))
    # Single-row leaf (Sec. II-B-3 worked example): rows = 't', b = gatttatgcagg.
    a1, b1 = b"t", b"gatttatgcagg"
    d = dist_buffer(12)
    B.lcs_strip_dist(ctx, dev(np.frombuffer(a1, np.uint8)), dev(np.frombuffer(b1, np.uint8)), d)
    B.lcs_sync(ctx)
    assert np.array_equal(d[:, :13].cpu().numpy(), oracle.dist(a1, b1))


# ------------------------------------------------------------------ merge
@pytest.mark.parametrize("n", [0, 1, 10, 63, 64, 65, 129, 200, 333])
def test_merge_matches_bruteforce(ctx, n):
    rng = np.random.default_rng(77 + n)
    m1, m2 = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    a1, a2 = inputs.uniform(rng, m1, inputs.ACGT), inputs.uniform(rng, m2, inputs.ACGT)
    b = inputs.uniform(rng, n, inputs.ACGT)
    U, L = oracle.dist(a1, b), oracle.dist(a2, b)
    D, K = oracle.merge(U, L)
    for dtype in (torch.int32, torch.int16):
        du, dl, dd = dist_buffer(n, dtype), dist_buffer(n, dtype), dist_buffer(n, dtype)
        Uc = U.astype(np.int64)
        Lc = L.astype(np.int64)
        if dtype == torch.int16:
            Uc[Uc < -40000] = -32768
            Lc[Lc < -40000] = -32768
        du[:, : n + 1] = torch.from_numpy(Uc).to(dtype).cuda()
        dl[:, : n + 1] = torch.from_numpy(Lc).to(dtype).cuda()
        km = torch.full(du.shape, -5, dtype=torch.int32, device="cuda")
        B.lcs_merge(ctx, du, dl, dd, km)
        B.lcs_sync(ctx)
        got = dd[:, : n + 1].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, oracle_dist(np.concatenate([a1, a2]), b, dtype))
        want = D.astype(np.int64)
        if dtype == torch.int16:
            want[want < -40000] = -32768
        assert np.array_equal(got, want)
        assert np.array_equal(km[:, : n + 1].cpu().numpy(), K)


def test_merge_degenerate_windows(ctx):
    """Strings that make the argmax windows wide (all-equal letters, no
    matches in one half) exercise the global-memory fallback of the tile."""
    n = 300
    cases = [
        (np.full(90, 65, np.uint8), np.full(90, 65, np.uint8), np.full(n, 65, np.uint8)),
        (np.full(70, 67, np.uint8), np.full(50, 65, np.uint8), np.full(n, 65, np.uint8)),
        (np.full(50, 65, np.uint8), np.full(70, 67, np.uint8), np.full(n, 65, np.uint8)),
    ]
    for a1, a2, b in cases:
        U, L = oracle.dist(a1, b), oracle.dist(a2, b)
        D, K = oracle.merge(U, L)
        du, dl, dd = dist_buffer(n), dist_buffer(n), dist_buffer(n)
        du[:, : n + 1] = torch.from_numpy(U).cuda()
        dl[:, : n + 1] = torch.from_numpy(L).cuda()
        km = torch.full(du.shape, -5, dtype=torch.int32, device="cuda")
        B.lcs_merge(ctx, du, dl, dd, km)
        B.lcs_sync(ctx)
        assert np.array_equal(dd[:, : n + 1].cpu().numpy(), D)
        assert np.array_equal(km[:, : n + 1].cpu().numpy(), K)


# ------------------------------------------------------------------ whole path
@pytest.mark.parametrize("h", [0, 1, 3, 8, 32, 100])
def test_dist_multi_strip(ctx, h):
    rng = np.random.default_rng(300 + h)
    for m, n in [(37, 45), (128, 64), (65, 200), (200, 129), (9, 300)]:
        a, b = inputs.random_pair(rng, m, n)
        assert np.array_equal(gpu_dist(ctx, a, b, h=h), oracle_dist(a, b))
        assert np.array_equal(gpu_dist(ctx, a, b, torch.int16, h=h), oracle_dist(a, b, torch.int16))


@pytest.mark.parametrize("h", [0, 1, 2, 7, 32, 64, 256])
def test_traceback_leftmost(ctx, h):
    rng = np.random.default_rng(500 + h)
    for m, n in [(1, 1), (1, 9), (9, 1), (40, 40), (100, 37), (37, 100), (257, 130), (130, 257)]:
        a, b = inputs.random_pair(rng, m, n, ALPH2 if (m + n) % 2 else inputs.ACGT)
        s_want, v_want = oracle.traceback(a, b)
        s, cross, L = gpu_solve(ctx, a, b, h=h)
        assert L == len(s_want) == oracle.lcs_length(a, b)
        assert s == s_want
        assert np.array_equal(cross, v_want)


def test_length_and_traceback_entry_points(ctx):
    rng = np.random.default_rng(9)
    a, b = inputs.random_pair(rng, 300, 280)
    B.lcs_set_strip_height(ctx, 0)
    assert B.lcs_length(ctx, dev(a), dev(b)) == oracle.lcs_length(a, b)
    out = torch.zeros(280, dtype=torch.uint8, device="cuda")
    L = B.lcs_traceback(ctx, dev(a), dev(b), out)
    assert bytes(out[:L].cpu().numpy()) == oracle.traceback(a, b)[0]


def test_edge_cases(ctx):
    B.lcs_set_strip_height(ctx, 0)
    empty = np.zeros(0, np.uint8)
    rng = np.random.default_rng(11)
    x = inputs.uniform(rng, 50, inputs.ACGT)
    # empty strings
    assert np.array_equal(gpu_dist(ctx, empty, x), oracle_dist(empty, x))
    assert np.array_equal(gpu_dist(ctx, x, empty), oracle_dist(x, empty))
    s, cross, L = gpu_solve(ctx, x, empty)
    assert L == 0 and s == b"" and np.all(cross == 0)
    # identical strings and disjoint alphabets
    s, cross, L = gpu_solve(ctx, x, x)
    assert L == 50 and s == bytes(x)
    other = np.frombuffer(b"XYZW" * 20, np.uint8)
    s, cross, L, D = gpu_solve(ctx, x, other, with_dist=True)
    assert L == 0 and s == b""
    assert np.array_equal(D, oracle_dist(x, other))
    # all-equal letters (widest argmax windows)
    aa = np.full(333, 65, np.uint8)
    bb = np.full(250, 65, np.uint8)
    s, cross, L, D = gpu_solve(ctx, aa, bb, h=16, with_dist=True)
    assert L == 250 and np.array_equal(D, oracle_dist(aa, bb))
    s_want, v_want = oracle.traceback(aa, bb)
    assert s == s_want and np.array_equal(cross, v_want)


@pytest.mark.parametrize("h", [0, 64, 256])
def test_long_horizontal_runs(ctx, h):
    """Paths whose part in one strip spans more than 1024 columns (a run of
    letters absent from the strip): the leaf takes its global-memory route."""
    cases = [
        (np.full(512, 65, np.uint8), np.concatenate([np.full(3000, 67, np.uint8), np.full(600, 65, np.uint8)])),
        (np.concatenate([np.full(300, 65, np.uint8), np.full(300, 71, np.uint8)]),
         np.concatenate([np.full(1500, 67, np.uint8), np.full(200, 65, np.uint8), np.full(1500, 84, np.uint8),
                         np.full(400, 71, np.uint8)])),
    ]
    for a, b in cases:
        s_want, v_want = oracle.traceback(a, b)
        s, cross, L = gpu_solve(ctx, a, b, h=h)
        assert L == len(s_want) and s == s_want
        assert np.array_equal(cross, v_want)


def test_invalid_arguments(ctx):
    a = dev(np.zeros(4, np.uint8))
    d = torch.zeros((5, 7), dtype=torch.int32, device="cuda")     # ld*4 not a multiple of 16
    with pytest.raises(B.LcsError) as e:
        B.lcs_dist(ctx, a, a, d)
    assert e.value.status == B.LCS_EINVAL
    with pytest.raises(ValueError):
        B._dtype_of(torch.zeros(1, dtype=torch.float32))


@pytest.mark.parametrize("host", ["pinned", "pinned_odd_pitch", "pageable", "pinned_i16", "pinned_no_lcs",
                                  "pinned_3_levels", "pinned_one_strip", "pinned_empty_a", "pinned_empty_b"])
def test_solve_host_roundtrip(ctx, host):
    """Pinned 16-byte-pitch DIST is written by the kernels directly (its
    lower triangle while the tree is built, the rest by the root merge); an
    odd pitch or pageable memory goes through device staging and a copy.
    Without an LCS to return the root merge runs on the caller's stream and
    waits for the side stream's fill.  Every entry starts at 5, so one the
    solve did not write shows."""
    rng = np.random.default_rng(12)
    m, n = {"pinned_3_levels": (1100, 900), "pinned_one_strip": (100, 300), "pinned_empty_a": (0, 37),
            "pinned_empty_b": (41, 0)}.get(host, (333, 444))
    a, b = inputs.random_pair(rng, m, n)
    B.lcs_set_strip_height(ctx, 0)
    ah = torch.from_numpy(a).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    dt = torch.int16 if host == "pinned_i16" else torch.int32
    ld = n + 2 if host == "pinned_odd_pitch" else (n + 1 + 7) // 8 * 8    # rows 16-byte aligned for both types
    dh = torch.full((n + 1, ld), 5, dtype=dt)
    if host != "pageable":
        dh = dh.pin_memory()
    lh = None if host == "pinned_no_lcs" else torch.zeros(max(m, 1), dtype=torch.uint8).pin_memory()
    L = B.lcs_solve_host(ctx, ah, bh, dist_host=dh, lcs_host=lh)
    s_want, _ = oracle.traceback(a, b)
    assert L == len(s_want)
    if lh is not None:
        assert bytes(lh[:L].numpy()) == s_want
    assert np.array_equal(dh[:, :n + 1].numpy().astype(np.int64), oracle_dist(a, b, dt))


# ------------------------------------------------------------------ the named workloads
def test_small_pair_64(ctx):
    """m = n = 64, uniform ACGT, seed 0: length, full DIST, LCS."""
    a, b = inputs.pair_small(0)
    s, cross, L, D = gpu_solve(ctx, a, b, with_dist=True)
    s_want, v_want = oracle.traceback(a, b)
    assert np.array_equal(D, oracle_dist(a, b))
    assert L == len(s_want) and s == s_want and np.array_equal(cross, v_want)


@pytest.mark.parametrize("variant", ["iid", "correlated"])
def test_pair_4096(ctx, variant):
    """m = n = 4096 (iid and correlated): full int32 DIST, length, LCS."""
    a, b = inputs.pair_4096(variant)
    s, cross, L, D = gpu_solve(ctx, a, b, with_dist=True)
    s_want, v_want = oracle.traceback(a, b)
    assert L == len(s_want) and s == s_want and np.array_equal(cross, v_want)
    assert np.array_equal(D, oracle.dist(a, b))


def test_pair_16384_full(ctx):
    """m = n = 16384, 20 letters Zipf(1.1), int16 DIST: every one of the
    16385 x 16385 entries against the oracle's per-source DP (about 2.2e12
    cell updates spread over the host cores, compared in blocks of rows);
    length; LCS."""
    a, b = inputs.pair_16384()
    n = len(b)
    B.lcs_set_strip_height(ctx, 0)
    d = dist_buffer(n, torch.int16)
    out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.lcs_solve(ctx, dev(a), dev(b), dist=d, out_lcs=out, out_len=ln)
    B.lcs_sync(ctx)
    L = int(ln.item())
    s_want, _ = oracle.traceback(a, b)
    assert L == len(s_want) and bytes(out[:L].cpu().numpy()) == s_want
    got = d[:, : n + 1].cpu().numpy()
    del d
    block = 1024
    for r0 in range(0, n + 1, block):
        rows = np.arange(r0, min(n + 1, r0 + block), dtype=np.int64)
        want = oracle.dist_rows(a, b, rows)
        want[want == np.iinfo(np.int32).min] = np.iinfo(np.int16).min
        bad = np.argwhere(got[rows].astype(np.int32) != want)
        assert bad.size == 0, f"first mismatch at (i, j) = ({rows[bad[0][0]]}, {bad[0][1]})"
