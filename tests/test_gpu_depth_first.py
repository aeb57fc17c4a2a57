"""Depth-first, memory-bounded tree (Sec. II-A's recursion scheduled so that
only a chunk of strips and one pending node per level are alive) with the
traceback recomputing the rows and columns of freed nodes (Sec. II-D's
argmax at every merge, Hirschberg's split).  Every output must equal the
oracle's bit for bit: DIST, length, LCS string and cross vertices, for any
chunk size, strip height, tree shape and budget.
"""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

from test_gpu_parity import ALPH2, dist_buffer, dev, oracle_dist

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    B.lcs_set_schedule(c, B.LCS_SCHED_DEPTH, 0)
    yield c
    B.lcs_destroy(c)


def solve(c, a, b, h=0, dtype=torch.int32, want_dist=True, want_lcs=True):
    B.lcs_set_strip_height(c, h)
    m, n = len(a), len(b)
    out = torch.zeros(max(1, min(m, n)), dtype=torch.uint8, device="cuda") if want_lcs else None
    cross = torch.full((m + 1,), -7, dtype=torch.int32, device="cuda") if want_lcs else None
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")
    d = dist_buffer(n, dtype) if want_dist else None
    B.lcs_solve(c, dev(a), dev(b), dist=d, out_lcs=out, cross=cross, out_len=ln)
    B.lcs_sync(c)
    L = int(ln.item())
    st = B.lcs_get_stats(c)
    res = {"L": L, "stats": st}
    if want_lcs:
        res["s"] = bytes(out[:L].cpu().numpy())
        res["cross"] = cross.cpu().numpy().astype(np.int64)
    if want_dist:
        res["D"] = d[:, : n + 1].cpu().numpy().astype(np.int64)
    return res


@pytest.mark.parametrize("chunk", [1, 2, 3, 4, 8])
def test_chunks_and_tree_shapes(ctx, chunk):
    B.lcs_set_schedule(ctx, B.LCS_SCHED_DEPTH, chunk)
    rng = np.random.default_rng(700 + chunk)
    try:
        for m, n, h in [(700, 500, 64), (2049, 300, 256), (130, 257, 32), (64 * 13 + 7, 161, 64)]:
            a, b = inputs.random_pair(rng, m, n, ALPH2 if m % 2 else inputs.ACGT)
            r = solve(ctx, a, b, h=h)
            assert r["stats"]["depth_first"] == 1
            # the host-only plan query reports the plan the solve used
            info, _ = B.lcs_plan(m, n, h, B.LCS_SCHED_DEPTH, chunk, want_lcs=True)
            st = r["stats"]
            assert (st["plan_bytes"], st["chunk_strips"], st["strips"], st["tree_levels"]) == (
                info["workspace_bytes"], info["chunk"], info["strips"], info["levels"])
            s_want, v_want = oracle.traceback(a, b)
            assert r["L"] == len(s_want) and r["s"] == s_want and np.array_equal(r["cross"], v_want)
            assert np.array_equal(r["D"], oracle_dist(a, b))
            r16 = solve(ctx, a, b, h=h, dtype=torch.int16, want_lcs=False)
            assert np.array_equal(r16["D"], oracle_dist(a, b, torch.int16))
    finally:
        B.lcs_set_schedule(ctx, B.LCS_SCHED_DEPTH, 0)


def test_length_and_traceback_without_dist(ctx):
    """No DIST wanted: no tree is built; the recomputed root split gives the
    length, and the per-depth splits the string."""
    rng = np.random.default_rng(71)
    for m, n in [(1000, 900), (513, 2000), (4096, 37)]:
        a, b = inputs.random_pair(rng, m, n, inputs.ACGT)
        B.lcs_set_strip_height(ctx, 64)
        assert B.lcs_length(ctx, dev(a), dev(b)) == oracle.lcs_length(a, b)
        r = solve(ctx, a, b, h=64, want_dist=False)
        s_want, v_want = oracle.traceback(a, b)
        assert r["L"] == len(s_want) and r["s"] == s_want and np.array_equal(r["cross"], v_want)


@pytest.mark.parametrize("variant", ["iid", "correlated"])
def test_pair_4096_depth_first(ctx, variant):
    a, b = inputs.pair_4096(variant)
    r = solve(ctx, a, b)
    s_want, v_want = oracle.traceback(a, b)
    assert r["stats"]["depth_first"] == 1
    assert r["L"] == len(s_want) and r["s"] == s_want and np.array_equal(r["cross"], v_want)
    assert np.array_equal(r["D"], oracle.dist(a, b))


def test_small_budget_uses_depth_first():
    """A budget below the retained tree's workspace: the automatic schedule
    builds the tree depth first within it, bit-exact."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a, b = inputs.pair_4096("iid")
    big = B.lcs_create(0, 0)
    try:
        solve(big, a, b, h=128, want_lcs=False)
        retained = B.lcs_get_stats(big)
        assert retained["depth_first"] == 0
        info, _ = B.lcs_plan(len(a), len(b), 128, want_lcs=False)
        assert info["depth_first"] == 0 and info["workspace_bytes"] == retained["plan_bytes"]
    finally:
        B.lcs_destroy(big)
    budget = retained["plan_bytes"] // 3
    c = B.lcs_create(0, budget)
    try:
        r = solve(c, a, b, h=128)
        assert r["stats"]["depth_first"] == 1
        assert r["stats"]["peak_workspace_bytes"] <= budget
        info, _ = B.lcs_plan(len(a), len(b), 128, B.LCS_SCHED_AUTO, 0, budget, want_lcs=True)
        assert info["depth_first"] == 1 and info["fits"] == 1
        assert (info["workspace_bytes"], info["chunk"]) == (r["stats"]["plan_bytes"], r["stats"]["chunk_strips"])
        s_want, v_want = oracle.traceback(a, b)
        assert r["L"] == len(s_want) and r["s"] == s_want and np.array_equal(r["cross"], v_want)
        assert np.array_equal(r["D"], oracle.dist(a, b))
    finally:
        B.lcs_destroy(c)


def test_schedule_rejects_bad_arguments(ctx):
    with pytest.raises(B.LcsError):
        B.lcs_set_schedule(ctx, 3, 0)
    with pytest.raises(B.LcsError):
        B.lcs_set_schedule(ctx, B.LCS_SCHED_DEPTH, -1)


@pytest.mark.parametrize("host", ["pinned", "pageable"])
def test_solve_host_depth_first(ctx, host):
    """lcs_solve_host on a depth-first plan: the pinned DIST's lower triangle
    is filled on a side stream while the tree is built, the root merge writes
    the rest over the link, and the traceback recomputes beside the tree."""
    a, b = inputs.random_pair(np.random.default_rng(72), 1500, 1300)
    m, n = len(a), len(b)
    B.lcs_set_strip_height(ctx, 128)
    ah = torch.from_numpy(a).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    dh = torch.full((n + 1, (n + 1 + 3) // 4 * 4), 5, dtype=torch.int32)
    if host == "pinned":
        dh = dh.pin_memory()
    lh = torch.zeros(min(m, n), dtype=torch.uint8).pin_memory()
    L = B.lcs_solve_host(ctx, ah, bh, dist_host=dh, lcs_host=lh)
    assert B.lcs_get_stats(ctx)["depth_first"] == 1
    s_want, _ = oracle.traceback(a, b)
    assert L == len(s_want) and bytes(lh[:L].numpy()) == s_want
    assert np.array_equal(dh[:, : n + 1].numpy().astype(np.int64), oracle_dist(a, b))


def test_graph_replay_depth_first(ctx):
    """CUDA-graph capture of a depth-first solve (side-stream fork and join
    inside the capture) replays to the same results."""
    a, b = inputs.random_pair(np.random.default_rng(73), 900, 1100)
    B.lcs_set_graphs(ctx, True)
    try:
        for _ in range(3):                                  # eager, capture, replay
            r = solve(ctx, a, b, h=64)
            s_want, v_want = oracle.traceback(a, b)
            assert r["stats"]["depth_first"] == 1
            assert r["L"] == len(s_want) and r["s"] == s_want and np.array_equal(r["cross"], v_want)
            assert np.array_equal(r["D"], oracle_dist(a, b))
    finally:
        B.lcs_set_graphs(ctx, False)
