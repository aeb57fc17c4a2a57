"""The tree planner, through the host-only lcs_plan query (no GPU).

The tree is Sec. II-A's recursion: strips of h rows of a combined pairwise,
the upper half's rows directly above the lower half's, up to one root that
covers all m rows.  lcs_plan runs the same strip-height rule and schedule
choice as a solve and reports every node's rows, its storage and grids in
the device workspace, and the launches that write and last read them.  The
depth-first schedule reuses a pool of slots, so what matters here is that
no two regions in use during the same launch overlap, for every schedule
and chunk, and that the automatic choice follows its documented rule.
"""
import itertools

import pytest

from paper_2309_09072_gb300 import binding as B

GiB = 1 << 30


def _check_tree(m, n, h, info, nodes):
    S = -(-m // h)
    assert info["strip_height"] == h and info["strips"] == S
    assert info["nodes"] == len(nodes) == 2 * S - 1
    root = info["root"]
    assert nodes[root]["row0"] == 0 and nodes[root]["rows"] == m and nodes[root]["parent"] == -1
    for s in range(S):
        nd = nodes[s]
        assert nd["row0"] == s * h and nd["rows"] == min(h, m - s * h)
        assert nd["upper"] == nd["lower"] == -1 and nd["level"] == 0
    parents = [nd["parent"] for nd in nodes]
    for v, nd in enumerate(nodes[S:], start=S):
        u, l = nodes[nd["upper"]], nodes[nd["lower"]]
        # Sec. II-A: the upper half's rows lie directly above the lower half's
        assert u["row0"] == nd["row0"] and l["row0"] == u["row0"] + u["rows"]
        assert nd["rows"] == u["rows"] + l["rows"]
        assert u["parent"] == v and l["parent"] == v
        assert nd["level"] > max(u["level"], l["level"])
    # every node but the root is consumed exactly once
    for v in range(len(nodes)):
        if v != root:
            assert sum(1 for x in nodes if v in (x["upper"], x["lower"])) == 1
            assert parents[v] >= S
    assert info["levels"] == max(nd["level"] for nd in nodes)


def _check_launches_and_storage(info, nodes):
    L = info["launches"]
    root = info["root"]
    for v, nd in enumerate(nodes):
        assert 0 <= nd["made_by"] < L
        if nd["upper"] >= 0:
            for c in (nd["upper"], nd["lower"]):
                assert nodes[c]["made_by"] < nd["made_by"]
                if info["depth_first"]:
                    assert nodes[c]["last_use"] == nd["made_by"]
        if info["depth_first"] and v != root:
            assert nd["last_use"] == nodes[nd["parent"]]["made_by"]
        else:
            assert nd["last_use"] == L
    # regions in use during each launch never overlap, and all lie in the workspace
    for t in range(L + 1):
        regions = []
        for v, nd in enumerate(nodes):
            if nd["bytes"] and nd["made_by"] <= t <= nd["last_use"]:
                regions.append((nd["offset"], nd["offset"] + nd["bytes"], "node", v))
            if nd["grid_bytes"] and nd["made_by"] <= t <= nd["grid_last_use"]:
                regions.append((nd["grid_offset"], nd["grid_offset"] + nd["grid_bytes"], "grid", v))
        regions.sort()
        for r in regions:
            assert 256 <= r[0] < r[1] <= info["workspace_bytes"], r
        for a, b in zip(regions, regions[1:]):
            assert a[1] <= b[0], (t, a, b)
    assert nodes[root]["bytes"] == 0        # the root is the caller's matrix


CASES = [
    (4096, 4096, 256), (4096, 4096, 64), (1000, 50, 64), (777, 300, 17), (130, 64, 1), (256, 10, 256),
    (5000, 700, 128), (33, 33, 8),
]


@pytest.mark.parametrize("m,n,h", CASES)
@pytest.mark.parametrize("schedule,chunk", [(B.LCS_SCHED_RETAIN, 0), (B.LCS_SCHED_DEPTH, 0), (B.LCS_SCHED_DEPTH, 1),
                                            (B.LCS_SCHED_DEPTH, 3), (B.LCS_SCHED_DEPTH, 4), (B.LCS_SCHED_DEPTH, 7)])
def test_tree_and_storage(m, n, h, schedule, chunk):
    info, nodes = B.lcs_plan(m, n, h, schedule, chunk, want_lcs=False)
    S = -(-m // h)
    _check_tree(m, n, h, info, nodes)
    _check_launches_and_storage(info, nodes)
    if S > 1:
        assert info["depth_first"] == (1 if schedule == B.LCS_SCHED_DEPTH else 0)
    if info["depth_first"]:
        c = min(chunk or 32, S) if chunk else info["chunk"]
        assert info["chunk"] == c
        strip_launches = -(-S // c)
        assert info["launches"] == strip_launches + sum(
            1 for t in range(info["launches"]) if any(nd["made_by"] == t and nd["upper"] >= 0 for nd in nodes))
    else:
        # one launch for the strips, then one per group of a tree level
        assert info["launches"] >= 1 + info["levels"]


@pytest.mark.parametrize("S,chunk", list(itertools.product([5, 8, 13, 16, 31, 64], [1, 2, 4, 8, 32])))
def test_depth_first_keeps_few_nodes_alive(S, chunk):
    """Only the chunk's nodes and one pending node per tree level are alive:
    during a launch at most chunk + chunk/2 (a merge's operands and output)
    plus one per level of the pending counter."""
    h = 64
    info, nodes = B.lcs_plan(S * h, 200, h, B.LCS_SCHED_DEPTH, chunk, want_lcs=False)
    c = info["chunk"]
    peak = max(sum(1 for nd in nodes if nd["bytes"] and nd["made_by"] <= t <= nd["last_use"])
               for t in range(info["launches"]))
    assert peak <= c + c // 2 + info["levels"] + 1
    retained, _ = B.lcs_plan(S * h, 200, h, B.LCS_SCHED_RETAIN, want_lcs=False)
    if c <= S // 4:
        assert info["workspace_bytes"] < retained["workspace_bytes"]


def test_automatic_schedule_rule():
    # small enough to retain (at most 4 GiB and within the budget)
    info, _ = B.lcs_plan(4096, 4096)
    assert info["depth_first"] == 0 and info["strip_height"] == 256 and info["fits"]
    assert info["workspace_bytes"] <= 4 * GiB
    # the 16384 pair: the retained tree needs more than 4 GiB, so depth first
    # with the largest chunk of 32, 16, .. whose plan stays within 16 GiB
    full, _ = B.lcs_plan(16384, 16384, 0, B.LCS_SCHED_RETAIN, dtype=B.LCS_I16)
    assert full["workspace_bytes"] > 16 * GiB
    auto, nodes = B.lcs_plan(16384, 16384, dtype=B.LCS_I16)
    assert auto["depth_first"] == 1 and auto["chunk"] == 32 and auto["workspace_bytes"] <= 16 * GiB
    _check_launches_and_storage(auto, nodes)
    # a smaller budget takes a smaller chunk that fits it
    small, _ = B.lcs_plan(16384, 16384, 0, B.LCS_SCHED_AUTO, 0, 8 * GiB, dtype=B.LCS_I16)
    assert small["depth_first"] == 1 and small["chunk"] < 32 and small["workspace_bytes"] <= 8 * GiB
    assert small["fits"]
    # nothing fits 64 KiB: the solve would return ENOMEM
    tiny, _ = B.lcs_plan(4096, 4096, 0, B.LCS_SCHED_AUTO, 0, 64 << 10)
    assert tiny["fits"] == 0


def test_lcs_keeps_retained_tree_for_tall_halves():
    """The recomputing traceback sweeps a tree half of at most 16384 rows;
    with an LCS wanted, a taller half keeps the retained tree."""
    m, n = 40000, 64
    with_lcs, _ = B.lcs_plan(m, n, 256, B.LCS_SCHED_DEPTH, 0, want_lcs=True)
    without, nodes = B.lcs_plan(m, n, 256, B.LCS_SCHED_DEPTH, 0, want_lcs=False)
    assert with_lcs["depth_first"] == 0 and without["depth_first"] == 1
    assert max(nodes[nd["upper"]]["rows"] for nd in nodes if nd["upper"] >= 0) > 16384
    short, _ = B.lcs_plan(16384, 64, 256, B.LCS_SCHED_DEPTH, 0, want_lcs=True)
    assert short["depth_first"] == 1


def test_strip_height_rule_and_degenerate_grids():
    for m in (1, 7, 255, 256, 257, 10000):
        info, _ = B.lcs_plan(m, 100)
        assert info["strip_height"] == min(m, 256)
    for m, n in ((0, 0), (0, 50), (50, 0)):
        info, nodes = B.lcs_plan(m, n)
        assert info["strips"] == 0 and info["nodes"] == 0 and nodes == [] and info["root"] == -1
        assert info["fits"] == 1 and info["workspace_bytes"] == 256
    one, nodes = B.lcs_plan(200, 300)
    assert one["strips"] == 1 and one["root"] == 0 and nodes[0]["bytes"] == 0 and one["launches"] == 1


def test_plan_argument_errors():
    lib = B.load()
    info = B.lcs_plan_info()
    recs = (B.lcs_plan_node * 4)()
    ref = __import__("ctypes").byref
    ok = lib.lcs_plan(100, 100, 0, 0, 0, 0, 1, B.LCS_I32, ref(info), recs, 4)
    assert ok == B.LCS_OK and info.nodes == 1
    bad = [
        (-1, 100, 0, 0, 0, 0, 1, B.LCS_I32, ref(info), recs, 4),
        (100, -1, 0, 0, 0, 0, 1, B.LCS_I32, ref(info), recs, 4),
        (100, 100, 257, 0, 0, 0, 1, B.LCS_I32, ref(info), recs, 4),
        (100, 100, -1, 0, 0, 0, 1, B.LCS_I32, ref(info), recs, 4),
        (100, 100, 0, 3, 0, 0, 1, B.LCS_I32, ref(info), recs, 4),
        (100, 100, 0, 0, -1, 0, 1, B.LCS_I32, ref(info), recs, 4),
        (100, 100, 0, 0, 0, 0, 1, 2, ref(info), recs, 4),
        (40000, 100, 0, 0, 0, 0, 1, B.LCS_I16, ref(info), recs, 4),
        (100, 100, 0, 0, 0, 0, 1, B.LCS_I32, None, recs, 4),
        (100, 100, 0, 0, 0, 0, 1, B.LCS_I32, ref(info), None, 4),
        (100, 100, 0, 0, 0, 0, 1, B.LCS_I32, ref(info), recs, -1),
    ]
    for args in bad:
        assert lib.lcs_plan(*args) == B.LCS_EINVAL, args
    # fewer records than nodes: the first `cap` are written, the count is reported
    few = (B.lcs_plan_node * 2)()
    assert lib.lcs_plan(1000, 100, 64, 1, 0, 0, 0, B.LCS_I32, ref(info), few, 2) == B.LCS_OK
    assert info.nodes == 31 and few[0].rows == 64 and few[1].row0 == 64
