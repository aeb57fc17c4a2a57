"""CUDA-graph replay of lcs_solve and the autotuner: same results as the
plain launches (the oracle's), whatever is replayed or chosen."""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

from test_gpu_parity import dist_buffer

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    yield c
    B.lcs_destroy(c)


class Slot:
    """Device buffers at fixed addresses (a graph replays pointers)."""

    def __init__(self, m, n):
        self.a = torch.zeros(m, dtype=torch.uint8, device="cuda")
        self.b = torch.zeros(n, dtype=torch.uint8, device="cuda")
        self.d = dist_buffer(n)
        self.out = torch.zeros(max(1, min(m, n)), dtype=torch.uint8, device="cuda")
        self.cross = torch.zeros(m + 1, dtype=torch.int32, device="cuda")
        self.ln = torch.zeros(1, dtype=torch.int64, device="cuda")

    def load(self, a, b):
        self.a.copy_(torch.from_numpy(a))
        self.b.copy_(torch.from_numpy(b))

    def solve(self, ctx):
        B.lcs_solve(ctx, self.a, self.b, dist=self.d, out_lcs=self.out, cross=self.cross, out_len=self.ln)
        B.lcs_sync(ctx)
        n = self.b.numel()
        L = int(self.ln.item())
        return (self.d[:, : n + 1].cpu().numpy(), bytes(self.out[:L].cpu().numpy()),
                self.cross.cpu().numpy().astype(np.int64))

    def check(self, ctx, a, b):
        D, s, v = self.solve(ctx)
        s_want, v_want = oracle.traceback(a, b)
        assert np.array_equal(D, oracle.dist(a, b))
        assert s == s_want and np.array_equal(v, v_want)


def test_graph_replay(ctx):
    rng = np.random.default_rng(61)
    B.lcs_set_graphs(ctx, True)
    B.lcs_set_strip_height(ctx, 64)
    A = Slot(300, 200)
    Bs = Slot(130, 257)
    a1, b1 = inputs.random_pair(rng, 300, 200)
    A.load(a1, b1)
    A.check(ctx, a1, b1)                   # eager run + capture
    A.check(ctx, a1, b1)                   # replay
    launches = B.lcs_get_stats(ctx)["kernel_launches"]
    assert launches > 1
    a2, b2 = inputs.random_pair(rng, 300, 200)
    A.load(a2, b2)                         # same addresses, new contents
    A.check(ctx, a2, b2)
    a3, b3 = inputs.random_pair(rng, 130, 257)
    Bs.load(a3, b3)
    Bs.check(ctx, a3, b3)                  # another shape: re-capture
    # A plain call on another shape rewrites the device plan: the next
    # replay of A must not use the stale graph.
    d = dist_buffer(77)
    a4, b4 = inputs.random_pair(rng, 90, 77)
    B.lcs_dist(ctx, torch.from_numpy(a4).cuda(), torch.from_numpy(b4).cuda(), d)
    B.lcs_sync(ctx)
    assert np.array_equal(d[:, :78].cpu().numpy(), oracle.dist(a4, b4))
    A.check(ctx, a2, b2)
    A.check(ctx, a2, b2)
    B.lcs_set_strip_height(ctx, 128)       # another plan for the same arguments
    A.check(ctx, a2, b2)
    B.lcs_set_graphs(ctx, False)
    A.check(ctx, a2, b2)


def test_autotune(ctx):
    a, b = inputs.pair_4096("iid")
    S = Slot(len(a), len(b))
    S.load(a, b)
    r = B.lcs_autotune(ctx, S.a, S.b, dist=S.d, out_lcs=S.out)
    assert r["strip_height"] in (64, 128, 256)
    assert r["merge_kernel"] in (B.LCS_MERGE_DPX, B.LCS_MERGE_EXACT)
    assert r["ms"] > 0
    B.lcs_set_strip_height(ctx, 0)
    S.check(ctx, a, b)
    assert B.lcs_get_stats(ctx)["strip_height"] == r["strip_height"]
    # graphs on top of the tuned choice
    B.lcs_set_graphs(ctx, True)
    S.check(ctx, a, b)
    S.check(ctx, a, b)


def test_autotune_rejects_empty(ctx):
    z = torch.zeros(0, dtype=torch.uint8, device="cuda")
    o = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.LcsError):
        B.lcs_autotune(ctx, z, o)
