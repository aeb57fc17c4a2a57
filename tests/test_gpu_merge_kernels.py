"""Both tree merge kernels (exact refinement, the DPX 64 x 64 tile band
product) give the oracle's DIST, length, LCS string and
cross vertices, bit for bit (Sec. II-B-3); lcs_merge's exact argmax is
unaffected by the selection.

The cases reuse the parity helpers; each kernel is selected on its own
context with lcs_set_merge_kernel.
"""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

from test_gpu_parity import ALPH2, dist_buffer, gpu_dist, gpu_solve, oracle_dist

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = {"exact": B.LCS_MERGE_EXACT, "dpx": B.LCS_MERGE_DPX}


@pytest.fixture(scope="module", params=sorted(KINDS))
def kctx(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    B.lcs_set_merge_kernel(c, KINDS[request.param])
    yield c
    B.lcs_destroy(c)


def test_set_merge_kernel_rejects_unknown():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    try:
        with pytest.raises(B.LcsError):
            B.lcs_set_merge_kernel(c, 3)
        with pytest.raises(B.LcsError):
            B.lcs_set_merge_kernel(c, -1)
    finally:
        B.lcs_destroy(c)


@pytest.mark.parametrize("n", [0, 1, 10, 63, 64, 65, 127, 128, 129, 200, 333])
def test_merge_argmax(kctx, n):
    rng = np.random.default_rng(900 + n)
    m1, m2 = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    alph = ALPH2 if n % 2 else inputs.ACGT
    a1, a2, b = inputs.uniform(rng, m1, alph), inputs.uniform(rng, m2, alph), inputs.uniform(rng, n, alph)
    U, L = oracle.dist(a1, b), oracle.dist(a2, b)
    D, K = oracle.merge(U, L)
    for dtype in (torch.int32, torch.int16):
        du, dl, dd = dist_buffer(n, dtype), dist_buffer(n, dtype), dist_buffer(n, dtype)
        Uc, Lc, want = U.astype(np.int64), L.astype(np.int64), D.astype(np.int64)
        if dtype == torch.int16:
            for x in (Uc, Lc, want):
                x[x < -40000] = -32768
        du[:, : n + 1] = torch.from_numpy(Uc).to(dtype).cuda()
        dl[:, : n + 1] = torch.from_numpy(Lc).to(dtype).cuda()
        km = torch.full(du.shape, -5, dtype=torch.int32, device="cuda")
        B.lcs_merge(kctx, du, dl, dd, km)
        B.lcs_sync(kctx)
        assert np.array_equal(dd[:, : n + 1].cpu().numpy().astype(np.int64), want)
        assert np.array_equal(km[:, : n + 1].cpu().numpy(), K)


def test_merge_wide_windows(kctx):
    """All-equal letters and halves without matches: windows span the row."""
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
        B.lcs_merge(kctx, du, dl, dd, km)
        B.lcs_sync(kctx)
        assert np.array_equal(dd[:, : n + 1].cpu().numpy(), D)
        assert np.array_equal(km[:, : n + 1].cpu().numpy(), K)


@pytest.mark.parametrize("h", [1, 8, 64, 0])
def test_tree_dist_and_traceback(kctx, h):
    rng = np.random.default_rng(40 + h)
    for m, n in [(37, 45), (200, 129), (9, 300), (257, 130), (130, 257), (700, 500)]:
        a, b = inputs.random_pair(rng, m, n, ALPH2 if (m + n) % 2 else inputs.ACGT)
        assert np.array_equal(gpu_dist(kctx, a, b, h=h), oracle_dist(a, b))
        assert np.array_equal(gpu_dist(kctx, a, b, torch.int16, h=h), oracle_dist(a, b, torch.int16))
        s_want, v_want = oracle.traceback(a, b)
        s, cross, L = gpu_solve(kctx, a, b, h=h)
        assert L == len(s_want) and s == s_want and np.array_equal(cross, v_want)


@pytest.mark.parametrize("n", [31, 32, 33, 95, 96, 97, 159, 160, 161, 1023, 1024, 1025])
def test_tree_ragged_quadrants(kctx, n):
    """Widths around multiples of the 32-vertex quadrant and the 64-vertex
    tile, three and more tree levels, both DIST types."""
    rng = np.random.default_rng(5000 + n)
    for m in (3 * 64 + 5, 8 * 64):
        a, b = inputs.random_pair(rng, m, n, inputs.ACGT)
        assert np.array_equal(gpu_dist(kctx, a, b, h=32), oracle_dist(a, b))
        assert np.array_equal(gpu_dist(kctx, a, b, torch.int16, h=64), oracle_dist(a, b, torch.int16))
        s_want, v_want = oracle.traceback(a, b)
        s, cross, L = gpu_solve(kctx, a, b, h=32)
        assert L == len(s_want) and s == s_want and np.array_equal(cross, v_want)


def test_pair_4096_iid(kctx):
    """m = n = 4096 iid ACGT through the tree: full int32 DIST, LCS, vertices."""
    a, b = inputs.pair_4096("iid")
    s, cross, L, D = gpu_solve(kctx, a, b, with_dist=True)
    s_want, v_want = oracle.traceback(a, b)
    assert L == len(s_want) and s == s_want and np.array_equal(cross, v_want)
    assert np.array_equal(D, oracle.dist(a, b))
