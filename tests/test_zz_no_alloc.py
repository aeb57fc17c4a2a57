"""lcs_merge_static: the merge for callers that may not allocate device memory.

Its scratch lives in a static device array inside the library, so it must
give exactly what lcs_merge gives (same D and same argmax), call after call,
even though every call reuses the same array; both must equal the oracle's
brute-force merge (every k, smallest maximiser).  This file is collected last so
that a run stopping at the first failure has already run everything else; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _operands(seed, n, dtype):
    rng = np.random.default_rng(seed)
    m1, m2 = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    b = inputs.uniform(rng, n, inputs.ACGT)
    U = oracle.dist(inputs.uniform(rng, m1, inputs.ACGT), b).astype(np.int64)
    L = oracle.dist(inputs.uniform(rng, m2, inputs.ACGT), b).astype(np.int64)
    elem = 4 if dtype == torch.int32 else 2
    ld = ((n + 1) * elem + 15) // 16 * 16 // elem
    sentinel = np.iinfo(np.int32).min if dtype == torch.int32 else np.iinfo(np.int16).min
    out = []
    Uo, Lo = U.astype(np.int32), L.astype(np.int32)
    for M in (U, L):
        M = M.copy()
        M[M < -40000] = sentinel
        t = torch.full((n + 1, ld), 0, dtype=dtype, device="cuda")
        t[:, : n + 1] = torch.from_numpy(M).to(dtype).cuda()
        out.append(t)
    return out[0], out[1], ld, Uo, Lo


def _oracle_merge(Uo, Lo, dtype):
    D, K = oracle.merge(Uo, Lo)
    D = D.astype(np.int64)
    if dtype == torch.int16:
        D[D == np.iinfo(np.int32).min] = np.iinfo(np.int16).min
    return D, K.astype(np.int64)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    yield c
    B.lcs_destroy(c)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int16])
def test_static_merge_matches_lcs_merge_twice(ctx, dtype):
    for call, (seed, n) in enumerate([(11, 1024), (12, 333)]):      # two calls in a row
        U, L, ld, Uo, Lo = _operands(seed + (dtype == torch.int16), n, dtype)
        d_ref = torch.full_like(U, 9)
        k_ref = torch.full(U.shape, -9, dtype=torch.int32, device="cuda")
        B.lcs_merge(ctx, U, L, d_ref, k_ref)
        B.lcs_sync(ctx)
        d_st = torch.full_like(U, 7)
        k_st = torch.full(U.shape, -7, dtype=torch.int32, device="cuda")
        B.lcs_merge_static(U, L, d_st, k_st)
        assert torch.equal(d_st[:, : n + 1], d_ref[:, : n + 1]), (call, n)
        assert torch.equal(k_st[:, : n + 1], k_ref[:, : n + 1]), (call, n)
        D_want, K_want = _oracle_merge(Uo, Lo, dtype)
        assert np.array_equal(d_st[:, : n + 1].cpu().numpy().astype(np.int64), D_want), (call, n)
        assert np.array_equal(k_st[:, : n + 1].cpu().numpy().astype(np.int64), K_want), (call, n)


def test_static_merge_without_argmax_and_limit(ctx):
    U, L, ld, Uo, Lo = _operands(21, 200, torch.int32)
    d_ref = torch.zeros_like(U)
    B.lcs_merge(ctx, U, L, d_ref)
    B.lcs_sync(ctx)
    d_st = torch.ones_like(U)
    B.lcs_merge_static(U, L, d_st)
    assert torch.equal(d_st[:, :201], d_ref[:, :201])
    assert np.array_equal(d_st[:, :201].cpu().numpy().astype(np.int64), _oracle_merge(Uo, Lo, torch.int32)[0])
    big = torch.zeros((1026, 1028), dtype=torch.int32, device="cuda")
    with pytest.raises(B.LcsError) as e:
        B.lcs_merge_static(big, big, torch.zeros_like(big))
    assert e.value.status == B.LCS_EINVAL
