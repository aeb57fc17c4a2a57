"""Failure detection on the GPU, exercised without faulting or hanging it.

* A device-side wait that runs out: lcs_set_fault_injection makes the first
  tile of an exact-merge launch announce its band on its mbarrier without
  copying anything, so the bounded wait (1 ms here) expires with nothing in
  flight.  The call must report LCS_ETIMEOUT through lcs_sync, and the same
  context must give oracle-exact results once the injection is off.
* A budget that no plan fits: LCS_ENOMEM, and the context stays usable.
"""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    yield c
    B.lcs_destroy(c)


def dev(x):
    return torch.from_numpy(np.array(x, dtype=np.uint8, copy=True)).cuda()


def _dense(M, ld):
    t = torch.zeros((M.shape[0], ld), dtype=torch.int32, device="cuda")
    t[:, : M.shape[1]] = torch.from_numpy(M.astype(np.int32)).cuda()
    return t


def test_merge_wait_runs_out_then_recovers(ctx):
    rng = np.random.default_rng(77)
    n = 300
    b = inputs.uniform(rng, n, inputs.ACGT)
    U = oracle.dist(inputs.uniform(rng, 40, inputs.ACGT), b)
    L = oracle.dist(inputs.uniform(rng, 50, inputs.ACGT), b)
    ld = (n + 1 + 3) // 4 * 4
    Ud, Ld = _dense(U, ld), _dense(L, ld)
    out = torch.zeros_like(Ud)
    B.lcs_set_fault_injection(ctx, True, 1_000_000)          # 1 ms
    try:
        B.lcs_merge(ctx, Ud, Ld, out)
        with pytest.raises(B.LcsError) as e:
            B.lcs_sync(ctx)
        assert e.value.status == B.LCS_ETIMEOUT
    finally:
        B.lcs_set_fault_injection(ctx, False, 0)
    k = torch.zeros_like(Ud)
    B.lcs_merge(ctx, Ud, Ld, out, k)
    B.lcs_sync(ctx)
    D_want, K_want = oracle.merge(U, L)
    assert np.array_equal(out[:, : n + 1].cpu().numpy(), D_want)
    assert np.array_equal(k[:, : n + 1].cpu().numpy(), K_want)


def test_solve_wait_runs_out_then_recovers(ctx):
    a, b = inputs.random_pair(np.random.default_rng(78), 700, 600)
    m, n = len(a), len(b)
    B.lcs_set_strip_height(ctx, 64)
    B.lcs_set_merge_kernel(ctx, B.LCS_MERGE_EXACT)
    ld = (n + 1 + 3) // 4 * 4
    d = torch.zeros((n + 1, ld), dtype=torch.int32, device="cuda")
    out = torch.zeros(min(m, n), dtype=torch.uint8, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")
    try:
        B.lcs_set_fault_injection(ctx, True, 1_000_000)
        B.lcs_dist(ctx, dev(a), dev(b), d)
        with pytest.raises(B.LcsError) as e:
            B.lcs_sync(ctx)
        assert e.value.status == B.LCS_ETIMEOUT
        B.lcs_set_fault_injection(ctx, False, 0)
        B.lcs_solve(ctx, dev(a), dev(b), dist=d, out_lcs=out, out_len=ln)
        B.lcs_sync(ctx)
    finally:
        B.lcs_set_fault_injection(ctx, False, 0)
        B.lcs_set_merge_kernel(ctx, B.LCS_MERGE_AUTO)
        B.lcs_set_strip_height(ctx, 0)
    s_want, _ = oracle.traceback(a, b)
    L = int(ln.item())
    assert L == len(s_want) and bytes(out[:L].cpu().numpy()) == s_want
    assert np.array_equal(d[:, : n + 1].cpu().numpy(), oracle.dist(a, b))


def test_budget_too_small_is_enomem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a, b = inputs.random_pair(np.random.default_rng(79), 1024, 1024)
    small = B.lcs_create(0, 64 << 10)                         # 64 KiB: no plan fits
    try:
        d = torch.zeros((1025, 1028), dtype=torch.int32, device="cuda")
        with pytest.raises(B.LcsError) as e:
            B.lcs_solve(small, dev(a), dev(b), dist=d)
        assert e.value.status == B.LCS_ENOMEM
        # Still usable for a problem that fits.
        x, y = inputs.random_pair(np.random.default_rng(80), 40, 50)
        assert B.lcs_length(small, dev(x), dev(y)) == oracle.lcs_length(x, y)
    finally:
        B.lcs_destroy(small)
