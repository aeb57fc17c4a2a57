"""Breakout (D-form) matrices on the GPU against the oracle, element by
element: the strip's D-form (Sec. II-B-1) and the combination of two
(Sec. II-B-3, by monotone column minima)."""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

from test_gpu_parity import ALPH2, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"i32": (torch.int32, np.iinfo(np.int32).max), "i16": (torch.int16, np.iinfo(np.int16).max)}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    yield c
    B.lcs_destroy(c)


def want_of(D, inf):
    D = D.astype(np.int64).copy()
    D[D == oracle.INF] = inf
    return D


def buffer(n, h, tdt, pad=3):
    return torch.full((n + 1, h + 1 + pad), -9, dtype=tdt, device="cuda")


def gpu_strip_dform(ctx, a, b, tdt):
    h, n = len(a), len(b)
    out = buffer(n, h, tdt)
    B.lcs_strip_dform(ctx, dev(a), dev(b), out)
    B.lcs_sync(ctx)
    return out, out[:, : h + 1].cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("dt", ["i32", "i16"])
@pytest.mark.parametrize("h", [1, 5, 32, 33, 64, 100, 256])
def test_strip_dform(ctx, dt, h):
    tdt, inf = TDT[dt]
    rng = np.random.default_rng(40 + h)
    for n in [0, 1, 63, 200, 700]:
        alph = ALPH2 if n % 2 else inputs.ACGT
        a, b = inputs.uniform(rng, h, alph), inputs.uniform(rng, n, alph)
        _, got = gpu_strip_dform(ctx, a, b, tdt)
        assert np.array_equal(got, want_of(oracle.dform(oracle.dist(a, b), h), inf))


def test_strip_dform_no_match(ctx):
    a, b = np.full(40, 65, np.uint8), np.full(90, 67, np.uint8)
    _, got = gpu_strip_dform(ctx, a, b, torch.int32)
    assert np.array_equal(got[:, 0], np.arange(91))
    assert (got[:, 1:] == np.iinfo(np.int32).max).all()


@pytest.mark.parametrize("dt", ["i32", "i16"])
@pytest.mark.parametrize("hu,hl", [(1, 1), (7, 3), (32, 32), (33, 64), (100, 7), (256, 256)])
def test_dform_merge(ctx, dt, hu, hl):
    tdt, inf = TDT[dt]
    rng = np.random.default_rng(hu * 1000 + hl)
    for n in [0, 1, 50, 333]:
        alph = ALPH2 if (n + hu) % 2 else inputs.ACGT
        a1, a2, b = inputs.uniform(rng, hu, alph), inputs.uniform(rng, hl, alph), inputs.uniform(rng, n, alph)
        DU, DL = oracle.dform(oracle.dist(a1, b), hu), oracle.dform(oracle.dist(a2, b), hl)
        want = want_of(oracle.dform_combine(DU, DL), inf)
        du, dl = buffer(n, hu, tdt), buffer(n, hl, tdt)
        du[:, : hu + 1] = torch.from_numpy(want_of(DU, inf)).to(tdt).cuda()
        dl[:, : hl + 1] = torch.from_numpy(want_of(DL, inf)).to(tdt).cuda()
        out = buffer(n, hu + hl, tdt)
        B.lcs_dform_merge(ctx, du, hu, dl, hl, out)
        B.lcs_sync(ctx)
        got = out[:, : hu + hl + 1].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want)
        # associativity: the D-form of the stacked strip's DIST
        assert np.array_equal(got, want_of(oracle.dform(oracle.dist(np.concatenate([a1, a2]), b), hu + hl), inf))


def test_strip_dform_many_strips(ctx):
    """All strips of a in one launch, the last one shorter than h."""
    rng = np.random.default_rng(5)
    a, b = inputs.random_pair(rng, 5 * 64 + 17, 300)
    n, h = len(b), 64
    S = -(-len(a) // h)
    out = torch.full((S, n + 1, h + 4), -9, dtype=torch.int32, device="cuda")
    B.lcs_strip_dform(ctx, dev(a), dev(b), out, h=h)
    B.lcs_sync(ctx)
    got = out[:, :, : h + 1].cpu().numpy().astype(np.int64)
    inf = np.iinfo(np.int32).max
    for s in range(S):
        strip = a[s * h:(s + 1) * h]
        want = np.full((n + 1, h + 1), inf, dtype=np.int64)
        want[:, : len(strip) + 1] = want_of(oracle.dform(oracle.dist(strip, b), len(strip)), inf)
        assert np.array_equal(got[s], want)


def test_dform_tree_4096(ctx):
    """Three levels on the 4096 iid pair's first 1024 rows: four 256-row strips
    in D-form, merged pairwise and then once more, against the D-form of the
    1024-row DIST."""
    a, b = inputs.pair_4096("iid")
    a = a[:1024]
    n = len(b)
    strips = torch.full((4, n + 1, 260), -9, dtype=torch.int16, device="cuda")
    B.lcs_strip_dform(ctx, dev(a), dev(b), strips, h=256)
    leaves = [strips[s] for s in range(4)]
    mids = []
    for q in range(2):
        out = buffer(n, 512, torch.int16)
        B.lcs_dform_merge(ctx, leaves[2 * q], 256, leaves[2 * q + 1], 256, out)
        mids.append(out)
    top = buffer(n, 1024, torch.int16)
    B.lcs_dform_merge(ctx, mids[0], 512, mids[1], 512, top)
    B.lcs_sync(ctx)
    got = top[:, :1025].cpu().numpy().astype(np.int64)
    want = want_of(oracle.dform(oracle.dist(a, b), 1024), np.iinfo(np.int16).max)
    assert np.array_equal(got, want)


def test_dform_invalid(ctx):
    a, b = dev(np.full(10, 65, np.uint8)), dev(np.full(10, 65, np.uint8))
    small = torch.zeros((11, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(B.LcsError):
        B.lcs_strip_dform(ctx, a, b, small)             # ldf < h + 1
    big = torch.zeros((11, 20), dtype=torch.int32, device="cuda")
    with pytest.raises(B.LcsError):
        B.lcs_dform_merge(ctx, big, 19, big, 19, small)   # ldo < hu + hl + 1
