"""lcs_path: the leftmost heaviest path's vertex list (Sec. II-D) equals the
oracle's, vertex for vertex."""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs

from test_gpu_parity import ALPH2, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 0)
    yield c
    B.lcs_destroy(c)


def gpu_path(ctx, a, b, h=0, cap=None):
    B.lcs_set_strip_height(ctx, h)
    m, n = len(a), len(b)
    cap = m + n + 1 if cap is None else cap
    out = torch.full((max(cap, 1), 2), -3, dtype=torch.int32, device="cuda")
    cnt = B.lcs_path(ctx, dev(a), dev(b), out[:cap] if cap else None)
    return out[:cnt].cpu().numpy().astype(np.int64), out


@pytest.mark.parametrize("h", [0, 1, 7, 64])
def test_path_matches_oracle(ctx, h):
    rng = np.random.default_rng(1100 + h)
    for m, n in [(1, 1), (1, 30), (30, 1), (40, 40), (100, 37), (37, 100), (257, 130), (130, 257), (600, 300)]:
        a, b = inputs.random_pair(rng, m, n, ALPH2 if (m + n) % 2 else inputs.ACGT)
        got, _ = gpu_path(ctx, a, b, h)
        assert np.array_equal(got, oracle.path(a, b))


def test_path_edge_cases(ctx):
    A = np.frombuffer(b"ACGTACGT", np.uint8)
    cases = [
        (np.zeros(0, np.uint8), np.zeros(0, np.uint8)),
        (np.zeros(0, np.uint8), A),
        (A, np.zeros(0, np.uint8)),
        (A, A.copy()),                                           # the diagonal
        (np.full(50, 65, np.uint8), np.full(70, 67, np.uint8)),   # no match: right then down
        (np.full(64, 65, np.uint8), np.full(64, 65, np.uint8)),
        (np.full(300, 65, np.uint8), np.full(5, 65, np.uint8)),
    ]
    for a, b in cases:
        got, _ = gpu_path(ctx, a, b)
        want = oracle.path(a, b)
        assert np.array_equal(got, want)
        assert len(got) == len(a) + len(b) + 1 - oracle.lcs_length(a, b)


def test_path_cap_too_small(ctx):
    rng = np.random.default_rng(3)
    a, b = inputs.random_pair(rng, 50, 60)
    need = len(oracle.path(a, b))
    with pytest.raises(B.LcsError) as e:
        gpu_path(ctx, a, b, cap=need - 1)
    assert e.value.status == B.LCS_EOVERFLOW
    got, out = gpu_path(ctx, a, b, cap=need)
    assert np.array_equal(got, oracle.path(a, b))


@pytest.mark.parametrize("variant", ["iid", "correlated"])
def test_path_4096(ctx, variant):
    a, b = inputs.pair_4096(variant)
    got, _ = gpu_path(ctx, a, b)
    assert np.array_equal(got, oracle.path(a, b))
