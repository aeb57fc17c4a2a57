"""The seeded input recipes (host logic, no GPU).

Each workload's generator is checked against its stated recipe: alphabet,
lengths, seeds, distributions, and the correlated partner's edit rates.
Where the LCS itself is the evidence, the oracle's two-row DP supplies it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import inputs

ACGT = set(b"ACGT")


def test_small_pair_and_determinism():
    a, b = inputs.pair_small(0)
    a2, b2 = inputs.pair_small(0)
    assert len(a) == len(b) == 64 and a.dtype == np.uint8
    assert set(a.tolist()) <= ACGT and set(b.tolist()) <= ACGT
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert not np.array_equal(inputs.pair_small(1)[0], a)


def test_pair_4096_iid_and_correlated():
    a, b = inputs.pair_4096("iid")
    assert len(a) == len(b) == 4096 and set(np.unique(a).tolist()) == ACGT
    for x in (a, b):
        freq = np.bincount(x, minlength=256)[list(ACGT)] / len(x)
        assert np.all(np.abs(freq - 0.25) < 0.03)
    ac, bc = inputs.pair_4096("correlated")
    assert np.array_equal(ac, a)                       # a is drawn first, from the same seed
    assert len(bc) == 4096 and set(bc.tolist()) <= ACGT
    # Two i.i.d. ACGT strings share about 0.65 of their length; a partner
    # with 10% substitutions and 5% indels about 0.88.
    assert oracle.lcs_length(a, b) < 0.70 * 4096
    assert oracle.lcs_length(ac, bc) > 0.85 * 4096
    with pytest.raises(ValueError):
        inputs.pair_4096("other")


def test_mutate_rates():
    rng = np.random.default_rng(7)
    a = inputs.uniform(rng, 8000, inputs.ACGT)
    # Substitutions only: 10% of the positions change, each to another letter.
    b = inputs.mutate(np.random.default_rng(8), a, 0.10, 0.0, inputs.ACGT)
    assert len(b) == len(a)
    assert abs(np.mean(a != b) - 0.10) < 0.012
    # Indels only: half of 5% delete a letter, half insert one, so a minus its
    # deleted letters (about 2.5%) is a common subsequence.
    b = inputs.mutate(np.random.default_rng(9), a, 0.0, 0.05, inputs.ACGT)
    assert abs(len(b) - len(a)) < 0.01 * len(a)
    lost = 1.0 - oracle.lcs_length(a, b) / len(a)
    assert 0.015 < lost < 0.035
    # A fixed output length truncates or pads.
    for want in (100, 9000):
        assert len(inputs.mutate(np.random.default_rng(10), a, 0.1, 0.05, inputs.ACGT, out_len=want)) == want


def test_zipf20_frequencies():
    a, b = inputs.pair_16384()
    assert len(a) == len(b) == 16384 and a.max() <= 19
    p = np.arange(1, 21, dtype=np.float64) ** -1.1
    p /= p.sum()
    freq = np.bincount(np.concatenate([a, b]), minlength=20) / (2 * 16384)
    # Rank r is byte r - 1; binomial standard error at 32768 draws is < 0.003.
    assert np.all(np.abs(freq - p) < 0.012)
    assert freq.argmax() == 0


def test_loguniform_lengths():
    rng = np.random.default_rng(11)
    x = inputs.loguniform_lengths(rng, 100000, 32, 2048)
    assert x.min() >= 32 and x.max() <= 2048
    mid = math.exp((math.log(32) + math.log(2049)) / 2)
    assert abs(np.median(x) / mid - 1.0) < 0.05
    # Equal mass per factor of two: [32, 64) and [1024, 2048) hold about 1/6 each.
    assert abs(np.mean(x < 64) - 1 / 6) < 0.01 and abs(np.mean(x >= 1024) - 1 / 6) < 0.01


def test_batch_pairs():
    pairs = inputs.batch_pairs()
    assert len(pairs) == 20000
    ms = np.array([len(p[0]) for p in pairs])
    ns = np.array([len(p[1]) for p in pairs])
    assert ms.min() >= 32 and ms.max() <= 2048 and ns.min() >= 32 and ns.max() <= 2048
    assert all(set(np.unique(x).tolist()) <= ACGT for x, _ in pairs[:200])


def test_serving_requests():
    times, req = inputs.serving_requests(duration_s=2.0)
    assert np.all(np.diff(times) >= 0) and times[0] >= 0 and times[-1] < 2.0
    assert abs(len(req) - 4000) < 5 * math.sqrt(4000)          # Poisson at 2,000 pairs/s for 2 s
    for k, (a, b) in enumerate(req):
        assert a.max(initial=0) <= 19 and b.max(initial=0) <= 19
        if (k + 1) % 50 == 0:
            # m = 16384; n = 16384 too, unless b is a's correlated partner,
            # which keeps the length its edits give it.
            assert len(a) == 16384 and abs(len(b) - 16384) < 0.02 * 16384
        else:
            assert 128 <= len(a) <= 8192
    # A correlated b keeps about a's length; two independent log-uniform
    # lengths rarely agree within 10%, so about 0.3 + 0.7 * 0.05 of the
    # ordinary pairs do.
    ordinary = [(a, b) for k, (a, b) in enumerate(req) if (k + 1) % 50]
    close = np.mean([abs(len(b) - len(a)) <= 0.1 * len(a) for a, b in ordinary])
    assert 0.27 < close < 0.42
    # Another rate scales the count.
    t8, r8 = inputs.serving_requests(duration_s=0.5, rate=8000.0)
    assert abs(len(r8) - 4000) < 5 * math.sqrt(4000)
