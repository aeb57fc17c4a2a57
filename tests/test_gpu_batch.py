"""Batches of independent pairs (lcs_batch_submit / lcs_batch_poll) against
the CPU oracle: every length and every LCS string bit-exact, the string being
the leftmost heaviest path's letters (the same rule as single pairs)."""
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
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint8)).cuda()


def run_batch(ctx, pairs, want=True):
    """pairs: list of (a, b) numpy arrays, or (a, b, want); returns results and strings."""
    tens = [(dev(p[0]), dev(p[1]), p[2] if len(p) > 2 else want) for p in pairs]
    t = B.lcs_batch_submit(ctx, tens)
    res = B.lcs_batch_poll(ctx, t, len(tens), -1)
    strings = B.lcs_batch_strings(ctx, t)
    B.lcs_batch_release(ctx, t)
    return res, strings


def is_subsequence(s, x):
    it = iter(x)
    return all(ch in it for ch in s)


def check_exact(pairs, res, strings, want=True):
    assert len(res) == len(pairs)
    for k, p in enumerate(pairs):
        a, b = p[0], p[1]
        w = p[2] if len(p) > 2 else want
        r = res[k]
        assert r["status"] == B.LCS_OK, k
        ref_s, _ = oracle.traceback(a, b)
        assert r["len"] == len(ref_s), (k, len(a), len(b))
        if w:
            got = strings[r["string_offset"]: r["string_offset"] + r["len"]]
            assert got == ref_s, (k, len(a), len(b))
        else:
            assert r["string_offset"] == -1


def test_batched_workload_sample(ctx):
    # The batched workload's generator (log-uniform lengths in [32, 2048],
    # ACGT): the first 300 pairs, every length and string against the oracle.
    pairs = inputs.batch_pairs(count=300)
    res, strings = run_batch(ctx, pairs)
    check_exact(pairs, res, strings)


def test_batch_edge_cases(ctx):
    rng = np.random.default_rng(11)
    acgt = inputs.ACGT
    many = np.arange(40, dtype=np.uint8) + 60                  # 40 letters: no shared mask table
    pairs = [
        (np.zeros(0, np.uint8), acgt[:5]),                       # empty a
        (acgt[:5], np.zeros(0, np.uint8)),                       # empty b
        (np.zeros(0, np.uint8), np.zeros(0, np.uint8)),
        (acgt[:1], acgt[:1]),                                    # 1 x 1 match
        (acgt[:1], acgt[1:2]),                                   # 1 x 1 mismatch
        (inputs.uniform(rng, 2048, acgt), inputs.uniform(rng, 700, acgt)),      # 64 words, tallest strip
        (inputs.uniform(rng, 2049, acgt), inputs.uniform(rng, 300, acgt)),      # next size class
        (inputs.uniform(rng, 4096, acgt), inputs.uniform(rng, 500, acgt)),
        (inputs.uniform(rng, 4097, acgt), inputs.uniform(rng, 500, acgt)),
        (inputs.uniform(rng, 8193, acgt), inputs.uniform(rng, 200, acgt)),
        (inputs.uniform(rng, 16384, acgt), inputs.uniform(rng, 150, acgt)),    # tallest one-strip pair
        (inputs.uniform(rng, 16385, acgt), inputs.uniform(rng, 120, acgt)),    # too tall: the strip tree
        (inputs.uniform(rng, 33, acgt), inputs.uniform(rng, 5000, acgt)),       # two words, long b
        (inputs.uniform(rng, 300, many), inputs.uniform(rng, 400, many)),       # > 32 letters in a
        (inputs.uniform(rng, 1100, acgt),) * 2,                                  # identical
        (np.full(100, 65, np.uint8), np.full(90, 66, np.uint8)),                # disjoint
        (inputs.uniform(rng, 31, acgt), inputs.uniform(rng, 64, acgt), False),  # length only
        (inputs.uniform(rng, 1024, acgt), inputs.uniform(rng, 1024, acgt), False),
    ]
    pairs = [p if len(p) != 2 or p[0] is not p[1] else (p[0], p[1].copy()) for p in pairs]
    res, strings = run_batch(ctx, pairs)
    check_exact(pairs, res, strings)


def test_batch_serving_mix(ctx):
    # Requests shaped like the serving workload (20-letter alphabet, 30% of
    # pairs correlated, lengths log-uniform, one m = n pair per batch taller
    # than 2048): exact against the oracle, and the same results whether a
    # pair runs alone or in the mix.
    rng = np.random.default_rng(21)
    alph = np.arange(20, dtype=np.uint8) + 65
    ms = inputs.loguniform_lengths(rng, 40, 128, 3000)
    pairs = []
    for k, m in enumerate(ms):
        a = inputs.uniform(rng, int(m), alph)
        if k % 10 < 3:
            b = inputs.mutate(rng, a, 0.10, 0.05, alph)
        else:
            b = inputs.uniform(rng, int(inputs.loguniform_lengths(rng, 1, 128, 3000)[0]), alph)
        pairs.append((a, b))
    res, strings = run_batch(ctx, pairs)
    check_exact(pairs, res, strings)
    for k in (0, 7, 33):
        r1, s1 = run_batch(ctx, [pairs[k]])
        assert r1[0]["len"] == res[k]["len"]
        assert s1[: r1[0]["len"]] == strings[res[k]["string_offset"]: res[k]["string_offset"] + res[k]["len"]]


def test_batch_matches_single_pair_path(ctx):
    rng = np.random.default_rng(5)
    pairs = [inputs.random_pair(rng, int(m), int(n)) for m, n in [(700, 900), (2048, 2048), (64, 3000)]]
    res, strings = run_batch(ctx, pairs)
    for k, (a, b) in enumerate(pairs):
        out = torch.zeros(max(1, min(len(a), len(b))), dtype=torch.uint8, device="cuda")
        ln = B.lcs_traceback(ctx, dev(a), dev(b), out)
        assert res[k]["len"] == ln
        s = strings[res[k]["string_offset"]: res[k]["string_offset"] + ln]
        assert s == bytes(out[:ln].cpu().numpy().tobytes())


def test_batched_workload_full_size(ctx):
    # The batched workload at its full size (20,000 pairs): sampled pairs
    # exact against the oracle, every pair's string a common subsequence of
    # both strings with the reported length.
    pairs = inputs.batch_pairs()
    res, strings = run_batch(ctx, pairs)
    assert len(res) == len(pairs)
    for k in range(0, len(pairs), 97):
        a, b = pairs[k]
        ref_s, _ = oracle.traceback(a, b)
        got = strings[res[k]["string_offset"]: res[k]["string_offset"] + res[k]["len"]]
        assert res[k]["len"] == len(ref_s) and got == ref_s, k
    for k, (a, b) in enumerate(pairs):
        r = res[k]
        assert r["status"] == B.LCS_OK
        s = strings[r["string_offset"]: r["string_offset"] + r["len"]]
        assert len(s) == r["len"] <= min(len(a), len(b))
        assert is_subsequence(s, a.tobytes()) and is_subsequence(s, b.tobytes()), k
        assert r["t_done"] >= r["t_submit"]


def test_batch_admission_and_tickets():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = B.lcs_create(0, 1 << 18)                 # 256 KiB budget
    try:
        rng = np.random.default_rng(2)
        big = [(dev(inputs.uniform(rng, 2048, inputs.ACGT)), dev(inputs.uniform(rng, 2048, inputs.ACGT)), True)]
        with pytest.raises(B.LcsError) as e:
            B.lcs_batch_submit(c, big)           # 2049 x 64 words of columns = 512 KiB
        assert e.value.status == B.LCS_EAGAIN
        small = [(dev(inputs.uniform(rng, 100, inputs.ACGT)), dev(inputs.uniform(rng, 100, inputs.ACGT)), True)]
        t = B.lcs_batch_submit(c, small)
        assert B.lcs_batch_poll(c, t, 1, -1)[0]["status"] == B.LCS_OK
        B.lcs_batch_release(c, t)
        with pytest.raises(B.LcsError) as e:
            B.lcs_batch_release(c, t)            # already released
        assert e.value.status == B.LCS_EINVAL
        t = B.lcs_batch_submit(c, [])            # an empty batch is legal
        assert B.lcs_batch_poll(c, t, 0, -1) == []
        B.lcs_batch_release(c, t)
    finally:
        B.lcs_destroy(c)


def test_batch_pairs_taller_than_one_strip(ctx):
    """Pairs of 16385 to 32768 rows: the batch splits each at its middle row
    by the recomputing sweeps (the split column is the smallest maximiser of
    U(0, k) + L(k, n)), runs the two halves as one-strip pairs beside the
    others, and joins their lengths and strings.  Every result must equal the
    oracle's leftmost LCS, with and without strings, mixed with small pairs."""
    rng = np.random.default_rng(2024)
    pairs = []
    for m, n, want in [(16385, 1500, True), (20001, 2000, True), (32768, 1200, True), (25000, 700, False),
                       (17000, 1, True), (16500, 0, True)]:
        pairs.append((inputs.uniform(rng, m, inputs.ACGT), inputs.uniform(rng, n, inputs.ACGT), want))
    a = inputs.uniform(rng, 20000, inputs.ACGT)
    pairs.append((a, inputs.mutate(rng, a[8000:11000], 0.10, 0.05, inputs.ACGT), True))   # split inside the match
    a = inputs.uniform(rng, 18000, inputs.AA20)
    pairs.append((a, inputs.mutate(rng, a[:2500], 0.10, 0.05, inputs.AA20), True))          # all in the upper half
    for m, n in [(40, 90), (3000, 200), (5000, 4100)]:
        pairs.append((inputs.uniform(rng, m, inputs.ACGT), inputs.uniform(rng, n, inputs.ACGT), True))
    res, strings = run_batch(ctx, pairs)
    check_exact(pairs, res, strings)
