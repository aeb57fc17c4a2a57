"""Continuous batching (serve.py over lcs_batch_submit/poll): requests that
arrive while others are on the GPU are admitted and overlap with them, and
every result is the same alone and in the mix (exactly: lengths and LCS
strings are integers)."""
import numpy as np
import pytest

import oracle
from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import inputs, serve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_serving_mix_equals_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    times, pairs = inputs.serving_requests(duration_s=0.25)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    ctx = B.lcs_create(0, 0)
    try:
        out = serve.serve(ctx, dev, times)
        assert out.batches > 1                    # arrivals spread over several batches
        assert (out.status == 0).all()
        assert np.isfinite(out.latency_s).all() and (out.latency_s > 0).all()
        for q, (a, b) in enumerate(dev):
            t = B.lcs_batch_submit(ctx, [(a, b, True)])
            r = B.lcs_batch_poll(ctx, t, 1, -1)[0]
            s = B.lcs_batch_strings(ctx, t)
            B.lcs_batch_release(ctx, t)
            assert r["len"] == out.length[q], q
            assert s[: r["len"]] == out.strings[q], q
        # Exact against the oracle on the pairs it runs in well under a second.
        small = [q for q, (a, b) in enumerate(pairs) if len(a) * len(b) <= 4_000_000][:40]
        for q in small:
            ref, _ = oracle.traceback(*pairs[q])
            assert out.length[q] == len(ref) and out.strings[q] == ref, q
        big = [q for q, (a, b) in enumerate(pairs) if len(a) == 16384]
        assert big, "the workload has pairs of 16384"
        a, b = pairs[big[0]]
        assert out.length[big[0]] == oracle.lcs_length(a, b)
    finally:
        B.lcs_destroy(ctx)
