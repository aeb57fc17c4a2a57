"""The serving loop's host logic against a fake of the batch entry points
(no GPU): admission, refusal (EAGAIN) and requeueing, polling, latency
bookkeeping, and result routing back to each request.

The fake's per-pair "result" is a stand-in (the length min(m, n) and a's
first min(m, n) letters): what is tested is the loop, not the LCS.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

from paper_2309_09072_gb300 import binding as B
from paper_2309_09072_gb300 import serve


class FakeBatchLib:
    """lcs_batch_submit / poll / strings / release with a fixed completion
    delay per batch and a cap on pairs in flight (EAGAIN beyond it)."""

    def __init__(self, delay_s=0.002, capacity=10 ** 9):
        self.delay_s, self.capacity = delay_s, capacity
        self.tickets, self.next = {}, 1
        self.refusals = 0
        self.max_inflight = 0

    def _inflight(self):
        return sum(len(t["pairs"]) for t in self.tickets.values())

    def lcs_batch_submit(self, ctx, arr, count, ticket_ref):
        if self.tickets and self._inflight() + count > self.capacity:
            self.refusals += 1
            return B.LCS_EAGAIN
        pairs = []
        for k in range(count):
            p = arr[k]
            a = ctypes.string_at(p.a, p.m) if p.m else b""
            b = ctypes.string_at(p.b, p.n) if p.n else b""
            pairs.append((a, b))
        t = self.next
        self.next += 1
        self.tickets[t] = {"pairs": pairs, "t_submit": time.monotonic()}
        ticket_ref._obj.value = t
        self.max_inflight = max(self.max_inflight, self._inflight())
        return B.LCS_OK

    def _strings(self, t):
        return b"".join(a[: min(len(a), len(b))] for a, b in self.tickets[t]["pairs"])

    def lcs_batch_poll(self, ctx, t, res, cap, done_ref, timeout_ms):
        if t not in self.tickets:
            return B.LCS_EINVAL
        rec = self.tickets[t]
        ready = time.monotonic() >= rec["t_submit"] + self.delay_s
        off = 0
        if ready:
            for k, (a, b) in enumerate(rec["pairs"][:cap]):
                L = min(len(a), len(b))
                res[k].len, res[k].string_offset, res[k].status = L, off, B.LCS_OK
                res[k].t_submit, res[k].t_done = rec["t_submit"], rec["t_submit"] + self.delay_s
                off += L
        done_ref._obj.value = len(rec["pairs"]) if ready else 0
        return B.LCS_OK

    def lcs_batch_strings(self, ctx, t, buf, cap, size_ref):
        s = self._strings(t)
        size_ref._obj.value = len(s)
        if buf is None or cap < len(s):
            return B.LCS_EOVERFLOW
        ctypes.memmove(buf, s, len(s))
        return B.LCS_OK

    def lcs_batch_release(self, ctx, t):
        return B.LCS_OK if self.tickets.pop(t, None) is not None else B.LCS_EINVAL

    def lcs_last_error(self, ctx):
        return b""


@pytest.fixture
def fake(monkeypatch):
    lib = FakeBatchLib()
    monkeypatch.setattr(B, "load", lambda *a, **k: lib)
    return lib


def _requests(count, seed=0):
    rng = np.random.default_rng(seed)
    pairs = []
    for _ in range(count):
        m, n = (int(x) for x in rng.integers(0, 40, size=2))
        pairs.append((torch.from_numpy(rng.integers(65, 69, size=m).astype(np.uint8)),
                      torch.from_numpy(rng.integers(65, 69, size=n).astype(np.uint8))))
    arrivals = np.sort(rng.uniform(0.0, 0.03, size=count))
    return pairs, arrivals


def _check_results(out, pairs, delay_s):
    for q, (a, b) in enumerate(pairs):
        L = min(a.numel(), b.numel())
        assert out.status[q] == B.LCS_OK and out.length[q] == L
        assert out.strings[q] == bytes(a[:L].numpy())
        # Completion is the batch's submit plus the delay, never before arrival + delay.
        assert delay_s - 1e-6 <= out.latency_s[q] < delay_s + 0.5


def test_every_request_completes_with_its_own_result(fake):
    pairs, arrivals = _requests(300)
    out = serve.serve(None, pairs, arrivals)
    _check_results(out, pairs, fake.delay_s)
    assert out.batches >= 1 and out.refused == 0 and not fake.tickets      # all released
    s = serve.summary(out, [(a.numel(), b.numel()) for a, b in pairs])
    assert s["requests"] == 300 and s["failed"] == 0 and s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    assert s["host_p50_ms"] <= s["host_p99_ms"] <= s["host_max_ms"]
    # The host receives a result only after the batch has completed.
    assert np.all(out.host_latency_s >= out.latency_s - 1e-6)


def test_refused_batches_wait_for_memory_and_still_complete(fake):
    fake.capacity = 20                    # pairs in flight
    pairs, arrivals = _requests(300, seed=1)
    out = serve.serve(None, pairs, arrivals, max_batch=16)
    _check_results(out, pairs, fake.delay_s)
    assert out.refused > 0 and fake.refusals == out.refused
    assert fake.max_inflight <= 20 and not fake.tickets


def test_without_strings(fake):
    pairs, arrivals = _requests(50, seed=2)
    out = serve.serve(None, pairs, arrivals, want_strings=False)
    assert all(s == b"" for s in out.strings)
    assert all(out.length[q] == min(a.numel(), b.numel()) for q, (a, b) in enumerate(pairs))
