"""Continuous batching of LCS requests over the library's batch entry points.

Requests (pairs of device strings) arrive over time.  Every tick the loop
submits the requests that have arrived and are not yet admitted as one batch
(lcs_batch_submit): each batch runs on streams of its own, so a batch
admitted while others are still on the GPU overlaps with them.  A batch that
does not fit the context's memory budget next to the batches in flight is
refused (EAGAIN) and its requests wait until finished batches have been
released.  Finished batches are found by non-blocking polls.  Each request
gets two latencies, both from its arrival on the monotonic clock the library
uses: to its batch's device completion, and to the loop's receipt of the
result on the host (after the poll and the copy of the batch's strings).

Each batch in flight has streams of its own, so a process that serves at a
high rate should raise CUDA_DEVICE_MAX_CONNECTIONS (32, say) before CUDA is
initialised.  With the default 8 hardware queues the streams of dozens of
batches share them, and a small batch's kernels wait behind another batch's
long sweeps.

This module schedules and records only; every computation runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque

import numpy as np

from . import binding as B


class ServeResult:
    def __init__(self, count):
        self.length = np.full(count, -1, dtype=np.int64)
        self.latency_s = np.full(count, np.nan)        # device completion - arrival
        self.host_latency_s = np.full(count, np.nan)   # receipt on the host - arrival
        self.strings = [b""] * count
        self.status = np.zeros(count, dtype=np.int64)
        self.batches = 0
        self.refused = 0
        self.wall_s = 0.0


def serve(ctx, pairs, arrivals, want_strings=True, max_batch=4096, tick_s=0.0005):
    """Run `pairs` (list of (a, b) device uint8 tensors) arriving at
    `arrivals` (seconds from the start, nondecreasing) through continuous
    batching on `ctx`.  Returns a ServeResult."""
    lib = B.load()
    count = len(pairs)
    out = ServeResult(count)
    order = np.argsort(arrivals, kind="stable")
    pending = deque()                     # arrived, not yet admitted
    nxt = 0                               # next request (in arrival order) to arrive
    inflight = {}                         # ticket -> (indices, lcs_result array)
    t0 = time.monotonic()
    done = 0
    while done < count:
        now = time.monotonic() - t0
        while nxt < count and arrivals[order[nxt]] <= now:
            pending.append(int(order[nxt]))
            nxt += 1
        if pending:
            idx = [pending.popleft() for _ in range(min(len(pending), max_batch))]
            arr = (B.lcs_pair * len(idx))()
            for k, q in enumerate(idx):
                a, b = pairs[q]
                arr[k].a = a.data_ptr() if a.numel() else None
                arr[k].m = int(a.numel())
                arr[k].b = b.data_ptr() if b.numel() else None
                arr[k].n = int(b.numel())
                arr[k].flags = B.LCS_WANT_STRING if want_strings else 0
            ticket = ctypes.c_uint64()
            st = lib.lcs_batch_submit(ctx, arr, len(idx), ctypes.byref(ticket))
            if st == B.LCS_OK:
                inflight[ticket.value] = (idx, (B.lcs_result * len(idx))())
                out.batches += 1
            elif st == B.LCS_EAGAIN and inflight:
                out.refused += 1
                pending.extendleft(reversed(idx))      # wait for memory to free up
            else:
                B._check(ctx, st)
        finished = []
        for tk, (idx, res) in inflight.items():
            n_done = ctypes.c_int64()
            B._check(ctx, lib.lcs_batch_poll(ctx, tk, res, len(idx), ctypes.byref(n_done), 0))
            if n_done.value:
                finished.append(tk)
        for tk in finished:
            idx, res = inflight.pop(tk)
            strings = B.lcs_batch_strings(ctx, tk) if want_strings else b""
            t_host = time.monotonic()
            B.lcs_batch_release(ctx, tk)
            for k, q in enumerate(idx):
                r = res[k]
                out.length[q] = r.len
                out.status[q] = r.status
                out.latency_s[q] = r.t_done - (t0 + arrivals[q])
                out.host_latency_s[q] = t_host - (t0 + arrivals[q])
                if want_strings and r.string_offset >= 0:
                    out.strings[q] = strings[r.string_offset: r.string_offset + r.len]
            done += len(idx)
        if not finished and not pending:
            wait = tick_s
            if nxt < count:
                wait = min(wait, max(0.0, arrivals[order[nxt]] - (time.monotonic() - t0)))
            if wait > 0:
                time.sleep(wait)
    out.wall_s = time.monotonic() - t0
    return out


def summary(out: ServeResult, pairs_mn):
    """p50/p99 latency (ms), throughput (GCUPS over the wall time), counts."""
    lat = out.latency_s[np.isfinite(out.latency_s)] * 1e3
    hl = out.host_latency_s[np.isfinite(out.host_latency_s)] * 1e3
    cells = float(sum(m * n for m, n in pairs_mn))
    pct = lambda x, q: float(np.percentile(x, q)) if len(x) else None
    return {"requests": len(out.length), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "max_ms": float(lat.max()) if len(lat) else None,
            "host_p50_ms": pct(hl, 50), "host_p99_ms": pct(hl, 99),
            "host_max_ms": float(hl.max()) if len(hl) else None, "gcups": cells / out.wall_s / 1e9,
            "wall_s": out.wall_s, "batches": out.batches, "refused_submits": out.refused,
            "failed": int((out.status != 0).sum())}
