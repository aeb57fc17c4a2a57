"""Seeded synthetic inputs for the LCS workloads (strings only, no LCS arithmetic).

This module is shared by the tests, the benchmark and the smoke check.  It draws
byte strings and nothing else: it holds none of the method's arithmetic, so the
CPU oracle and the CUDA path can both be fed from it without sharing any code.

The paper states neither the alphabet nor the distribution of its inputs
(Sec. III-B), so the workloads are synthetic:

* ``uniform``: i.i.d. letters of an alphabet (``ACGT`` bytes 65/67/71/84 for the
  4-letter workloads, bytes 0..19 for the 20-letter ones).
* ``zipf20``: 20 letters with P(rank r) proportional to r**-s, r = 1..20.
* ``mutate``: a correlated partner of ``a``: a walk over ``a`` that, per
  position, makes an indel event with probability ``p_indel`` (50/50 insert a
  uniform letter before the position or delete it) or else substitutes a
  different uniform letter with probability ``p_sub``; the result is truncated
  or padded with uniform letters to the requested length.
* ``loguniform_lengths``: floor(exp(U(ln lo, ln (hi + 1)))) clipped to [lo, hi].
* ``serving_requests``: Poisson arrivals (exponential gaps), every 50th pair
  m = n = 16384, the others log-uniform in [128, 8192], 30% correlated.

Seeds: ``numpy.random.default_rng(seed)``; ``a`` is drawn before ``b``.
"""
from __future__ import annotations

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8).copy()
AA20 = np.arange(20, dtype=np.uint8)


def uniform(rng: np.random.Generator, length: int, alphabet: np.ndarray) -> np.ndarray:
    """``length`` i.i.d. letters drawn uniformly from ``alphabet`` (uint8)."""
    idx = rng.integers(0, len(alphabet), size=int(length))
    return np.ascontiguousarray(alphabet[idx], dtype=np.uint8)


def zipf20(rng: np.random.Generator, length: int, s: float = 1.1) -> np.ndarray:
    """``length`` letters over bytes 0..19 with Zipf(s) rank frequencies."""
    ranks = np.arange(1, 21, dtype=np.float64)
    p = ranks ** (-s)
    p /= p.sum()
    return rng.choice(AA20, size=int(length), p=p).astype(np.uint8)


def mutate(rng: np.random.Generator, a: np.ndarray, p_sub: float, p_indel: float,
           alphabet: np.ndarray, out_len: int | None = None) -> np.ndarray:
    """Correlated partner of ``a`` (substitutions + insertions/deletions)."""
    a = np.asarray(a, dtype=np.uint8)
    k = len(alphabet)
    u = rng.random(len(a))
    coin = rng.random(len(a))
    ins_letter = rng.integers(0, k, size=len(a))
    sub_shift = rng.integers(1, k, size=len(a))   # a *different* letter
    pos_of = np.zeros(256, dtype=np.int64)
    pos_of[np.asarray(alphabet, dtype=np.uint8)] = np.arange(k)
    indel = u < p_indel
    ins = indel & (coin < 0.5)                    # a uniform letter, then the position's
    dele = indel & (coin >= 0.5)                  # the position's letter is dropped
    sub = ~indel & (u < p_indel + p_sub)
    letter = a.copy()
    letter[sub] = np.asarray(alphabet, dtype=np.uint8)[(pos_of[a[sub]] + sub_shift[sub]) % k]
    counts = 1 - dele.astype(np.int64) + ins.astype(np.int64)
    start = np.cumsum(counts) - counts
    b = np.empty(int(counts.sum()), dtype=np.uint8)
    keep = counts > 0
    b[start[keep] + ins[keep]] = letter[keep]
    b[start[ins]] = np.asarray(alphabet, dtype=np.uint8)[ins_letter[ins]]
    if out_len is not None:
        if len(b) >= out_len:
            b = b[:out_len]
        else:
            b = np.concatenate([b, uniform(rng, out_len - len(b), alphabet)])
    return np.ascontiguousarray(b)


def loguniform_lengths(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    x = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=int(count))))
    return np.clip(x, lo, hi).astype(np.int64)


# --------------------------------------------------------------------------
# The named workloads.  Each returns (a, b) as contiguous uint8 arrays.
# --------------------------------------------------------------------------

def pair_small(seed: int = 0, m: int = 64, n: int = 64):
    """Single pair m = n = 64, uniform ACGT (the small parity workload)."""
    rng = np.random.default_rng(seed)
    return uniform(rng, m, ACGT), uniform(rng, n, ACGT)


def pair_4096(variant: str = "iid", seed: int = 1, m: int = 4096, n: int = 4096):
    """Single pair m = n = 4096 over ACGT: ``iid`` or ``correlated``
    (b = a with 10% substitutions and 5% insertions/deletions)."""
    rng = np.random.default_rng(seed)
    a = uniform(rng, m, ACGT)
    if variant == "iid":
        b = uniform(rng, n, ACGT)
    elif variant == "correlated":
        b = mutate(rng, a, 0.10, 0.05, ACGT, out_len=n)
    else:
        raise ValueError(variant)
    return a, b


def pair_16384(seed: int = 2, m: int = 16384, n: int = 16384):
    """Single pair m = n = 16384 over 20 letters with Zipf(1.1) frequencies."""
    rng = np.random.default_rng(seed)
    return zipf20(rng, m), zipf20(rng, n)


def batch_pairs(count: int = 20000, seed: int = 3, lo: int = 32, hi: int = 2048):
    """``count`` independent pairs, m and n log-uniform in [lo, hi], ACGT."""
    rng = np.random.default_rng(seed)
    ms = loguniform_lengths(rng, count, lo, hi)
    ns = loguniform_lengths(rng, count, lo, hi)
    pairs = []
    for m, n in zip(ms, ns):
        a = uniform(rng, m, ACGT)
        b = uniform(rng, n, ACGT)
        pairs.append((a, b))
    return pairs


def serving_requests(duration_s: float = 60.0, rate: float = 2000.0, seed: int = 4,
                     lo: int = 128, hi: int = 8192, every_big: int = 50, big: int = 16384,
                     p_correlated: float = 0.30):
    """Poisson arrivals at ``rate`` pairs/s for ``duration_s`` seconds over the
    20 letters (bytes 0..19, uniform): lengths log-uniform in [lo, hi], every
    ``every_big``-th pair m = n = ``big``; a fraction ``p_correlated`` of the
    pairs have b = a with 10% substitutions and 5% insertions/deletions.
    Returns (arrival times in seconds, list of (a, b))."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(duration_s * rate * 1.2) + 16)
    times = np.cumsum(gaps)
    times = times[times < duration_s]
    pairs = []
    for k in range(len(times)):
        if (k + 1) % every_big == 0:
            m = n = big
        else:
            m, n = (int(x) for x in loguniform_lengths(rng, 2, lo, hi))
        a = uniform(rng, m, AA20)
        if rng.random() < p_correlated:
            b = mutate(rng, a, 0.10, 0.05, AA20)
        else:
            b = uniform(rng, n, AA20)
        pairs.append((a, b))
    return times, pairs


def random_pair(rng: np.random.Generator, m: int, n: int, alphabet: np.ndarray = ACGT):
    return uniform(rng, m, alphabet), uniform(rng, n, alphabet)
