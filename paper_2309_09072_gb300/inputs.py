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
    pos_of = {int(c): i for i, c in enumerate(alphabet)}
    out = []
    for x in range(len(a)):
        ch = int(a[x])
        if u[x] < p_indel:
            if coin[x] < 0.5:
                out.append(int(alphabet[ins_letter[x]]))
                out.append(ch)
            # else: deletion, the letter is dropped
        elif u[x] < p_indel + p_sub:
            out.append(int(alphabet[(pos_of[ch] + sub_shift[x]) % k]))
        else:
            out.append(ch)
    b = np.array(out, dtype=np.uint8)
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


def random_pair(rng: np.random.Generator, m: int, n: int, alphabet: np.ndarray = ACGT):
    return uniform(rng, m, alphabet), uniform(rng, n, alphabet)
