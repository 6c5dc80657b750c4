"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module holds no sorting arithmetic: it only draws keys.  Every generator
is built on raw 32-bit outputs of the Mersenne Twister MT19937 with the
standard integer seeding (the paper's generator, Sec. 5 "Input
permutations"), read through numpy's ``RandomState`` bit generator, so a given
seed gives the same keys on every machine.

Distributions (shapes of the paper's workloads, Sec. 5):

``uniform``   i.i.d. uniform uint32.
``zipf``      Zipf(s=1.1) ranks over 2**20 values by inverse-CDF sampling with
              an fp64 table; rank r maps to key r * 0x9E3779B1 mod 2**32 (a
              bijection of ranks, so distinct ranks give distinct keys).
``runs``      uniform keys, then consecutive segments of Geometric length
              (support 1, 2, ...; mean ``mean_run``) each sorted ascending --
              the paper's presortedness construction with S = mean_run.
``paper``     the paper's own recipe: values uniform in [100, 10**9], then the
              Geometric presort with parameter 1/S.
``updown``    like ``runs``, but a fair coin sorts each segment ascending or
              descending (inputs for the decreasing-run variant of Sec. 5).
``bands``     sorted blocks of 2**13 uniform keys, each block drawn from a
              value band below the previous block's (data appended in
              reverse order of a partitioning key): every merge puts one run
              wholly before the other.
``sorted`` / ``reversed`` / ``equal`` / ``few``   degenerate cases.
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0x9E3779B1


def mt_raw(seed: int, count: int) -> np.ndarray:
    """``count`` raw MT19937 outputs (uint32) after standard seeding with ``seed``."""
    rs = np.random.RandomState(seed)
    bg = rs._bit_generator  # legacy-seeded MT19937
    return bg.random_raw(count).astype(np.uint32)


def _unit_doubles(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits from pairs of raw outputs."""
    raw = mt_raw(seed, 2 * count).astype(np.uint64)
    a = raw[0::2] >> np.uint64(5)
    b = raw[1::2] >> np.uint64(6)
    return (a.astype(np.float64) * 67108864.0 + b.astype(np.float64)) / 9007199254740992.0


def uniform(n: int, seed: int) -> np.ndarray:
    return mt_raw(seed, n)


def zipf(n: int, seed: int, s: float = 1.1, values: int = 1 << 20) -> np.ndarray:
    ranks = np.arange(1, values + 1, dtype=np.float64)
    w = ranks ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = _unit_doubles(seed, n)
    r = np.searchsorted(cdf, u, side="right").astype(np.uint64) + np.uint64(1)
    r = np.minimum(r, np.uint64(values))
    return ((r * np.uint64(GOLDEN)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def geometric_lengths(total: int, seed: int, mean_run: float) -> np.ndarray:
    """Geometric(p = 1/mean_run) lengths on {1, 2, ...} covering ``total``."""
    if total <= 0:
        return np.zeros(0, np.int64)
    p = 1.0 / mean_run
    out = []
    covered = 0
    chunk_seed = seed
    while covered < total:
        need = max(16, int((total - covered) / mean_run * 1.2) + 16)
        u = _unit_doubles(chunk_seed, need)
        chunk_seed = (chunk_seed * 1103515245 + 12345) & 0x7FFFFFFF
        if p >= 1.0:
            lens = np.ones(need, np.int64)
        else:
            lens = np.floor(np.log1p(-u) / np.log1p(-p)).astype(np.int64) + 1
        out.append(lens)
        covered += int(lens.sum())
    lens = np.concatenate(out)
    cs = np.cumsum(lens)
    last = int(np.searchsorted(cs, total, side="left"))
    lens = lens[: last + 1].copy()
    lens[-1] -= int(cs[last] - total)
    return lens[lens > 0]


def presort_segments(keys: np.ndarray, lens: np.ndarray) -> np.ndarray:
    """Sort each consecutive segment of the given lengths ascending."""
    out = keys.copy()
    pos = 0
    for ln in lens.tolist():
        out[pos: pos + ln] = np.sort(out[pos: pos + ln], kind="stable")
        pos += ln
    return out


def presort_segments_fast(keys: np.ndarray, lens: np.ndarray) -> np.ndarray:
    """Vectorised :func:`presort_segments` (same result): lexsort by (segment, key)."""
    seg = np.repeat(np.arange(lens.size, dtype=np.int64), lens)
    order = np.lexsort((keys, seg))
    return keys[order]


def runs(n: int, seed: int, mean_run: float = 1024.0) -> np.ndarray:
    keys = mt_raw(seed, n)
    lens = geometric_lengths(n, seed + 7919, mean_run)
    return presort_segments_fast(keys, lens)


def updown(n: int, seed: int, mean_run: float = 1024.0) -> np.ndarray:
    """Geometric segments as in :func:`runs`, each sorted ascending or (coin) descending."""
    keys = mt_raw(seed, n)
    lens = geometric_lengths(n, seed + 7919, mean_run)
    down = (mt_raw(seed + 104729, lens.size) & np.uint32(1)).astype(bool)
    seg = np.repeat(np.arange(lens.size, dtype=np.int64), lens)
    sk = np.where(np.repeat(down, lens), ~keys, keys)
    return keys[np.lexsort((sk, seg))]


def bands(n: int, seed: int, block: int = 1 << 13) -> np.ndarray:
    """Sorted blocks of ``block`` keys in descending value bands (see module doc)."""
    nb = max(1, -(-n // block))
    width = (1 << 32) // nb
    raw = mt_raw(seed, n).astype(np.uint64)
    b = np.arange(n, dtype=np.int64) // block
    keys = ((nb - 1 - b).astype(np.uint64) * np.uint64(width) + raw % np.uint64(width)).astype(np.uint32)
    return presort_segments_fast(keys, np.diff(np.append(np.arange(0, n, block), n)))


def paper(n: int, seed: int, S: float = 2.0) -> np.ndarray:
    """Sec. 5 recipe: values uniform in [100, 10**9], presorted with parameter S."""
    raw = mt_raw(seed, n).astype(np.uint64)
    keys = (np.uint64(100) + raw % np.uint64(10 ** 9 - 100 + 1)).astype(np.uint32)
    if S <= 1:
        return keys
    lens = geometric_lengths(n, seed + 7919, S)
    return presort_segments_fast(keys, lens)


def make(dist: str, n: int, seed: int) -> np.ndarray:
    """Keys of one distribution by name."""
    if dist == "uniform":
        return uniform(n, seed)
    if dist == "zipf":
        return zipf(n, seed)
    if dist == "runs":
        return runs(n, seed)
    if dist == "paper":
        return paper(n, seed)
    if dist == "updown":
        return updown(n, seed)
    if dist == "bands":
        return bands(n, seed)
    if dist == "sorted":
        return np.sort(uniform(n, seed))
    if dist == "reversed":
        return np.sort(uniform(n, seed))[::-1].copy()
    if dist == "equal":
        return np.full(n, 7, np.uint32)
    if dist == "few":
        return (uniform(n, seed) % np.uint32(4)).astype(np.uint32)
    raise ValueError(f"unknown distribution {dist!r}")


def records(kind: str, n: int, seed: int, words: int = 30, S: float = 0.0) -> np.ndarray:
    """Records of ``words`` 32-bit words (rows of an (n, words) array), the
    paper's data types (Sec. 5 "Input data types"), values uniform in
    [100, 10**9]:

    ``random``  every word random (``randomBlob30``: most comparisons end at
                the first word);
    ``zero``    every word but the last is 0 (``zeroBlob30``, and the rows the
                ``ptr`` type points to: every comparison reads all words);
    ``few``     every word drawn from {100, 101, 102}: long common prefixes.

    With S > 1, consecutive segments of Geometric(1/S) length are sorted
    (lexicographically), the paper's presort."""
    raw = mt_raw(seed, n * words).astype(np.uint64).reshape(n, words) if n else np.zeros((0, words), np.uint64)
    if kind == "few":
        rec = (np.uint64(100) + raw % np.uint64(3)).astype(np.uint32)
    else:
        rec = (np.uint64(100) + raw % np.uint64(10 ** 9 - 100 + 1)).astype(np.uint32)
        if kind == "zero":
            rec[:, :-1] = 0
        elif kind != "random":
            raise ValueError(f"unknown record kind {kind!r}")
    if S > 1 and n:
        lens = geometric_lengths(n, seed + 7919, S)
        seg = np.repeat(np.arange(lens.size, dtype=np.int64), lens)
        order = np.lexsort(tuple(rec[:, w] for w in range(words - 1, -1, -1)) + (seg,))
        rec = rec[order]
    return np.ascontiguousarray(rec)


def batch_lengths(count: int, seed: int, lo_log2: float = 8.0, hi_log2: float = 20.0) -> np.ndarray:
    """Instance lengths floor(2**(lo + (hi-lo) u)), u uniform (log-uniform sizes)."""
    u = _unit_doubles(seed, count)
    return np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)


def batch(count: int, seed: int, dist: str = "uniform", lo_log2: float = 8.0,
          hi_log2: float = 20.0):
    """(keys, offsets) of ``count`` independent instances concatenated."""
    lens = batch_lengths(count, seed, lo_log2, hi_log2)
    offsets = np.zeros(count + 1, np.uint64)
    offsets[1:] = np.cumsum(lens).astype(np.uint64)
    total = int(offsets[-1])
    if dist == "uniform":
        keys = mt_raw(seed + 1, total)
    else:
        parts = [make(dist, int(ln), seed + 1 + i) for i, ln in enumerate(lens.tolist())]
        keys = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
    return keys, offsets


def poisson_requests(rate: float, duration: float, seed: int, lo_log2: float = 10.0,
                     hi_log2: float = 24.0):
    """Arrival times (s) of a Poisson stream and log-uniform request sizes."""
    expect = int(rate * duration * 1.3) + 64
    u = _unit_doubles(seed, expect)
    gaps = -np.log1p(-u) / rate
    t = np.cumsum(gaps)
    t = t[t < duration]
    sizes = batch_lengths(t.size, seed + 1, lo_log2, hi_log2)
    return t, sizes
