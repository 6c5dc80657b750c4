"""Checks that pin results without reusing the oracle's code.

* :func:`check_stable_sort` -- the O(n) characterisation of the unique stable
  sort: keys non-decreasing, perm a permutation, perm increasing inside every
  group of equal keys, keys_out[r] == keys_in[perm[r]].
* :func:`cartesian_nodes` -- the merge tree as the Cartesian tree of the
  boundary powers, found by brute force (nearest smaller power on each side).
* :func:`run_entropy` -- H of Sec. 2 from the run lengths.
* :func:`runs_by_rule_descending` -- run starts of the decreasing-run variant
  (Sec. 5) by a plain scan.
"""
from __future__ import annotations

import math

import numpy as np


def check_stable_sort(keys_in: np.ndarray, keys_out: np.ndarray, perm: np.ndarray | None) -> None:
    keys_in = np.asarray(keys_in, dtype=np.uint32)
    keys_out = np.asarray(keys_out, dtype=np.uint32)
    n = keys_in.size
    assert keys_out.size == n
    if n == 0:
        return
    assert np.all(keys_out[1:] >= keys_out[:-1]), "keys not non-decreasing"
    if perm is None:
        assert np.array_equal(np.sort(keys_in), keys_out), "keys are not a permutation of the input"
        return
    perm = np.asarray(perm, dtype=np.int64)
    assert perm.min() >= 0 and perm.max() < n, "perm out of range"
    seen = np.zeros(n, np.int8)
    seen[perm] = 1
    assert seen.all(), "perm is not a permutation"
    assert np.array_equal(keys_in[perm], keys_out), "keys_out != keys_in[perm]"
    eq = keys_out[1:] == keys_out[:-1]
    assert np.all(perm[1:][eq] > perm[:-1][eq]), "equal keys out of input order"


def cartesian_nodes(run_starts: np.ndarray, powers: np.ndarray) -> dict:
    """{mid: (lo, hi)} for every boundary, by brute-force nearest smaller power."""
    rs = [int(x) for x in run_starts]
    pw = [int(x) for x in powers]
    R = len(rs) - 1
    out = {}
    for t in range(1, R):          # boundary t sits at rs[t], power pw[t-1]
        p = pw[t - 1]
        # Algorithm 1 merges a stack entry whose power is >= the new one, so an
        # equal power on the left ends up below t, an equal one on the right above.
        a = t - 1
        while a >= 1 and pw[a - 1] >= p:
            a -= 1
        # a == 0, or boundary a has power < p
        b = t + 1
        while b <= R - 1 and pw[b - 1] > p:
            b += 1
        out[rs[t]] = (rs[a] if a >= 1 else 0, rs[b] if b <= R - 1 else rs[R])
    return out


def run_entropy(run_starts: np.ndarray) -> float:
    rs = np.asarray(run_starts, dtype=np.float64)
    n = rs[-1]
    lens = np.diff(rs)
    return float(sum((l / n) * math.log2(n / l) for l in lens if l > 0))


def naive_stable_insertion_sort(keys):
    """Textbook stable insertion sort on (key, index) pairs, pure Python."""
    a = [(int(k), i) for i, k in enumerate(keys)]
    for x in range(1, len(a)):
        v = a[x]
        y = x
        while y > 0 and a[y - 1][0] > v[0]:
            a[y] = a[y - 1]
            y -= 1
        a[y] = v
    return np.array([k for k, _ in a], np.uint32), np.array([i for _, i in a], np.uint32)


def runs_by_rule_descending(keys, m):
    """Run starts by a plain scan of the decreasing-run variant's rule: a run
    whose first pair is strictly decreasing continues while strictly
    decreasing and is reversed; otherwise it continues while non-decreasing;
    a run shorter than m is extended to m elements (or the end) and sorted."""
    a = [int(x) for x in keys]
    n = len(a)
    starts, s = [0], 0
    while s < n:
        e = s + 1
        if e < n and a[s] > a[e]:
            while e < n and a[e - 1] > a[e]:
                e += 1
            a[s:e] = a[s:e][::-1]
        else:
            while e < n and a[e - 1] <= a[e]:
                e += 1
        if e - s < m:
            e = min(s + m, n)
            a[s:e] = sorted(a[s:e])
        s = e
        starts.append(s)
    return starts
