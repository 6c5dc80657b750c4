"""Pins of the oracle's decreasing-run variant (Sec. 5 "Algorithm variants":
Powersort may also take strictly decreasing runs, reversing them).

The checks come from outside the oracle's code: closed forms of inputs whose
runs are known by construction (a strictly decreasing array is one run; a
zig-zag of blocks has its block starts as run starts and the balanced-tree
merge cost), the O(n) stable-sort characterisation and numpy's stable
argsort, the run rule restated as a plain scan, the brute-force Cartesian
tree of the powers, and the paper's bounds.
"""
import math

import numpy as np
import pytest

from checks import cartesian_nodes, check_stable_sort, run_entropy, runs_by_rule_descending as runs_by_rule
from paper_2605_27147_gb300 import inputs


def zigzag(K, L):
    """K blocks of L keys: even blocks L .. 2L-1 ascending, odd blocks L-1 .. 0
    descending.  Every block boundary breaks the run before it (an ascending
    block ends above the next block's first key, a descending block ends at 0),
    so with L >= minrun the runs are exactly the blocks."""
    up = np.arange(L, 2 * L, dtype=np.uint32)
    down = np.arange(L - 1, -1, -1, dtype=np.uint32)
    return np.concatenate([up if b % 2 == 0 else down for b in range(K)])


@pytest.mark.parametrize("n", [2, 3, 63, 64, 65, 1000, 1 << 16])
def test_strictly_decreasing_is_one_run(oracle_mod, n):
    keys = np.arange(n, 0, -1, dtype=np.uint32) * np.uint32(3)
    r = oracle_mod.powersort(keys, descending_runs=True)
    assert r.stats["runs"] == 1 and r.stats["merge_cost"] == 0 and r.stats["merges"] == 0
    assert r.stats["reversed_runs"] == 1 and r.stats["reverse_moves"] == 2 * (n // 2)
    assert np.array_equal(r.keys, keys[::-1]) and np.array_equal(r.perm, np.arange(n - 1, -1, -1))
    # without the variant the same input is nothing but forced runs
    a = oracle_mod.powersort(keys)
    m = oracle_mod.minrun(n)
    assert a.run_starts.tolist() == list(range(0, n, m)) + [n]
    assert a.stats["reversed_runs"] == 0
    v = oracle_mod.powersort_vm(keys, 16, descending_runs=True)
    assert v.stats["runs"] == 1 and np.array_equal(v.perm, r.perm)


@pytest.mark.parametrize("K,m", [(10, 5), (12, 6), (14, 8), (16, 10)])
def test_zigzag_closed_form(oracle_mod, K, m):
    n, L = 1 << K, 1 << m
    keys = zigzag(n // L, L)
    r = oracle_mod.powersort(keys, descending_runs=True)
    assert r.run_starts.tolist() == list(range(0, n + 1, L))
    assert r.stats["reversed_runs"] == n // L // 2
    # equal aligned runs of 2^m: a perfect tree, every level moves all n
    assert r.stats["merge_cost"] == n * (K - m)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(r.perm, ref)
    check_stable_sort(keys, r.keys, r.perm)


@pytest.mark.parametrize("dist", ["updown", "uniform", "few", "equal", "reversed", "runs", "zipf"])
def test_variant_result_and_runs(oracle_mod, dist):
    for n in (1, 2, 63, 64, 65, 1000, 5003, 20000):
        keys = inputs.make(dist, n, 11 + n)
        r = oracle_mod.powersort(keys, descending_runs=True)
        check_stable_sort(keys, r.keys, r.perm)
        assert np.array_equal(r.perm, np.argsort(keys, kind="stable"))
        m = oracle_mod.minrun(n)
        assert r.run_starts.tolist() == runs_by_rule(keys, m)
        got = {int(mid): (int(lo), int(hi)) for lo, mid, hi in r.merges.tolist()}
        nodes = cartesian_nodes(r.run_starts, r.powers)
        assert got == nodes
        assert r.stats["merge_cost"] == sum(h - l for l, h in nodes.values())
        v = oracle_mod.powersort_vm(keys, 32, descending_runs=True)
        assert v.run_starts.tolist() == r.run_starts.tolist()
        assert v.merges.tolist() == r.merges.tolist()
        assert np.array_equal(v.keys, r.keys) and np.array_equal(v.perm, r.perm)


def test_equal_keys_never_reverse(oracle_mod):
    # pairs of equal keys going down: every strictly decreasing stretch has
    # length 2 at most, so stability is never at stake
    n = 4000
    keys = np.repeat(np.arange(n // 2, 0, -1, dtype=np.uint32), 2)
    r = oracle_mod.powersort(keys, descending_runs=True)
    assert np.array_equal(r.perm, np.argsort(keys, kind="stable"))
    assert r.run_starts.tolist() == runs_by_rule(keys, oracle_mod.minrun(n))
    e = oracle_mod.powersort(np.full(n, 5, np.uint32), descending_runs=True)
    assert e.stats["runs"] == 1 and e.stats["reversed_runs"] == 0


@pytest.mark.parametrize("dist", ["updown", "uniform", "reversed"])
def test_variant_bounds(oracle_mod, dist):
    for n in (64, 1000, 30011, 1 << 16):
        keys = inputs.make(dist, n, 3 * n + 5)
        r = oracle_mod.powersort(keys, descending_runs=True)
        s = r.stats
        assert s["max_stack"] <= math.ceil(math.log2(n)) + 1
        assert s["merge_cost"] <= n * (run_entropy(r.run_starts) + 2) + 1e-6
        assert s["moves"] <= s["merge_cost"] + n
        lens = np.diff(r.run_starts.astype(np.int64))
        if lens.size > 1:
            assert lens[:-1].min() >= oracle_mod.minrun(n)
        # the variant never finds more runs than the plain rule on these inputs
        # with long decreasing stretches
        if dist != "uniform":
            assert s["runs"] <= oracle_mod.powersort(keys).stats["runs"]
