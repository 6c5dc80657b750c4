"""Pins of the oracle's records (wide elements ordered lexicographically, the
paper's blob types, Sec. 5 "Input data types").

Outside references: numpy's stable lexsort; reductions to the pinned 32-bit
oracle (records that differ only in one word sort exactly as that word, with
the same runs, powers, merges and merge cost); the run rule as a plain scan
over Python tuples; the brute-force Cartesian tree of the powers.
"""
import numpy as np
import pytest

from checks import cartesian_nodes
from paper_2605_27147_gb300 import inputs


def lex_order(rec):
    return np.lexsort(tuple(rec[:, w] for w in range(rec.shape[1] - 1, -1, -1)))


def runs_by_rule(rows, m):
    a = [tuple(int(x) for x in r) for r in rows]
    n = len(a)
    starts, s = [0], 0
    while s < n:
        e = s + 1
        while e < n and a[e - 1] <= a[e]:
            e += 1
        if e - s < m:
            e = min(s + m, n)
            a[s:e] = sorted(a[s:e])
        s = e
        starts.append(s)
    return starts


@pytest.mark.parametrize("kind", ["random", "zero", "few"])
@pytest.mark.parametrize("n", [1, 2, 63, 64, 1000, 5003])
def test_records_match_lexsort_and_rule(oracle_mod, kind, n):
    rec = inputs.records(kind, n, n + 1, words=30 if kind != "few" else 6)
    r = oracle_mod.powersort_records(rec)
    ref = lex_order(rec)
    assert np.array_equal(r.perm, ref)
    assert np.array_equal(oracle_mod.stable_sort_records(rec), ref)
    assert r.run_starts.tolist() == runs_by_rule(rec, oracle_mod.minrun(n))
    got = {int(mid): (int(lo), int(hi)) for lo, mid, hi in r.merges.tolist()}
    assert got == cartesian_nodes(r.run_starts, r.powers)


@pytest.mark.parametrize("col", [0, 29])
def test_records_reduce_to_one_word(oracle_mod, col):
    # rows equal except in one word (distinct in word 0, repeated in word 29):
    # the records sort exactly as that word does, schedule included
    n = 20000
    w = inputs.make("runs" if col == 0 else "few", n, 7)
    if col == 0:
        w = np.random.RandomState(3).permutation(n).astype(np.uint32) * np.uint32(997)
    rec = np.zeros((n, 30), np.uint32)
    rec[:, col] = w
    r = oracle_mod.powersort_records(rec)
    k = oracle_mod.powersort(w)
    assert np.array_equal(r.perm, k.perm)
    assert r.run_starts.tolist() == k.run_starts.tolist()
    assert r.powers.tolist() == k.powers.tolist()
    assert r.merges.tolist() == k.merges.tolist()
    assert r.stats["merge_cost"] == k.stats["merge_cost"]


def test_presorted_records(oracle_mod):
    rec = inputs.records("random", 30000, 5, S=500.0)
    r = oracle_mod.powersort_records(rec)
    assert np.array_equal(r.perm, lex_order(rec))
    assert r.stats["runs"] < 30000 // oracle_mod.minrun(30000)
    d = oracle_mod.powersort_records(rec[::-1].copy(), descending_runs=True)
    assert np.array_equal(d.perm, lex_order(rec[::-1]))
