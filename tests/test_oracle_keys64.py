"""Pins of the oracle's 64-bit keys (unsigned, int64, IEEE 754 binary64
totalOrder): numpy's stable argsort on uint64 / int64 / float64 views, a
hand-worked binary64 totalOrder fixture, the run rule as a plain scan over
Python numbers, and a reduction to the pinned 32-bit oracle (64-bit keys
whose high words are all zero sort, schedule included, as their low words).
"""
import numpy as np
import pytest

from checks import cartesian_nodes
from conftest import golden_rows
from paper_2605_27147_gb300 import inputs


def _runs_by_rule(vals, m):
    a = list(vals)
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


def keys64(kind, n, seed):
    hi = inputs.make("runs", n, seed).astype(np.uint64)
    lo = inputs.make("few", n, seed + 1).astype(np.uint64)
    bits = (hi << np.uint64(32)) | lo
    if kind == "f64":
        # finite doubles of both signs (no NaN, no signed-zero pair)
        v = (hi.astype(np.float64) - 2.0 ** 31) * 1.3e-2 + lo.astype(np.float64) * 1e-9
        return v.astype(np.float64).view(np.uint64)
    return bits


@pytest.mark.parametrize("kind,view", [("u64", np.uint64), ("i64", np.int64), ("f64", np.float64)])
@pytest.mark.parametrize("n", [1, 63, 64, 1000, 20011])
def test_keys64_match_numpy_and_rule(oracle_mod, kind, view, n):
    k = keys64(kind, n, n)
    vals = k.view(view)
    r = oracle_mod.powersort_keys64(k, kind)
    ref = np.argsort(vals, kind="stable")
    assert np.array_equal(r.perm, ref)
    assert np.array_equal(r.keys, k[ref])
    pyvals = [float(x) for x in vals] if kind == "f64" else [int(x) for x in vals]
    assert r.run_starts.tolist() == _runs_by_rule(pyvals, oracle_mod.minrun(n))
    got = {int(mid): (int(lo), int(hi)) for lo, mid, hi in r.merges.tolist()}
    assert got == cartesian_nodes(r.run_starts, r.powers)


def test_keys64_reduce_to_32_bits(oracle_mod):
    lo = inputs.make("runs", 30011, 4)
    r = oracle_mod.powersort_keys64(lo.astype(np.uint64), "u64")
    k = oracle_mod.powersort(lo)
    assert np.array_equal(r.perm, k.perm)
    assert r.run_starts.tolist() == k.run_starts.tolist()
    assert r.merges.tolist() == k.merges.tolist()
    assert r.stats["merge_cost"] == k.stats["merge_cost"]


def test_f64_total_order_golden(oracle_mod):
    rows = golden_rows("f64_total_order.txt")
    bits = np.zeros(len(rows), np.uint64)
    for rank, idx, b in rows:
        bits[int(idx)] = int(b, 16)
    r = oracle_mod.powersort_keys64(bits, "f64")
    assert r.perm.tolist() == [int(idx) for rank, idx, b in rows]
