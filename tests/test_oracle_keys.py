"""Pins of the oracle's typed key orders (the key-value generalisation):
32-bit keys read as two's-complement integers or as IEEE 754 binary32
values under totalOrder.

The checks come from outside the oracle's code: numpy's stable argsort on
int32 / float32 views (which agree with totalOrder when no NaN and no
signed zero pair is present), a hand-worked totalOrder fixture with every
special value (tests/golden/f32_total_order.txt), closed forms of inputs
sorted under the typed order (one run, M = 0, while the unsigned reading of
the same bits has more runs), and the run rule restated as a plain scan over
Python numbers.
"""
import numpy as np
import pytest

from checks import cartesian_nodes
from conftest import golden_rows
from paper_2605_27147_gb300 import inputs


def _runs_by_rule(vals, m):
    """Run starts of Sec. 5's rule over comparable Python values."""
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


def signed_keys(n, seed):
    k = inputs.make("runs", n, seed).view(np.int32).copy()
    k[:: max(1, n // 7)] = np.int32(-2 ** 31)
    k[1:: max(1, n // 5)] = np.int32(2 ** 31 - 1)
    return k


def float_keys(n, seed):
    u = inputs.make("runs", n, seed).astype(np.float64)
    return ((u - 2.0 ** 31) * 1.7e-3).astype(np.float32)   # both signs, no -0


def test_total_order_golden(oracle_mod):
    rows = golden_rows("f32_total_order.txt")
    bits = np.zeros(len(rows), np.uint32)
    for rank, idx, b in rows:
        bits[int(idx)] = int(b, 16)
    want = [int(idx) for rank, idx, b in rows]
    ko, po = oracle_mod.stable_sort(bits, key_type="f32")
    assert po.tolist() == want
    r = oracle_mod.powersort(bits, key_type="f32")
    assert r.perm.tolist() == want and np.array_equal(r.keys, bits[want])
    # the same bits read as unsigned integers order differently
    assert oracle_mod.stable_sort(bits)[1].tolist() != want


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 20011])
def test_i32_matches_numpy_and_rule(oracle_mod, n):
    k = signed_keys(n, n)
    bits = k.view(np.uint32)
    ref = np.argsort(k, kind="stable")
    for fn in (lambda: oracle_mod.powersort(bits, key_type="i32"),
               lambda: oracle_mod.powersort_vm(bits, 64, key_type="i32")):
        r = fn()
        assert np.array_equal(r.perm, ref)
        assert np.array_equal(r.keys.view(np.int32), k[ref])
        assert r.run_starts.tolist() == _runs_by_rule([int(x) for x in k], oracle_mod.minrun(n))
        nodes = cartesian_nodes(r.run_starts, r.powers)
        assert {int(mid): (int(lo), int(hi)) for lo, mid, hi in r.merges.tolist()} == nodes
    assert np.array_equal(oracle_mod.stable_sort(bits, key_type="i32")[1], ref)


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 20011])
def test_f32_matches_numpy_and_rule(oracle_mod, n):
    k = float_keys(n, n + 3)
    bits = k.view(np.uint32)
    ref = np.argsort(k, kind="stable")
    r = oracle_mod.powersort(bits, key_type="f32")
    assert np.array_equal(r.perm, ref)
    assert r.run_starts.tolist() == _runs_by_rule([float(x) for x in k], oracle_mod.minrun(n))
    d = oracle_mod.powersort(bits, key_type="f32", descending_runs=True)
    assert np.array_equal(d.perm, ref)
    assert np.array_equal(oracle_mod.stable_sort(bits, key_type="f32")[1], ref)


def test_typed_sorted_input_is_one_run(oracle_mod):
    n = 5000
    ints = np.arange(-2500, 2500, dtype=np.int32) * np.int32(7)
    floats = np.linspace(-3.5e6, 2.5e6, n).astype(np.float32)
    for vals, kt in ((ints, "i32"), (floats, "f32")):
        bits = vals.view(np.uint32)
        r = oracle_mod.powersort(bits, key_type=kt)
        assert r.stats["runs"] == 1 and r.stats["merge_cost"] == 0
        assert np.array_equal(r.perm, np.arange(n))
        # read as unsigned, the negative half sorts after the positive one
        assert oracle_mod.powersort(bits).stats["runs"] > 1
    # a strictly decreasing float array is one reversed run with the variant
    dec = floats[::-1].copy().view(np.uint32)
    r = oracle_mod.powersort(dec, key_type="f32", descending_runs=True)
    assert r.stats["runs"] == 1 and np.array_equal(r.perm, np.arange(n - 1, -1, -1))


def test_typed_results_are_stable(oracle_mod):
    # many equal values, both orders
    k = (inputs.make("few", 30000, 5).astype(np.int64) - 2).astype(np.int32)
    r = oracle_mod.powersort(k.view(np.uint32), key_type="i32")
    assert np.array_equal(r.perm, np.argsort(k, kind="stable"))
    f = k.astype(np.float32) * np.float32(0.5)
    r = oracle_mod.powersort(f.view(np.uint32), key_type="f32")
    assert np.array_equal(r.perm, np.argsort(f, kind="stable"))
    assert np.all(np.diff(r.keys.view(np.float32)) >= 0)
