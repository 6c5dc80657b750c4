"""Plant plausible mistakes in a copy of the oracle and check a pin catches each.

Every mutation is a one-token edit of ``oracle/powersort_oracle.c`` (a flipped
tie rule, an off-by-one power, a wrong index, a dropped term, a wrong minrun
loop); the copy is compiled with gcc into a temporary directory and the pins
below -- the same kinds of check as in test_oracle.py -- must fail on it.
The shipped oracle must pass them all.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import oracle as ocore
from checks import cartesian_nodes, check_stable_sort, runs_by_rule_descending
from conftest import golden_rows
from paper_2605_27147_gb300 import inputs

SRC = os.path.join(os.path.dirname(ocore.__file__), "powersort_oracle.c")

MUTATIONS = {
    "merge ties take the right run": ("if (!key_gt(bkey[xa], key[xb]))", "if (key_gt(key[xb], bkey[xa]))"),
    "right-to-left merge ties take the left run": ("if (key_gt(bkey[xa - 1], key[xb - 1]))",
                                                   "if (!key_gt(key[xb - 1], bkey[xa - 1]))"),
    "insertion sort unstable": ("if (!key_gt(key[y - 1], v)) break;", "if (key_gt(v, key[y - 1])) break;"),
    "power off by one": ("if (hi > lo) return p;", "if (hi > lo) return p + 1;"),
    "power uses wrong index": ("(((unsigned __int128)(i + j)) << p)", "(((unsigned __int128)(i + k)) << p)"),
    "minrun loop bound": ("while (l >= 64) l = (l + 1) / 2;", "while (l > 64) l = (l + 1) / 2;"),
    "minrun rounds down": ("while (l >= 64) l = (l + 1) / 2;", "while (l >= 64) l = l / 2;"),
    "merge cost drops the left input": ("st->merge_cost += cj - ti;\n            ci = ti;\n            --top;                                     /* Pop */",
                                        "st->merge_cost += cj - ci;\n            ci = ti;\n            --top;                                     /* Pop */"),
    "runs strictly increasing": ("if (key_gt(key[e - 1], key[e])) break;   /* first descent: run ends here */",
                                 "if (!key_gt(key[e], key[e - 1])) break;   /* first descent: run ends here */"),
    "forced run one short": ("uint64_t end = s + minrun < n ? s + minrun : n;",
                             "uint64_t end = s + minrun - 1 < n ? s + minrun - 1 : n;"),
    "decreasing runs take equal keys": ("if (!key_gt(key[e - 1], key[e])) break;",
                                        "if (key_gt(key[e], key[e - 1])) break;"),
    "decreasing run starts on a tie": ("down = key_gt(key[s], key[e]);", "down = !key_gt(key[e], key[s]);"),
    "reversal leaves the permutation": ("key[x] = key[y]; perm[x] = perm[y];", "key[x] = key[y];"),
    "paged decreasing runs take equal keys": (
        "const int desc = key_gt(*vm_kslot(m, work, e - 1), *vm_kslot(m, work, e));",
        "const int desc = !key_gt(*vm_kslot(m, work, e), *vm_kslot(m, work, e - 1));"),
    "paged reversal off by one": ("for (uint64_t x = 0, y = e - 1; x < y; ++x, --y) {",
                                  "for (uint64_t x = 0, y = e - 2; x < y; ++x, --y) {"),
    "signed keys compared unsigned": ("if (g_key_order & ORACLE_KEY_I32) return (int32_t)a > (int32_t)b;",
                                      "if (g_key_order & ORACLE_KEY_I32) return a > b;"),
    "negative floats not reversed": ("return na ? ma < mb : ma > mb;", "return ma > mb;"),
    "float signs in the wrong order": ("if (na != nb) return nb;", "if (na != nb) return na;"),
    "int64 keys compared unsigned": ("if (g_key_order & ORACLE_KEY_I32) return (int64_t)x > (int64_t)y;",
                                     "if (g_key_order & ORACLE_KEY_I32) return x > y;"),
    "negative doubles not reversed": ("return nx ? mx < my : mx > my;", "return mx > my;"),
    "records skip their first word": ("for (uint32_t w = 0; w < g_rec_words; ++w)",
                                      "for (uint32_t w = 1; w < g_rec_words; ++w)"),
    "records compare the wrong way": ("if (ra[w] != rb[w]) return ra[w] > rb[w];",
                                      "if (ra[w] != rb[w]) return ra[w] < rb[w];"),
    "stable rank counts the element itself": ("(j < i && !key_gt(keys[j], keys[i]))",
                                              "(j <= i && !key_gt(keys[j], keys[i]))"),
    "stable rank drops the equal keys before it": (
        "r += key_gt(keys[i], keys[j]) || (j < i && !key_gt(keys[j], keys[i]));",
        "r += key_gt(keys[i], keys[j]);"),
}


def run_pins(lib):
    """Raise AssertionError if the library fails any pin."""
    for n, i, j, k, p in golden_rows("power_worked_example.txt"):
        assert oracle.power(int(n), int(i), int(j), int(k), lib=lib) == int(p)
    for n, m in golden_rows("minrun_rule.txt"):
        assert oracle.minrun(int(n), lib=lib) == int(m)
    # closed form: 2^16 uniform keys -> 2048 runs of 32, M = 11 * 2^16
    r = oracle.powersort(inputs.uniform(1 << 16, 0), lib=lib)
    assert r.stats["runs"] == 2048 and r.stats["merge_cost"] == 11 << 16
    for dist, n in [("few", 5000), ("uniform", 3001), ("runs", 20000), ("zipf", 4099), ("equal", 3000)]:
        keys = inputs.make(dist, n, n)
        r = oracle.powersort(keys, lib=lib)
        check_stable_sort(keys, r.keys, r.perm)
        assert np.array_equal(r.perm, np.argsort(keys, kind="stable"))
        # runs from the rule, by a plain scan
        a = [int(x) for x in keys]
        m = oracle.minrun(n, lib=lib)
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
        assert r.run_starts.tolist() == starts
        got = {int(mid): (int(lo), int(hi)) for lo, mid, hi in r.merges.tolist()}
        nodes = cartesian_nodes(r.run_starts, r.powers)
        assert got == nodes
        assert r.stats["merge_cost"] == sum(h - l for l, h in nodes.values())
    # the decreasing-run variant (Sec. 5), both storages: a strictly
    # decreasing array is one reversed run; results and runs by the rule
    dec = np.arange(3000, 0, -1, dtype=np.uint32)
    d = oracle.powersort(dec, lib=lib, descending_runs=True)
    assert d.stats["runs"] == 1 and np.array_equal(d.perm, np.arange(2999, -1, -1))
    for dist, n in [("updown", 20000), ("few", 3000), ("reversed", 1000)]:
        keys = inputs.make(dist, n, n)
        starts = runs_by_rule_descending(keys, oracle.minrun(n, lib=lib))
        for vm in (False, True):
            if vm:
                r = oracle.powersort_vm(keys, 32, lib=lib, descending_runs=True)
            else:
                r = oracle.powersort(keys, lib=lib, descending_runs=True)
            assert np.array_equal(r.perm, np.argsort(keys, kind="stable"))
            assert np.array_equal(r.keys, keys[r.perm])
            assert r.run_starts.tolist() == starts
    # typed key orders: numpy's stable argsort on int32 / float32 views, and
    # the hand-worked totalOrder fixture
    ik = (inputs.make("runs", 20000, 3).astype(np.int64) - (1 << 31)).astype(np.int32)
    r = oracle.powersort(ik.view(np.uint32), lib=lib, key_type="i32")
    assert np.array_equal(r.perm, np.argsort(ik, kind="stable"))
    fk = (ik.astype(np.float32) * np.float32(1e-3))
    r = oracle.powersort(fk.view(np.uint32), lib=lib, key_type="f32")
    assert np.array_equal(r.perm, np.argsort(fk, kind="stable"))
    rows = golden_rows("f32_total_order.txt")
    bits = np.zeros(len(rows), np.uint32)
    for rank, idx, b in rows:
        bits[int(idx)] = int(b, 16)
    r = oracle.powersort(bits, lib=lib, key_type="f32")
    assert r.perm.tolist() == [int(idx) for rank, idx, b in rows]
    # 64-bit keys: numpy's stable argsort
    k64 = (ik.astype(np.int64) << np.int64(20)) - np.int64(12345)
    r = oracle.powersort_keys64(k64.view(np.uint64), "i64", lib=lib)
    assert np.array_equal(r.perm, np.argsort(k64, kind="stable"))
    f64 = k64.astype(np.float64) * 1e-7
    r = oracle.powersort_keys64(f64.view(np.uint64), "f64", lib=lib)
    assert np.array_equal(r.perm, np.argsort(f64, kind="stable"))
    # one output at a time: stable positions are the inverse of numpy's
    # stable argsort
    sk = inputs.make("few", 300, 7)
    inv = np.empty(sk.size, np.int64)
    inv[np.argsort(sk, kind="stable")] = np.arange(sk.size)
    assert [oracle.stable_rank(sk, i, lib=lib) for i in range(sk.size)] == inv.tolist()
    # records: numpy's stable lexsort
    rec = inputs.records("few", 3000, 2, words=5)
    r = oracle.powersort_records(rec, lib=lib)
    assert np.array_equal(r.perm, np.lexsort(tuple(rec[:, w] for w in range(4, -1, -1))))


def test_shipped_oracle_passes_pins(oracle_mod):
    run_pins(None)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor missing: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mut.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = ocore.compile_source(path, os.path.join(d, "libmut.so"))
        lib = ocore.open_library(so)
        with pytest.raises(AssertionError):
            run_pins(lib)
