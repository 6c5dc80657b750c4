"""Helpers for the GPU tests: run the library on numpy keys, compare to the oracle."""
from __future__ import annotations

import numpy as np


def to_dev(keys: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(keys, dtype=np.uint32).view(np.int32)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def gpu_sort(ctx, keys: np.ndarray, want_perm: bool = True):
    """Sort through ps_run; returns (keys, perm or None, stats)."""
    import torch

    dk = to_dev(keys)
    dp = torch.empty(keys.size, dtype=torch.int32, device="cuda") if want_perm else None
    st = ctx.run(dk, dp, stats=True)
    return to_host(dk), (to_host(dp) if dp is not None else None), st


def assert_matches_oracle(ctx, keys: np.ndarray, ref, got_keys, got_perm, stats, q: int = 0):
    """Element-by-element parity: keys, perm, runs, powers, merge tree, M."""
    assert np.array_equal(got_keys, ref.keys), _first_diff("keys", got_keys, ref.keys)
    if got_perm is not None:
        assert np.array_equal(got_perm, ref.perm), _first_diff("perm", got_perm, ref.perm)
    runs = ctx.runs(q)
    assert np.array_equal(runs, ref.run_starts), _first_diff("runs", runs, ref.run_starts)
    pw = ctx.powers(q)
    assert np.array_equal(pw, ref.powers), _first_diff("powers", pw, ref.powers)
    nodes = ctx.nodes(q)
    want = {int(m): (int(lo), int(hi)) for lo, m, hi in ref.merges.tolist()}
    got = {int(ref.run_starts[t + 1]): (int(lo), int(hi)) for t, (lo, hi) in enumerate(nodes.tolist())}
    assert got == want, "merge tree differs"
    ist = ctx.instance_stats(q)
    assert ist["merge_cost"] == ref.stats["merge_cost"]
    assert ist["runs"] == ref.stats["runs"]
    assert ist["minrun"] == ref.stats["minrun"]
    if stats is not None and q == 0 and stats.get("instances", 1) == 1:
        assert stats["merge_cost"] == ref.stats["merge_cost"]
    ctx.check_guards()   # no kernel wrote past the end of a buffer the context owns


def _first_diff(name, a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape:
        return f"{name}: shapes {a.shape} vs {b.shape}"
    idx = np.flatnonzero(a != b)
    i = int(idx[0]) if idx.size else -1
    return f"{name}: {idx.size} mismatches, first at {i}: got {a[i]} want {b[i]}"
