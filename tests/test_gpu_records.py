"""Records (rows of 32-bit words ordered lexicographically, the paper's blob
types) on the GPU vs the oracle, through the C ABI (ps_sort_records):
permutation, rows, runs, powers, merge tree and merge cost, bit-exact."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _ctx(max_n, **kw):
    from paper_2605_27147_gb300 import binding

    return binding.Context(max_n, want_perm=True, flags=binding.PS_FLAG_RECORDS, **kw)


@pytest.fixture(scope="module")
def rctx():
    with _ctx(1 << 20) as c:
        yield c


def gpu_records(ctx, rec):
    n = rec.shape[0]
    d = torch.from_numpy(np.ascontiguousarray(rec).view(np.int32)).cuda()
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")[:n]
    out = torch.empty_like(d)
    st = ctx.sort_records(d, perm, out, stats=True)
    assert torch.equal(d.cpu(), torch.from_numpy(np.ascontiguousarray(rec).view(np.int32)))   # input untouched
    return to_host(perm), out.cpu().numpy().view(np.uint32), st


def check(ctx, oracle_mod, rec):
    ref = oracle_mod.powersort_records(rec)
    perm, out, st = gpu_records(ctx, rec)
    assert np.array_equal(perm, ref.perm)
    assert np.array_equal(out, rec[ref.perm])
    if rec.shape[0] == 0:
        return st
    assert np.array_equal(ctx.runs(), ref.run_starts)
    assert np.array_equal(ctx.powers(), ref.powers)
    nodes = ctx.nodes()
    want = {int(m): (int(lo), int(hi)) for lo, m, hi in ref.merges.tolist()}
    got = {int(ref.run_starts[t + 1]): (int(lo), int(hi)) for t, (lo, hi) in enumerate(nodes.tolist())}
    assert got == want
    assert st["merge_cost"] == ref.stats["merge_cost"] and st["runs"] == ref.stats["runs"]
    return st


EDGE = [1, 2, 63, 64, 65, 1000, 4097, 70001, 300007]


@pytest.mark.parametrize("kind,words", [("random", 30), ("zero", 30), ("few", 6), ("random", 1), ("few", 2)])
def test_records_edge_sizes(rctx, oracle_mod, kind, words):
    for n in EDGE:
        check(rctx, oracle_mod, inputs.records(kind, n, 3 + n, words=words))


def test_records_presorted(rctx, oracle_mod):
    for S in (64.0, 1000.0, 100000.0):
        st = check(rctx, oracle_mod, inputs.records("random", 200003, 9, S=S))
        assert st["runs"] < 200003 // 32


def test_records_large_tie_groups(rctx, oracle_mod):
    # six words from {100, 101, 102}: the window (word 0) leaves three groups of
    # about n / 3 rows, sorted by the merge passes of the fix-up
    check(rctx, oracle_mod, inputs.records("few", 100003, 4, words=6))
    # equal windows everywhere but one row: one group of n - 1 rows
    rec = inputs.records("random", 50000, 6, words=3)
    rec[:, 0] = 7
    rec[123, 0] = 8
    check(rctx, oracle_mod, rec)


def test_records_two_words_many_big_groups(rctx, oracle_mod):
    # two-word rows: the first word leaves 40 groups of 2049 .. 9000 rows (the
    # nested batched sort of their last words) between groups of a few rows
    # (the shared-memory fix-up); the last word takes 5 values, so ties inside
    # a group show the nested sort's stability in the permutation
    u = inputs.uniform(300000, 17)
    sizes = [2049 + int(x) % 6952 for x in u[:40]] + [1 + int(x) % 40 for x in u[40:1040]]
    word0 = np.repeat(np.arange(len(sizes), dtype=np.uint32) * 7, sizes)
    n = word0.size
    order = np.argsort(inputs.uniform(n, 18), kind="stable")
    rec = np.stack([word0[order], inputs.uniform(n, 19) % 5], axis=1).astype(np.uint32)
    for _ in range(2):   # twice on one context: the group tables start over
        check(rctx, oracle_mod, rec)
    # then a call with no big group at all
    check(rctx, oracle_mod, inputs.records("random", 70001, 3, words=2))


def test_records_all_equal_and_sorted(rctx, oracle_mod):
    rec = np.full((5000, 4), 9, np.uint32)
    st = check(rctx, oracle_mod, rec)
    assert st["runs"] == 1 and st["merge_cost"] == 0
    srt = inputs.records("random", 5000, 2, words=4)
    srt = srt[np.lexsort(tuple(srt[:, w] for w in range(3, -1, -1)))]
    st = check(rctx, oracle_mod, srt)
    assert st["runs"] == 1


def test_records_blob30_2_20(oracle_mod):
    with _ctx(1 << 20) as c:
        for kind in ("random", "zero"):
            check(c, oracle_mod, inputs.records(kind, 1 << 20, 1))


def test_records_need_the_flag():
    from paper_2605_27147_gb300 import binding

    rec = torch.zeros((10, 3), dtype=torch.int32, device="cuda")
    perm = torch.empty(10, dtype=torch.int32, device="cuda")
    with binding.Context(1 << 10, want_perm=True) as c:
        with pytest.raises(binding.PowersortError):
            c.sort_records(rec, perm)
    with _ctx(1 << 10) as c:
        with pytest.raises(binding.PowersortError):
            c.sort_records(torch.zeros((10, 0), dtype=torch.int32, device="cuda"), perm)


def test_records_with_vm_storage(oracle_mod):
    # the window keys go through the paged merge rounds instead of Pingpong
    from paper_2605_27147_gb300 import binding

    with _ctx(1 << 20, mode=binding.PS_MODE_VM, page_log2=8) as c:
        for kind, n in (("random", 300007), ("few", 100003)):
            check(c, oracle_mod, inputs.records(kind, n, 8, words=30 if kind == "random" else 6))
