"""64-bit keys on the GPU (ps_sort_keys64: unsigned, int64, IEEE 754 binary64
totalOrder) vs the oracle's 64-bit keys: sorted keys, permutation, runs,
powers, merge tree and merge cost, bit-exact."""
import numpy as np
import pytest

from conftest import golden_rows
from gpu_util import to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

KT = {"u64": 0, "i64": 1, "f64": 2}


@pytest.fixture(scope="module")
def kctx():
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 21, want_perm=True, flags=binding.PS_FLAG_RECORDS) as c:
        yield c


def gen(kind, dist, n, seed):
    hi = inputs.make(dist, n, seed).astype(np.uint64)
    lo = inputs.make("uniform", n, seed + 1).astype(np.uint64)
    bits = (hi << np.uint64(32)) | lo
    if kind == "i64" and dist == "few":
        # small magnitudes of both signs: every high word is 0 or all ones
        bits = (lo.astype(np.int64) - (1 << 31)).view(np.uint64)
    return bits


def gpu64(ctx, bits, kind):
    d = torch.from_numpy(bits.view(np.int64)).cuda()
    perm = torch.empty(max(bits.size, 1), dtype=torch.int32, device="cuda")[:bits.size]
    st = ctx.sort_keys64(d, perm, KT[kind], stats=True)
    return d.cpu().numpy().view(np.uint64), to_host(perm), st


def check(ctx, oracle_mod, bits, kind):
    ref = oracle_mod.powersort_keys64(bits, kind)
    k, p, st = gpu64(ctx, bits, kind)
    assert np.array_equal(p, ref.perm)
    assert np.array_equal(k, ref.keys)
    if bits.size:
        assert np.array_equal(ctx.runs(), ref.run_starts)
        assert np.array_equal(ctx.powers(), ref.powers)
        assert st["merge_cost"] == ref.stats["merge_cost"]
    return st


@pytest.mark.parametrize("kind", ["u64", "i64", "f64"])
@pytest.mark.parametrize("dist", ["uniform", "runs", "few", "sorted", "reversed"])
def test_keys64_edge_sizes(kctx, oracle_mod, kind, dist):
    for n in (1, 2, 63, 64, 65, 1000, 4097, 70001, 300007):
        check(kctx, oracle_mod, gen(kind, dist, n, 7 + n), kind)


def test_keys64_small_ints_big_groups(kctx, oracle_mod):
    # int64 values within +-2^31: two groups of equal high words of ~n/2,
    # sorted by the grid-wide merge passes of the fix-up
    check(kctx, oracle_mod, gen("i64", "few", (1 << 21) - 3, 5), "i64")


def test_f64_special_values(kctx, oracle_mod):
    rows = golden_rows("f64_total_order.txt")
    bits = np.zeros(len(rows), np.uint64)
    for rank, idx, b in rows:
        bits[int(idx)] = int(b, 16)
    k, p, st = gpu64(kctx, bits, "f64")
    assert p.tolist() == [int(idx) for rank, idx, b in rows]
    rng = np.random.RandomState(3)
    pool = bits.copy()
    mixed = rng.randint(0, 2 ** 63, size=200003, dtype=np.int64).view(np.uint64) * np.uint64(3)
    pick = rng.rand(mixed.size) < 0.3
    mixed[pick] = pool[rng.randint(0, pool.size, size=int(pick.sum()))]
    check(kctx, oracle_mod, mixed, "f64")


def test_keys64_2_21(kctx, oracle_mod):
    for kind in ("u64", "f64"):
        check(kctx, oracle_mod, gen(kind, "uniform", 1 << 21, 11), kind)


def test_keys64_with_vm_storage(oracle_mod):
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 20, mode=binding.PS_MODE_VM, page_log2=9, want_perm=True,
                         flags=binding.PS_FLAG_RECORDS) as c:
        for kind in ("u64", "i64"):
            check(c, oracle_mod, gen(kind, "few" if kind == "i64" else "runs", 500009, 3), kind)
