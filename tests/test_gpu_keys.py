"""The key-value generalisation on the GPU vs the oracle, through the C ABI:
signed 32-bit and IEEE 754 binary32 keys (ps_config.key_type), bit-exact in
keys, permutation, runs, powers, merge tree and merge cost; and payload rows
of any width gathered through the permutation (ps_gather_rows)."""
import numpy as np
import pytest

from conftest import golden_rows
from gpu_util import assert_matches_oracle, gpu_sort, to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

KT = {"i32": 1, "f32": 2}


def _ctx(max_n, key_type, **kw):
    from paper_2605_27147_gb300 import binding

    return binding.Context(max_n, key_type=KT[key_type], want_perm=True, **kw)


def typed_keys(kt, dist, n, seed):
    u = inputs.make(dist, n, seed)
    if kt == "i32":
        return u.view(np.int32).copy()
    # floats of both signs and many magnitudes, some equal values
    x = (u.astype(np.float64) - 2.0 ** 31) * np.float64(2.0) ** ((u % 61).astype(np.float64) - 30.0)
    return x.astype(np.float32)


def special_floats(n, seed):
    rng = np.random.RandomState(seed)
    pool = np.array([0x00000000, 0x80000000, 0x7f800000, 0xff800000, 0x7fc00000, 0xffc00000, 0x7f800001,
                     0xff800001, 0x00000001, 0x80000001, 0x3f800000, 0xbf800000, 0x7f7fffff, 0xff7fffff],
                    dtype=np.uint32)
    bits = rng.randint(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    pick = rng.rand(n) < 0.3
    bits[pick] = pool[rng.randint(0, pool.size, size=int(pick.sum()))]
    return bits


EDGE = [1, 2, 63, 64, 65, 1000, 4097, 8193, 65537, 262147]


@pytest.mark.parametrize("kt", ["i32", "f32"])
@pytest.mark.parametrize("dist", ["uniform", "runs", "few", "sorted", "reversed"])
def test_typed_edge_sizes(oracle_mod, kt, dist):
    with _ctx(1 << 20, kt) as ctx:
        for n in EDGE:
            k = typed_keys(kt, dist, n, 5 + n).view(np.uint32)
            ref = oracle_mod.powersort(k, key_type=kt)
            gk, gp, st = gpu_sort(ctx, k)
            assert_matches_oracle(ctx, k, ref, gk, gp, st)


def test_f32_special_values(oracle_mod):
    rows = golden_rows("f32_total_order.txt")
    gold = np.zeros(len(rows), np.uint32)
    for rank, idx, b in rows:
        gold[int(idx)] = int(b, 16)
    with _ctx(1 << 20, "f32") as ctx:
        gk, gp, st = gpu_sort(ctx, gold)
        assert gp.tolist() == [int(idx) for rank, idx, b in rows]
        for n in (100, 70001, 1 << 20):
            k = special_floats(n, n)
            ref = oracle_mod.powersort(k, key_type="f32")
            gk, gp, st = gpu_sort(ctx, k)
            assert_matches_oracle(ctx, k, ref, gk, gp, st)


@pytest.mark.parametrize("kt", ["i32", "f32"])
def test_typed_full_2_24(oracle_mod, kt):
    k = typed_keys(kt, "uniform", 1 << 24, 3).view(np.uint32)
    ref = oracle_mod.powersort(k, key_type=kt)
    with _ctx(1 << 24, kt) as ctx:
        gk, gp, st = gpu_sort(ctx, k)
        assert_matches_oracle(ctx, k, ref, gk, gp, st)
        assert st["launches"] == 13


def test_typed_vm_and_descending(oracle_mod):
    from paper_2605_27147_gb300 import binding

    k = typed_keys("f32", "runs", (1 << 20) + 9, 8).view(np.uint32)
    with _ctx(1 << 21, "f32", mode=binding.PS_MODE_VM, page_log2=9) as ctx:
        ref = oracle_mod.powersort(k, key_type="f32")
        gk, gp, st = gpu_sort(ctx, k)
        assert_matches_oracle(ctx, k, ref, gk, gp, st)
    d = (-np.sort(typed_keys("f32", "uniform", 300007, 2))).astype(np.float32).view(np.uint32)
    with _ctx(1 << 20, "f32", flags=binding.PS_FLAG_DESCENDING_RUNS) as ctx:
        ref = oracle_mod.powersort(d, key_type="f32", descending_runs=True)
        gk, gp, st = gpu_sort(ctx, d)
        assert_matches_oracle(ctx, d, ref, gk, gp, st)


def test_typed_batched(oracle_mod):
    sizes = [0, 1, 64, 1000, 4097, 70001, 3]
    parts = [typed_keys("i32", "runs", n, 20 + i).view(np.uint32) for i, n in enumerate(sizes)]
    keys = np.concatenate(parts)
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(sizes, dtype=np.uint64))
    with _ctx(1 << 17, "i32", max_total=1 << 18, max_count=16) as ctx:
        dk, dp = to_dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
        ctx.run_batched(dk, torch.from_numpy(off.astype(np.int64)).cuda(), dp, stats=True)
        gk, gp = to_host(dk), to_host(dp)
        for q, part in enumerate(parts):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(part, key_type="i32")
            assert np.array_equal(gk[a:b], ref.keys) and np.array_equal(gp[a:b], ref.perm), q


@pytest.mark.parametrize("row_bytes", [1, 3, 4, 8, 12, 16, 24, 120])
def test_gather_rows(oracle_mod, row_bytes):
    n = 100003
    k = typed_keys("f32", "few", n, row_bytes).view(np.uint32)
    rng = np.random.RandomState(row_bytes)
    payload = rng.randint(0, 256, size=(n, row_bytes)).astype(np.uint8)
    ref = oracle_mod.powersort(k, key_type="f32")
    with _ctx(1 << 17, "f32") as ctx:
        gk, gp, st = gpu_sort(ctx, k)
        assert np.array_equal(gp, ref.perm)
        perm = to_dev(gp)
        for shift in (0, 1):                    # 16-byte aligned rows, then byte-shifted arrays
            sbuf = torch.zeros(n * row_bytes + 16, dtype=torch.uint8, device="cuda")
            dbuf = torch.zeros(n * row_bytes + 16, dtype=torch.uint8, device="cuda")
            src = sbuf[shift:shift + n * row_bytes].view(n, row_bytes)
            dst = dbuf[shift:shift + n * row_bytes].view(n, row_bytes)
            src.copy_(torch.from_numpy(payload))
            ctx.gather_rows(perm, src, dst)
            ctx.sync()
            assert np.array_equal(dst.cpu().numpy(), payload[ref.perm])


def test_gather_rows_batched_and_bad_perm(oracle_mod):
    from paper_2605_27147_gb300 import binding

    sizes = [5, 0, 1000, 7, 4096]
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(sizes, dtype=np.uint64))
    total = int(off[-1])
    rng = np.random.RandomState(1)
    perm = np.concatenate([rng.permutation(s).astype(np.uint32) for s in sizes])
    payload = rng.randint(0, 2 ** 31, size=(total, 6)).astype(np.int32)
    want = np.concatenate([payload[int(off[q]):int(off[q + 1])][perm[int(off[q]):int(off[q + 1])]]
                           for q in range(len(sizes))])
    with _ctx(1 << 13, "i32", max_total=1 << 14, max_count=8) as ctx:
        dperm = to_dev(perm)
        doff = torch.from_numpy(off.astype(np.int64)).cuda()
        src = torch.from_numpy(payload).cuda()
        dst = torch.zeros_like(src)
        ctx.gather_rows(dperm, src, dst, offsets=doff)
        ctx.sync()
        assert np.array_equal(dst.cpu().numpy(), want)
        # an entry outside its instance copies nothing for that row and reports
        bad = perm.copy()
        bad[2] = 5                               # instance 0 has 5 rows
        ctx.gather_rows(to_dev(bad), src, dst, offsets=doff)
        with pytest.raises(binding.PowersortError):
            ctx.sync()
        # the next sort starts clean
        k = typed_keys("i32", "uniform", 1000, 1).view(np.uint32)
        gk, gp, st = gpu_sort(ctx, k)
        assert np.array_equal(gp, oracle_mod.powersort(k, key_type="i32").perm)
