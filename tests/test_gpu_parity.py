"""GPU path vs the CPU oracle, through the C ABI (bit-exact: keys, stable
permutation, run starts, powers, merge tree, merge cost)."""
import numpy as np
import pytest

from checks import check_stable_sort
from gpu_util import assert_matches_oracle, gpu_sort, to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 24, want_perm=True) as c:
        yield c


def test_config_1_uniform_2_16(ctx, oracle_mod):
    keys = inputs.uniform(1 << 16, 0)
    ref = oracle_mod.powersort(keys)
    k, p, st = gpu_sort(ctx, keys)
    assert_matches_oracle(ctx, keys, ref, k, p, st)
    assert st["merge_cost"] == 11 << 16 and st["runs"] == 2048


EDGE = [0, 1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 1000, 4095, 4096, 4097, 8191, 8193,
        12345, 65535, 65537, 100003, 262147]
DISTS = ["uniform", "zipf", "runs", "paper", "sorted", "reversed", "equal", "few", "bands"]


@pytest.mark.parametrize("dist", DISTS)
def test_edge_sizes(ctx, oracle_mod, dist):
    for n in EDGE:
        keys = inputs.make(dist, n, 31 + n)
        ref = oracle_mod.powersort(keys)
        k, p, st = gpu_sort(ctx, keys)
        if n == 0:
            assert k.size == 0
            continue
        assert_matches_oracle(ctx, keys, ref, k, p, st)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs"])
def test_config_2_full_2_24(ctx, oracle_mod, dist):
    n = 1 << 24
    keys = inputs.make(dist, n, 1)
    ref = oracle_mod.powersort(keys)
    k, p, st = gpu_sort(ctx, keys)
    assert_matches_oracle(ctx, keys, ref, k, p, st)


def test_keys_only(ctx, oracle_mod):
    for n in (5000, 1 << 20):
        keys = inputs.make("few", n, 3)
        ref = oracle_mod.powersort(keys)
        k, p, st = gpu_sort(ctx, keys, want_perm=False)
        assert p is None
        assert np.array_equal(k, ref.keys)
        assert st["merge_cost"] == ref.stats["merge_cost"]


def test_repeated_calls_same_result(ctx, oracle_mod):
    keys = inputs.make("paper", 300007, 9)
    ref = oracle_mod.powersort(keys)
    for _ in range(3):
        k, p, st = gpu_sort(ctx, keys)
        assert np.array_equal(k, ref.keys) and np.array_equal(p, ref.perm)


def test_adversarial_run_lengths(ctx, oracle_mod):
    # long natural runs of varied lengths (unbalanced trees, runs longer than a
    # tile and than a run-detection chunk, runs just under / over minrun)
    rng = np.random.RandomState(5)
    for trial in range(6):
        lens = rng.choice([1, 5, 31, 32, 33, 100, 4095, 4097, 9000, 70000], size=40)
        keys = inputs.presort_segments(inputs.uniform(int(lens.sum()), trial), lens)
        ref = oracle_mod.powersort(keys)
        k, p, st = gpu_sort(ctx, keys)
        assert_matches_oracle(ctx, keys, ref, k, p, st)


def test_result_is_stable_sort_large(oracle_mod):
    # full-size property check at 2^26 (the oracle-free characterisation)
    from paper_2605_27147_gb300 import binding

    n = 1 << 26
    keys = inputs.make("few", n, 4)
    with binding.Context(n, want_perm=True) as c:
        dk = to_dev(keys)
        dp = torch.empty(n, dtype=torch.int32, device="cuda")
        st = c.run(dk, dp, stats=True)
        check_stable_sort(keys, to_host(dk), to_host(dp))
        assert st["n"] == n


@pytest.mark.parametrize("storage", ["pingpong", "vm"])
def test_config_3_full_2_28(oracle_mod, storage):
    """n = 2^28 uniform (seed 2), one call with keys and permutation as the
    benchmark makes it: every output by the O(n) stable-sort
    characterisation; the run starts, powers and merge cost by their closed
    forms (2^23 forced runs of minrun = 32 make a perfectly balanced tree:
    p_t = 23 - v2(t), M = 23 n); sampled outputs ranked one by one by the
    oracle's definition."""
    from paper_2605_27147_gb300 import binding

    n = 1 << 28
    keys = inputs.make("uniform", n, 2)
    kw = {"mode": binding.PS_MODE_VM} if storage == "vm" else {}
    with binding.Context(n, want_perm=True, **kw) as c:
        dk = to_dev(keys)
        dp = torch.empty(n, dtype=torch.int32, device="cuda")
        st = c.run(dk, dp, stats=True)
        runs, pw = c.runs(), c.powers()
        gk, gp = to_host(dk), to_host(dp)
        del dk, dp
    # no natural run of these keys reaches 32 elements: every run is forced
    assert st["runs"] == n // 32
    assert np.array_equal(runs.astype(np.int64), np.arange(0, n + 1, 32, dtype=np.int64))
    t = np.arange(1, n // 32, dtype=np.int64)
    assert np.array_equal(pw.astype(np.int64), 23 - np.log2(t & -t).astype(np.int64))
    assert st["merge_cost"] == 23 * n
    check_stable_sort(keys, gk, gp)
    rng = np.random.RandomState(6)
    for r in rng.randint(0, n, size=6).tolist() + [0, n - 1]:
        assert oracle_mod.stable_rank(keys, int(gp[r])) == r


@pytest.mark.parametrize("tile_log2", [10, 11])
def test_smaller_tiles(oracle_mod, tile_log2):
    # smaller on-chip tiles leave more of the tree to the HBM merge kernel
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 22, want_perm=True, tile_log2=tile_log2) as c:
        for dist, n in (("uniform", 3000017), ("runs", (1 << 22) - 5), ("few", 1234567)):
            keys = inputs.make(dist, n, 17 + tile_log2)
            ref = oracle_mod.powersort(keys)
            k, p, st = gpu_sort(c, keys)
            assert_matches_oracle(c, keys, ref, k, p, st)


def test_unaligned_caller_arrays(ctx, oracle_mod):
    # arrays starting 4, 8 and 12 bytes past a 16-byte boundary
    for shift in (1, 2, 3):
        n = 300007 + shift
        keys = inputs.make("runs", n, 40 + shift)
        ref = oracle_mod.powersort(keys)
        kbuf = torch.empty(n + 4, dtype=torch.int32, device="cuda")
        pbuf = torch.empty(n + 4, dtype=torch.int32, device="cuda")
        dk, dp = kbuf[shift:shift + n], pbuf[shift:shift + n]
        dk.copy_(torch.from_numpy(keys.view(np.int32)))
        st = ctx.run(dk, dp, stats=True)
        assert np.array_equal(to_host(dk), ref.keys)
        assert np.array_equal(to_host(dp), ref.perm)
        assert st["merge_cost"] == ref.stats["merge_cost"]


def test_host_arrays(oracle_mod):
    # ps_run_host: pinned host arrays in and out, copies inside the call
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 20, want_perm=True, flags=binding.PS_FLAG_HOST_IO) as c:
        for n in (1, 2, 3, 4097, 300007, 1 << 20):
            keys = inputs.make("runs", n, 70 + n)
            ref = oracle_mod.powersort(keys)
            hk = torch.from_numpy(keys.view(np.int32).copy()).pin_memory()
            hp = torch.empty(n, dtype=torch.int32).pin_memory()
            st = c.run_host(hk.data_ptr(), n, hp.data_ptr(), stats=True)
            assert np.array_equal(hk.numpy().view(np.uint32), ref.keys)
            assert np.array_equal(hp.numpy().view(np.uint32), ref.perm)
            assert st["merge_cost"] == ref.stats["merge_cost"]
            hk2 = torch.from_numpy(keys.view(np.int32).copy()).pin_memory()
            c.run_host(hk2.data_ptr(), n, None)              # keys only
            assert np.array_equal(hk2.numpy().view(np.uint32), ref.keys)
        c.check_guards()
