"""The decreasing-run variant (Sec. 5 "Algorithm variants") on the GPU vs the
oracle's variant, through the C ABI (PS_FLAG_DESCENDING_RUNS): keys, stable
permutation, run starts, powers, merge tree and merge cost, bit-exact."""
import numpy as np
import pytest

from checks import check_stable_sort
from gpu_util import assert_matches_oracle, gpu_sort, to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _ctx(max_n, **kw):
    from paper_2605_27147_gb300 import binding

    kw.setdefault("want_perm", True)
    return binding.Context(max_n, flags=binding.PS_FLAG_DESCENDING_RUNS, **kw)


@pytest.fixture(scope="module")
def dctx():
    with _ctx(1 << 24) as c:
        yield c


def zigzag(K, L):
    up = np.arange(L, 2 * L, dtype=np.uint32)
    down = np.arange(L - 1, -1, -1, dtype=np.uint32)
    return np.concatenate([up if b % 2 == 0 else down for b in range(K)])


def segments(rng, n, lengths):
    """Segments of the given length choices, each ascending, strictly
    descending or a plateau of equal keys, at random levels (boundaries fall
    anywhere, including chunk and tile edges)."""
    parts, tot = [], 0
    while tot < n:
        L = min(int(rng.choice(lengths)), n - tot)
        base = int(rng.randint(0, 1 << 30))
        seg = np.sort(rng.randint(base, base + 3 * L + 2, size=L)).astype(np.uint32)
        d = rng.randint(4)
        if d == 1:
            seg = np.unique(seg)[::-1].copy()
            L = seg.size
        elif d == 2:
            seg = np.full(L, base, np.uint32)
        parts.append(seg)
        tot += L
    return np.concatenate(parts)[:n]


EDGE = [1, 2, 3, 63, 64, 65, 127, 1000, 4095, 4096, 4097, 8191, 8193, 12345, 65537, 262147]


@pytest.mark.parametrize("dist", ["updown", "reversed", "uniform", "few", "runs", "equal", "sorted"])
def test_edge_sizes(dctx, oracle_mod, dist):
    for n in EDGE:
        keys = inputs.make(dist, n, 51 + n)
        ref = oracle_mod.powersort(keys, descending_runs=True)
        k, p, st = gpu_sort(dctx, keys)
        assert_matches_oracle(dctx, keys, ref, k, p, st)


@pytest.mark.parametrize("L", [32, 33, 63, 64, 65, 100, 4096, 5000, 20000])
def test_zigzag(dctx, oracle_mod, L):
    # runs exactly the blocks (L >= minrun): the reversal of every second block,
    # on chip (L <= tile) or streamed (L > tile)
    keys = zigzag(max(2, (1 << 20) // L), L)
    ref = oracle_mod.powersort(keys, descending_runs=True)
    assert ref.stats["reversed_runs"] > 0
    k, p, st = gpu_sort(dctx, keys)
    assert_matches_oracle(dctx, keys, ref, k, p, st)


def test_long_decreasing_runs_cross_chunks(dctx, oracle_mod):
    for mean in (300.0, 5000.0, 70000.0):
        keys = inputs.updown((1 << 21) + 77, 9, mean_run=mean)
        ref = oracle_mod.powersort(keys, descending_runs=True)
        k, p, st = gpu_sort(dctx, keys)
        assert_matches_oracle(dctx, keys, ref, k, p, st)


def test_strictly_decreasing_one_run(dctx, oracle_mod):
    for n in (100, 5000, (1 << 20) + 3):
        keys = np.arange(n, 0, -1, dtype=np.uint32)
        ref = oracle_mod.powersort(keys, descending_runs=True)
        k, p, st = gpu_sort(dctx, keys)
        assert st["runs"] == 1 and st["merge_cost"] == 0
        assert_matches_oracle(dctx, keys, ref, k, p, st)


def test_adversarial_segments(dctx, oracle_mod):
    rng = np.random.RandomState(11)
    lengths = [1, 2, 3, 31, 32, 33, 62, 63, 64, 65, 4095, 4096, 4097, 8191, 8193, 9000, 70000]
    for trial in range(8):
        n = int(rng.choice([5000, 100003, 1 << 20]))
        keys = segments(rng, n, lengths)
        ref = oracle_mod.powersort(keys, descending_runs=True)
        k, p, st = gpu_sort(dctx, keys)
        assert_matches_oracle(dctx, keys, ref, k, p, st)


@pytest.mark.parametrize("dist", ["updown", "uniform"])
def test_full_2_24(dctx, oracle_mod, dist):
    keys = inputs.make(dist, 1 << 24, 2)
    ref = oracle_mod.powersort(keys, descending_runs=True)
    k, p, st = gpu_sort(dctx, keys)
    assert_matches_oracle(dctx, keys, ref, k, p, st)


def test_keys_only(dctx, oracle_mod):
    for n in (70001, (1 << 20) + 5):
        keys = inputs.updown(n, 4, mean_run=9000.0)
        ref = oracle_mod.powersort(keys, descending_runs=True)
        k, p, st = gpu_sort(dctx, keys, want_perm=False)
        assert p is None and np.array_equal(k, ref.keys)
        assert st["merge_cost"] == ref.stats["merge_cost"]


def test_variant_off_is_unchanged(oracle_mod):
    # the same input without the flag follows the plain rule
    from paper_2605_27147_gb300 import binding

    keys = inputs.updown(300007, 5, mean_run=2000.0)
    with binding.Context(1 << 20, want_perm=True) as c:
        ref = oracle_mod.powersort(keys)
        k, p, st = gpu_sort(c, keys)
        assert_matches_oracle(c, keys, ref, k, p, st)
    alt = oracle_mod.powersort(keys, descending_runs=True)
    assert alt.stats["runs"] < ref.stats["runs"]


def test_vm_storage(oracle_mod):
    from paper_2605_27147_gb300 import binding

    with _ctx(1 << 21, mode=binding.PS_MODE_VM, page_log2=8) as c:
        for dist, n in (("updown", (1 << 21) - 9), ("reversed", 300007), ("uniform", 65537)):
            keys = inputs.make(dist, n, 8)
            ref = oracle_mod.powersort(keys, descending_runs=True)
            k, p, st = gpu_sort(c, keys)
            assert_matches_oracle(c, keys, ref, k, p, st)


def test_batched(oracle_mod):
    sizes = [0, 1, 2, 63, 64, 65, 1000, 4097, 5000, 65536, 70001, 1 << 18, 3]
    parts = [inputs.updown(int(n), 60 + i, mean_run=float(1 + 50 * i)) if n else np.zeros(0, np.uint32)
             for i, n in enumerate(sizes)]
    keys = np.concatenate(parts)
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(sizes, dtype=np.uint64))
    with _ctx(1 << 20, max_total=1 << 22, max_count=64) as c:
        dk, dp = to_dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
        c.run_batched(dk, torch.from_numpy(off.astype(np.int64)).cuda(), dp, stats=True)
        gk, gp = to_host(dk), to_host(dp)
        for q, part in enumerate(parts):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(part, descending_runs=True)
            assert np.array_equal(gk[a:b], ref.keys), q
            assert np.array_equal(gp[a:b], ref.perm), q
            if part.size:
                assert np.array_equal(c.runs(q), ref.run_starts), q
                assert np.array_equal(c.powers(q), ref.powers), q


def test_result_is_stable_sort_2_26():
    n = 1 << 26
    keys = inputs.updown(n, 3, mean_run=4096.0) % np.uint32(1 << 20)   # many equal keys
    with _ctx(n) as c:
        dk = to_dev(keys)
        dp = torch.empty(n, dtype=torch.int32, device="cuda")
        c.run(dk, dp)
        check_stable_sort(keys, to_host(dk), to_host(dp))
