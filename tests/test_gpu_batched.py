"""Batched sorting (ps_run_batched and its captured CUDA graph) vs the oracle
and vs the single-instance entry point, through the C ABI."""
import numpy as np
import pytest

from gpu_util import to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _batch(sizes, dists, seed):
    parts = [inputs.make(dists[i % len(dists)], int(n), seed + i) for i, n in enumerate(sizes)]
    keys = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(sizes, dtype=np.uint64))
    return keys, off, parts


def _dev_offsets(off):
    return torch.from_numpy(off.astype(np.int64)).cuda()


SIZES = [0, 1, 2, 31, 63, 64, 65, 100, 1000, 4095, 4096, 4097, 5000, 8193, 12345, 65536, 70001, 1 << 18, 3, 0]
DISTS = ["uniform", "zipf", "runs", "paper", "few", "sorted", "reversed", "equal"]


@pytest.fixture(scope="module")
def bctx():
    from paper_2605_27147_gb300 import binding

    stream = torch.cuda.Stream()
    with binding.Context(1 << 20, want_perm=True, max_total=1 << 22, max_count=512, stream=stream) as c:
        yield c


def test_batched_matches_oracle_per_instance(bctx, oracle_mod):
    keys, off, parts = _batch(SIZES, DISTS, 100)
    dk, dp = to_dev(keys), torch.empty(max(1, keys.size), dtype=torch.int32, device="cuda")
    st = bctx.run_batched(dk, _dev_offsets(off), dp, stats=True)
    assert st["instances"] == len(SIZES) and st["n"] == keys.size
    gk, gp = to_host(dk), to_host(dp)
    total_M = 0
    for q, part in enumerate(parts):
        a, b = int(off[q]), int(off[q + 1])
        ref = oracle_mod.powersort(part)
        assert np.array_equal(gk[a:b], ref.keys), q
        assert np.array_equal(gp[a:b], ref.perm), q
        assert np.array_equal(bctx.runs(q), ref.run_starts), q
        assert np.array_equal(bctx.powers(q), ref.powers), q
        ist = bctx.instance_stats(q)
        assert ist["merge_cost"] == ref.stats["merge_cost"] and ist["runs"] == ref.stats["runs"]
        total_M += ref.stats["merge_cost"]
    assert st["merge_cost"] == total_M


def test_batched_equals_single_instance_calls(bctx):
    rng = np.random.RandomState(7)
    # (the context holds at most 2^22 elements per batched call)
    sizes = np.floor(2.0 ** (8 + 8 * rng.rand(200))).astype(np.int64)   # about 2.4M elements
    keys, off, parts = _batch(sizes, ["uniform", "runs", "zipf"], 5)
    dk, dp = to_dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
    bctx.run_batched(dk, _dev_offsets(off), dp)
    bctx.sync()
    gk, gp = to_host(dk), to_host(dp)
    for q in range(0, len(parts), 7):
        a, b = int(off[q]), int(off[q + 1])
        sk, sp = to_dev(parts[q]), torch.empty(b - a, dtype=torch.int32, device="cuda")
        bctx.run(sk, sp)
        bctx.sync()                 # the context works on its own stream
        assert np.array_equal(to_host(sk), gk[a:b]) and np.array_equal(to_host(sp), gp[a:b])


def test_batched_bad_offsets_rejected_on_device(bctx):
    from paper_2605_27147_gb300 import binding

    keys = inputs.uniform(1000, 1)
    dk, dp = to_dev(keys), torch.empty(1000, dtype=torch.int32, device="cuda")
    for bad in ([0, 600, 500, 1000], [5, 600, 1000], [0, 1 << 21, 1 << 22]):
        with pytest.raises(binding.PowersortError) as e:
            bctx.run_batched(dk, _dev_offsets(np.array(bad, np.uint64)), dp, stats=True)
        assert e.value.status == binding.PS_EINVAL
    # the context stays usable
    off = np.array([0, 400, 1000], np.uint64)
    bctx.run_batched(dk, _dev_offsets(off), dp, stats=True)
    assert np.array_equal(to_host(dk)[:400], np.sort(keys[:400]))


def test_graph_replays_match(bctx, oracle_mod):
    rng = np.random.RandomState(11)
    sizes = np.floor(2.0 ** (6 + 10 * rng.rand(200))).astype(np.int64)   # about 1.9M elements
    keys1, off, parts1 = _batch(sizes, ["uniform", "paper"], 21)
    keys2 = np.concatenate([inputs.make("zipf", int(n), 900 + i) for i, n in enumerate(sizes)])
    dk = to_dev(keys1)
    dp = torch.empty(keys1.size, dtype=torch.int32, device="cuda")
    doff = _dev_offsets(off)
    g = bctx.graph_batched(dk, doff, dp)
    for keys in (keys1, keys2, keys1):
        dk.copy_(to_dev(keys))
        torch.cuda.synchronize()    # the refill (default stream) before the replay (context stream)
        g.launch()
        bctx.sync()
        gk, gp = to_host(dk), to_host(dp)
        for q in range(0, len(sizes), 9):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(keys[a:b])
            assert np.array_equal(gk[a:b], ref.keys) and np.array_equal(gp[a:b], ref.perm)
    g.close()


def test_config_4_full_4096(oracle_mod):
    """4096 instances of log-uniform length in [2^8, 2^20] (seed 3, about
    5.2 x 10^8 elements), sorted as the benchmark sorts them: the autotuned
    tile size and one replay of the captured batched graph.  Every instance
    by the stable-sort characterisation (vectorised over the batch), and 48
    sampled instances element by element against the oracle's Algorithm 1
    (keys, permutation, runs, powers, merge cost)."""
    from paper_2605_27147_gb300 import autotune, binding

    keys, off = inputs.batch(4096, 3)
    sizes = np.diff(off.astype(np.int64))
    total, count, max_n = int(keys.size), int(sizes.size), int(sizes.max())
    stream = torch.cuda.Stream()
    dk = to_dev(keys)
    dp = torch.empty(total, dtype=torch.int32, device="cuda")
    doff = _dev_offsets(off)
    tuned = autotune.tune(dk, doff, dp, max_n, stream=stream)
    with binding.Context(max_n, want_perm=True, max_total=total, max_count=count, tile_log2=tuned["tile_log2"],
                         merge_lanes=tuned["merge_lanes"], stream=stream) as c:
        g = c.graph_batched(dk, doff, dp)
        torch.cuda.synchronize()
        g.launch()
        c.sync()
        gk, gp = to_host(dk), to_host(dp)
        rng = np.random.RandomState(12)
        for q in sorted(rng.choice(count, size=48, replace=False).tolist()):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(keys[a:b])
            assert np.array_equal(gk[a:b], ref.keys) and np.array_equal(gp[a:b], ref.perm), q
            assert np.array_equal(c.runs(q), ref.run_starts) and np.array_equal(c.powers(q), ref.powers), q
            assert c.instance_stats(q)["merge_cost"] == ref.stats["merge_cost"], q
        g.close()
    del dk, dp, doff
    # every instance: a permutation of its own slice, keys non-decreasing,
    # equal keys in input order
    inst = np.repeat(np.arange(count, dtype=np.int32), sizes)
    assert np.all(gp < sizes[inst]), "a permutation entry outside its instance"
    src = off[:-1].astype(np.uint32)[inst] + gp
    seen = np.zeros(total, np.int8)
    seen[src] = 1
    assert seen.all(), "not a permutation within each instance"
    del seen
    assert np.array_equal(keys[src], gk)
    same = inst[1:] == inst[:-1]
    assert np.all(gk[1:][same] >= gk[:-1][same]), "keys not non-decreasing"
    eq = same & (gk[1:] == gk[:-1])
    assert np.all(gp[1:][eq] > gp[:-1][eq]), "equal keys out of input order"


def test_batched_many_small_instances(oracle_mod):
    from paper_2605_27147_gb300 import binding

    sizes = [1 + (i * 37) % 300 for i in range(4096)]
    keys, off, parts = _batch(sizes, ["uniform", "few"], 3)
    with binding.Context(512, want_perm=True, max_total=keys.size, max_count=4096) as c:
        dk, dp = to_dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
        st = c.run_batched(dk, _dev_offsets(off), dp, stats=True)
        gk, gp = to_host(dk), to_host(dp)
        for q in range(0, 4096, 97):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(parts[q])
            assert np.array_equal(gk[a:b], ref.keys) and np.array_equal(gp[a:b], ref.perm)
        assert st["instances"] == 4096


@pytest.mark.parametrize("lanes,ctas", [(1, 1), (4, 2), (16, 1), (2, 0)])
def test_merge_kernel_knobs_keep_the_result(oracle_mod, lanes, ctas):
    """The merge kernel's tuning knobs (search lanes per CTA, CTAs per SM)
    change its schedule only: every instance still equals the oracle."""
    from paper_2605_27147_gb300 import binding

    rng = np.random.RandomState(21)
    sizes = [int(x) for x in np.floor(2.0 ** (8 + 11 * rng.rand(120)))]
    parts = [inputs.make(("uniform", "zipf", "runs", "few")[i % 4], n, 300 + i) for i, n in enumerate(sizes)]
    keys = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    dk, doff = to_dev(keys), _dev_offsets(off)
    dp = torch.empty(keys.size, dtype=torch.int32, device="cuda")
    with binding.Context(max(sizes), want_perm=True, max_total=keys.size, max_count=len(sizes),
                         merge_lanes=lanes, merge_ctas=ctas) as c:
        st = c.run_batched(dk, doff, dp, stats=True)
        gk, gp = to_host(dk), to_host(dp)
        for q, part in enumerate(parts):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(part)
            assert np.array_equal(gk[a:b], ref.keys) and np.array_equal(gp[a:b], ref.perm), q
        assert st["global_nodes"] > 0
        c.check_guards()
