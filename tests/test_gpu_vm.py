"""Virtual-memory storage (Sec. 4) on the GPU: the same stable sort as the
oracle (keys, permutation, runs, powers, merge tree, merge cost) with a small
recycled page pool instead of an n-element scratch buffer."""
import numpy as np
import pytest

from gpu_util import assert_matches_oracle, gpu_sort
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _vm(max_n, **kw):
    from paper_2605_27147_gb300 import binding

    return binding.Context(max_n, mode=binding.PS_MODE_VM, want_perm=True, **kw)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs", "bands"])
def test_vm_batched_copy_matches_oracle(oracle_mod, dist):
    """The batched Copy order (PS_FLAG_VM_BATCHED_COPY: each batch's targets
    moved out to free pages, then filled) gives the same sort as the default
    chain walk, element for element against the oracle."""
    from paper_2605_27147_gb300 import binding

    with _vm(1 << 20, page_log2=8, flags=binding.PS_FLAG_VM_BATCHED_COPY) as ctx:
        for n in (1, 4097, 65537, 300007, 1 << 20):
            keys = inputs.make(dist, n, 7 + n)
            ref = oracle_mod.powersort(keys)
            k, p, st = gpu_sort(ctx, keys)
            assert_matches_oracle(ctx, keys, ref, k, p, st)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs", "paper", "few", "sorted", "reversed", "equal", "bands"])
def test_vm_matches_oracle(oracle_mod, dist):
    with _vm(1 << 20, page_log2=8) as ctx:          # small pages: many pages, many waves
        for n in (1, 63, 64, 1000, 4097, 8193, 65537, 300007, 1 << 20):
            keys = inputs.make(dist, n, 3 + n)
            ref = oracle_mod.powersort(keys)
            k, p, st = gpu_sort(ctx, keys)
            assert_matches_oracle(ctx, keys, ref, k, p, st)


def test_vm_tiny_pool_recycles_pages(oracle_mod):
    # a pool barely larger than one wave: every wave must reuse freed pages
    with _vm(1 << 22, page_log2=10, tile_log2=12, pool_pages=64) as ctx:
        for dist, n in (("uniform", (1 << 22) - 12345), ("runs", 3000001), ("zipf", 1 << 22)):
            keys = inputs.make(dist, n, 7)
            ref = oracle_mod.powersort(keys)
            k, p, st = gpu_sort(ctx, keys)
            assert_matches_oracle(ctx, keys, ref, k, p, st)
            assert 0 < st["peak_pages"]


def test_vm_uses_far_less_memory_than_pingpong(oracle_mod):
    from paper_2605_27147_gb300 import binding

    n = 1 << 24
    keys = inputs.make("uniform", n, 5)
    with _vm(n) as vm, binding.Context(n, want_perm=True) as pp:
        kv, pv, sv = gpu_sort(vm, keys)
        kp, ppm, sp = gpu_sort(pp, keys)
    assert np.array_equal(kv, kp) and np.array_equal(pv, ppm)
    assert sv["merge_cost"] == sp["merge_cost"]
    # Pingpong holds n keys + n permutation entries of scratch (8n bytes); VM
    # holds a pool of about one wave of pages (a few per CTA), tens of MB here
    assert sp["scratch_bytes"] - sv["scratch_bytes"] > 6 * n
    assert sv["peak_pages"] > 0


def vm_extra_bound(n, page_size, pool_pages, tile=4096):
    """Device memory a VM context may hold for one instance of n keys with
    their permutation: the page pool (keys + permutation) + the run list
    (start and power per run slot, n/32 + 4 slots) + the page tables (about
    330 bytes per virtual page: page table, round records and splits, the
    free-page ring) + the merge tables (fewer than 4n/T HBM merges, about
    120 bytes each) + 1 MB of fixed-size tables and guards."""
    pages = -(-n // page_size)
    return (pool_pages * page_size * 8 + 5 * (n // 32 + 4) + 330 * pages + 120 * (4 * n // tile + 8)
            + (1 << 20))


def test_vm_extra_memory_bound(oracle_mod):
    """VM storage's extra memory (Sec. 4 "Pages needed") is the page pool plus
    tables of n/32 run slots, n/P pages and 4n/T HBM merges: at n = 2^24 it is
    within the stated bound and under a quarter of Pingpong's scratch."""
    from paper_2605_27147_gb300 import binding

    n = 1 << 24
    keys = inputs.make("uniform", n, 6)
    with _vm(n) as vm, binding.Context(n, want_perm=True) as pp:
        kv, pv, sv = gpu_sort(vm, keys)
        pp_bytes = pp.scratch_bytes()
        assert vm.scratch_bytes() == sv["scratch_bytes"]
    ref_k, ref_p = oracle_mod.stable_sort(keys)
    assert np.array_equal(pv, ref_p) and np.array_equal(kv, ref_k)
    assert sv["page_size"] > 0 and sv["pool_pages"] >= 16
    assert 0 < sv["peak_pages"] <= sv["pool_pages"]
    assert sv["scratch_bytes"] <= vm_extra_bound(n, sv["page_size"], sv["pool_pages"]), sv
    assert 4 * sv["scratch_bytes"] < pp_bytes, (sv["scratch_bytes"], pp_bytes)


def test_vm_keys_only(oracle_mod):
    with _vm(1 << 20, page_log2=9) as ctx:
        for n in (5000, 654321):
            keys = inputs.make("few", n, 2)
            ref = oracle_mod.powersort(keys)
            k, p, st = gpu_sort(ctx, keys, want_perm=False)
            assert np.array_equal(k, ref.keys)
            assert st["merge_cost"] == ref.stats["merge_cost"]


def test_vm_unaligned_caller_arrays(oracle_mod):
    # the caller's arrays start 4 bytes past a 16-byte boundary: the page
    # copies must not assume vector alignment
    with _vm(1 << 20, page_log2=8) as ctx:
        for n in (70001, (1 << 20) - 3):
            keys = inputs.make("uniform", n, 12)
            ref = oracle_mod.powersort(keys)
            kbuf = torch.empty(n + 1, dtype=torch.int32, device="cuda")
            pbuf = torch.empty(n + 1, dtype=torch.int32, device="cuda")
            dk, dp = kbuf[1:], pbuf[1:]
            dk.copy_(torch.from_numpy(keys.view(np.int32)))
            st = ctx.run(dk, dp, stats=True)
            assert np.array_equal(dk.cpu().numpy().view(np.uint32), ref.keys)
            assert np.array_equal(dp.cpu().numpy().view(np.uint32), ref.perm)
            assert st["merge_cost"] == ref.stats["merge_cost"]


def test_vm_page_splicing(oracle_mod):
    # ascending blocks of 8192 keys with every block below the one before it:
    # each merge outputs its right run and then its left run unchanged, every
    # slice is a whole page-aligned input page, so every output page takes
    # over an input page and no element moves in the merges: the spliced
    # pages are exactly M / P
    with _vm(1 << 20, page_log2=8) as ctx:
        L, K = 8192, 64
        blocks = [np.arange(L, dtype=np.uint32) + np.uint32((K - 1 - b) * L) for b in range(K)]
        keys = np.concatenate(blocks)
        ref = oracle_mod.powersort(keys)
        k, p, st = gpu_sort(ctx, keys)
        assert_matches_oracle(ctx, keys, ref, k, p, st)
        assert st["merge_cost"] == keys.size * 6
        assert st["pages_spliced"] == st["merge_cost"] // 256
        # blocks shifted off the page grid: fewer splices, the same result
        keys2 = np.concatenate([np.arange(100, dtype=np.uint32) + np.uint32(K * L), keys])
        ref2 = oracle_mod.powersort(keys2)
        k2, p2, st2 = gpu_sort(ctx, keys2)
        assert_matches_oracle(ctx, keys2, ref2, k2, p2, st2)
        assert st2["pages_spliced"] < st["pages_spliced"]
        # unsorted data interleaves every page: nothing to splice
        keys3 = inputs.make("uniform", 1 << 20, 4)
        k3, p3, st3 = gpu_sort(ctx, keys3)
        assert np.array_equal(k3, oracle_mod.powersort(keys3).keys)
        assert st3["pages_spliced"] == 0
