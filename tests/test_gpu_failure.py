"""Failure detection and self-checks on the GPU, none of which faults, traps
or hangs it: the bounded device wait gives up and reports PS_ETIMEOUT with
the context still usable; canary words after every device buffer the
context owns survive every kind of call; a sweep of a thousand small seeded
instances matches the oracle."""
import time

import numpy as np
import pytest

from gpu_util import gpu_sort, to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def test_bounded_wait_reports_timeout(oracle_mod):
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 16, want_perm=True) as ctx:
        t0 = time.time()
        st = ctx.selftest_wait_timeout()
        dt = time.time() - t0
        assert st == binding.PS_ETIMEOUT
        assert 0.3 < dt < 30.0, dt                 # the spin limit, about two seconds
        # the context still works: the next call starts from a clean status
        keys = inputs.make("uniform", 50000, 1)
        k, p, s = gpu_sort(ctx, keys)
        ref = oracle_mod.powersort(keys)
        assert np.array_equal(k, ref.keys) and np.array_equal(p, ref.perm)
        ctx.check_guards()


def test_guards_after_every_kind_of_call(oracle_mod):
    from paper_2605_27147_gb300 import binding

    with binding.Context(1 << 20, want_perm=True, flags=binding.PS_FLAG_RECORDS, max_total=1 << 20,
                         max_count=8) as ctx:
        gpu_sort(ctx, inputs.make("runs", (1 << 20) - 3, 2))
        ctx.check_guards()
        rec = inputs.records("few", 100003, 3, words=6)
        d = torch.from_numpy(rec.view(np.int32)).cuda()
        perm = torch.empty(rec.shape[0], dtype=torch.int32, device="cuda")
        out = torch.empty_like(d)
        ctx.sort_records(d, perm, out)
        ctx.check_guards()
        k64 = torch.from_numpy((inputs.uniform(1 << 20, 4).astype(np.int64) - (1 << 31))).cuda()
        ctx.sort_keys64(k64, torch.empty(1 << 20, dtype=torch.int32, device="cuda"), binding.PS_KEY_I32)
        ctx.check_guards()
    with binding.Context(1 << 20, mode=binding.PS_MODE_VM, page_log2=8, want_perm=True) as vm:
        gpu_sort(vm, inputs.make("uniform", (1 << 20) - 7, 5))
        vm.check_guards()


def test_small_seed_sweep(oracle_mod):
    # a thousand instances of 0 .. 4096 keys (seeds 0 .. 999, mixed shapes) in
    # one batched call, each compared with the oracle
    from paper_2605_27147_gb300 import binding

    rng = np.random.RandomState(0)
    dists = ["uniform", "few", "runs", "sorted", "reversed", "equal", "paper", "updown"]
    sizes = rng.randint(0, 4097, size=1000)
    parts = [inputs.make(dists[s % len(dists)], int(n), s) for s, n in enumerate(sizes)]
    keys = np.concatenate(parts)
    off = np.zeros(len(parts) + 1, np.uint64)
    off[1:] = np.cumsum(sizes.astype(np.uint64))
    with binding.Context(4096, want_perm=True, max_total=int(off[-1]), max_count=1000) as ctx:
        dk, dp = to_dev(keys), torch.empty(keys.size, dtype=torch.int32, device="cuda")
        ctx.run_batched(dk, torch.from_numpy(off.astype(np.int64)).cuda(), dp, stats=True)
        gk, gp = to_host(dk), to_host(dp)
        for q, part in enumerate(parts):
            a, b = int(off[q]), int(off[q + 1])
            ref = oracle_mod.powersort(part)
            assert np.array_equal(gk[a:b], ref.keys), q
            assert np.array_equal(gp[a:b], ref.perm), q
            if q % 50 == 0 and part.size:
                assert np.array_equal(ctx.runs(q), ref.run_starts), q
                assert np.array_equal(ctx.powers(q), ref.powers), q
        ctx.check_guards()
