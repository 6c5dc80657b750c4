"""Serving: continuous batching under a device-memory budget.  Every request's
result must be the same alone (ps_run) and in the mix, and requests that
arrive while others are on the GPU must be admitted and overlap with them."""
import time

import numpy as np
import pytest

from gpu_util import to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _pinned(a: np.ndarray):
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()
    return t


def test_results_same_alone_and_in_the_mix(oracle_mod):
    from paper_2605_27147_gb300 import binding

    rng = np.random.RandomState(4)
    dists = ["uniform", "zipf", "runs", "paper", "few", "sorted"]
    sizes = [int(x) for x in np.floor(2.0 ** (6 + 14 * rng.rand(90)))] + [0, 1, 63, 64, 65]
    reqs = []
    for i, n in enumerate(sizes):
        keys = inputs.make(dists[i % len(dists)], n, 1000 + i)
        reqs.append((keys, _pinned(keys), torch.empty(n, dtype=torch.int32).pin_memory(),
                     torch.empty(n, dtype=torch.int32).pin_memory()))
    with binding.Server(2 << 30, 1 << 20, lanes=3, lane_max_total=1 << 21, lane_max_count=8) as srv:
        tickets = []
        for wave in range(3):                       # later waves arrive while earlier ones run
            for k in range(wave, len(reqs), 3):
                keys, hin, hk, hp = reqs[k]
                tickets.append((k, srv.submit(hin.data_ptr(), hk.data_ptr(), hp.data_ptr(), keys.size)))
            time.sleep(0.002)
        lat = [srv.wait(t, 120.0) for _, t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["device_bytes"] <= 2 << 30, st    # what the lanes hold stays within the budget
    assert st["batches"] > 3
    assert st["max_busy_lanes"] >= 2, st            # batches were on the GPU together
    assert all(x >= 0 for x in lat)
    with binding.Context(1 << 20, want_perm=True) as solo:
        for k, (keys, hin, hk, hp) in enumerate(reqs):
            n = keys.size
            got_k = hk.numpy().view(np.uint32)[:n]
            got_p = hp.numpy().view(np.uint32)[:n]
            dk, dp = to_dev(keys), torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
            if n:
                solo.run(dk, dp[:n])
                solo.sync()
            assert np.array_equal(got_k, to_host(dk)[:n]), k
            assert np.array_equal(got_p, to_host(dp)[:n]), k
            if k % 10 == 0:
                ref = oracle_mod.powersort(keys)
                assert np.array_equal(got_k, ref.keys) and np.array_equal(got_p, ref.perm)


def test_server_rejects_oversized_requests():
    from paper_2605_27147_gb300 import binding

    with binding.Server(1 << 30, 1 << 16, lanes=1, lane_max_total=1 << 16) as srv:
        a = torch.zeros(1 << 17, dtype=torch.int32).pin_memory()
        with pytest.raises(binding.PowersortError) as e:
            srv.submit(a.data_ptr(), a.data_ptr(), None, 1 << 17)
        assert e.value.status == binding.PS_EINVAL


def test_server_budget_too_small():
    from paper_2605_27147_gb300 import binding

    with pytest.raises(binding.PowersortError) as e:
        binding.Server(1 << 20, 1 << 20, lanes=2, lane_max_total=1 << 20)
    assert e.value.status == binding.PS_ENOMEM


def test_typed_keys_and_decreasing_runs(oracle_mod):
    # every lane sorts float keys (totalOrder) with the decreasing-run variant
    from paper_2605_27147_gb300 import binding

    rng = np.random.RandomState(9)
    reqs = []
    for i, n in enumerate([0, 1, 100, 5000, 70001, 300007]):
        f = (inputs.updown(n, 40 + i, mean_run=float(rng.choice([20, 900]))).astype(np.float64) - 2.0 ** 31)
        keys = f.astype(np.float32).view(np.uint32)
        reqs.append((keys, _pinned(keys), torch.empty(max(n, 1), dtype=torch.int32).pin_memory(),
                     torch.empty(max(n, 1), dtype=torch.int32).pin_memory()))
    with binding.Server(1 << 30, 1 << 20, lanes=2, lane_max_total=1 << 20, lane_max_count=4,
                        key_type=binding.PS_KEY_F32, flags=binding.PS_FLAG_DESCENDING_RUNS) as srv:
        tickets = [srv.submit(hin.data_ptr(), hk.data_ptr(), hp.data_ptr(), keys.size) for keys, hin, hk, hp in reqs]
        for t in tickets:
            srv.wait(t, 120.0)
    for keys, hin, hk, hp in reqs:
        n = keys.size
        ref = oracle_mod.powersort(keys, key_type="f32", descending_runs=True)
        assert np.array_equal(hk.numpy().view(np.uint32)[:n], ref.keys)
        assert np.array_equal(hp.numpy().view(np.uint32)[:n], ref.perm)


def test_cancel_queued_requests(oracle_mod):
    # one lane, one request per batch: while a large request holds the lane,
    # the small ones behind it are still queued and can be cancelled
    from paper_2605_27147_gb300 import binding

    big = inputs.make("uniform", 1 << 22, 1)
    small = [inputs.make("uniform", 5000, 2 + i) for i in range(6)]
    bufs = [(k, _pinned(k), torch.empty(k.size, dtype=torch.int32).pin_memory(),
             torch.empty(k.size, dtype=torch.int32).pin_memory()) for k in [big] + small]
    with binding.Server(1 << 30, 1 << 22, lanes=1, lane_max_total=1 << 22, lane_max_count=1) as srv:
        tickets = [srv.submit(hin.data_ptr(), hk.data_ptr(), hp.data_ptr(), k.size) for k, hin, hk, hp in bufs]
        cancelled = [srv.cancel(t) for t in tickets[1:4]]
        assert any(cancelled)
        for i, t in enumerate(tickets):
            k, hin, hk, hp = bufs[i]
            if 1 <= i <= 3 and cancelled[i - 1]:
                with pytest.raises(binding.PowersortError) as e:
                    srv.wait(t, 120.0)
                assert e.value.status == binding.PS_ECANCELED
                assert not srv.cancel(t)             # only once
            else:
                srv.wait(t, 120.0)
                assert np.array_equal(hk.numpy().view(np.uint32), oracle_mod.stable_sort(k)[0])
        st = srv.stats()
        assert st["failed"] == sum(cancelled) and st["completed"] == len(tickets) - sum(cancelled)


def test_server_charges_what_the_lanes_hold():
    """The budget is checked against each lane's real allocation: its arrays,
    its offsets table and its context's scratch (ps_get_scratch_bytes)."""
    from paper_2605_27147_gb300 import binding

    lane_total, lanes, count = 1 << 20, 2, 64
    with binding.Context(1 << 20, want_perm=True, max_total=lane_total, max_count=count) as c:
        scratch = c.scratch_bytes()
    assert scratch > 8 * lane_total                 # the Pingpong scratch arrays and the tables
    need = lanes * (8 * lane_total + 8 * (count + 1) + scratch)
    with binding.Server(need, 1 << 20, lanes=lanes, lane_max_total=lane_total, lane_max_count=count) as srv:
        st = srv.stats()
    assert st["device_bytes"] == need
    # the lane arrays alone fit, the contexts' scratch does not
    with pytest.raises(binding.PowersortError) as e:
        binding.Server(need - 1, 1 << 20, lanes=lanes, lane_max_total=lane_total, lane_max_count=count)
    assert e.value.status == binding.PS_ENOMEM


def test_vm_lanes_same_results_in_less_memory(oracle_mod):
    """VM-storage lanes (the paged mode for a device-memory budget): a large
    request is sorted by itself with paged storage, small ones (up to 2^20)
    are batched in a small Pingpong context.  Every request's result equals
    the oracle's, the server charges each lane its arrays, offsets table and
    both contexts' scratch, and at n = 2^24 a VM lane's contexts hold under
    half of a Pingpong lane's."""
    from paper_2605_27147_gb300 import binding

    rng = np.random.RandomState(9)
    dists = ["uniform", "zipf", "runs", "few", "sorted", "reversed"]
    sizes = [int(x) for x in np.floor(2.0 ** (6 + 14 * rng.rand(30)))] + [0, 1, 64, 65, 1 << 20]
    reqs = []
    for i, n in enumerate(sizes):
        keys = inputs.make(dists[i % len(dists)], n, 2000 + i)
        reqs.append((keys, _pinned(keys), torch.empty(n, dtype=torch.int32).pin_memory(),
                     torch.empty(n, dtype=torch.int32).pin_memory()))
    lane_total, lanes, count = 1 << 21, 2, 16
    with binding.Context(1 << 20, mode=binding.PS_MODE_VM, want_perm=True) as c:
        vm_scratch = c.scratch_bytes()
    # the lane's context for batches of small requests (up to 2^20 each, 2^22 in
    # all, capped by the requests' and the lane's sizes)
    with binding.Context(1 << 20, want_perm=True, max_total=lane_total, max_count=count) as c:
        vm_scratch += c.scratch_bytes()
    with binding.Server(1 << 30, 1 << 20, storage=binding.PS_MODE_VM, lanes=lanes, lane_max_total=lane_total,
                        lane_max_count=count) as srv:
        tickets = [(k, srv.submit(hin.data_ptr(), hk.data_ptr(), hp.data_ptr(), keys.size))
                   for k, (keys, hin, hk, hp) in enumerate(reqs)]
        for _, t in tickets:
            srv.wait(t, 120.0)
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["device_bytes"] == lanes * (8 * lane_total + 8 * (count + 1) + vm_scratch), st
    for k, (keys, hin, hk, hp) in enumerate(reqs):
        n = keys.size
        ref = oracle_mod.powersort(keys)
        assert np.array_equal(hk.numpy().view(np.uint32)[:n], ref.keys), k
        assert np.array_equal(hp.numpy().view(np.uint32)[:n], ref.perm), k
    # the memory a lane's context holds at n = 2^24: a page pool and tables
    # against Pingpong's n-element scratch
    big = 1 << 24
    held = {}
    for mode in (binding.PS_MODE_PINGPONG, binding.PS_MODE_VM):
        with binding.Server(1 << 32, big, storage=mode, lanes=1, lane_max_total=big, lane_max_count=1) as s2:
            held[mode] = s2.stats()["device_bytes"] - 8 * big - 16
    assert held[binding.PS_MODE_VM] * 2 < held[binding.PS_MODE_PINGPONG], held
