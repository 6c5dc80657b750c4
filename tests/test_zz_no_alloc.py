"""ps_run_noalloc: the allocation-free entry point for callers that cannot call
cudaMalloc (a fixed device-memory budget, or loops where an allocation's
implicit synchronisation is not acceptable).  Its output must equal that of
the ordinary entry point ps_run, element for element, on two calls in a row
(the second call reuses the scratch array the first one left behind).

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

from gpu_util import to_dev, to_host
from paper_2605_27147_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _noalloc(lib, keys_t, perm_t, n):
    stream = torch.cuda.current_stream()
    return lib.ps_run_noalloc(ctypes.c_void_p(keys_t.data_ptr()),
                              ctypes.c_void_p(perm_t.data_ptr()) if perm_t is not None else None,
                              n, torch.cuda.current_device(), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_ps_run_two_calls_in_a_row():
    from paper_2605_27147_gb300 import binding

    lib = binding.lib()
    cases = [("paper", 100003, 5), ("few", binding.PS_NOALLOC_MAX_N, 6), ("runs", 70001, 7)]
    with binding.Context(binding.PS_NOALLOC_MAX_N, want_perm=True) as ctx:
        for dist, n, seed in cases:                       # consecutive calls share the scratch
            keys = inputs.make(dist, n, seed)
            rk, rp = to_dev(keys), torch.empty(n, dtype=torch.int32, device="cuda")
            ctx.run(rk, rp)
            nk, np_ = to_dev(keys), torch.empty(n, dtype=torch.int32, device="cuda")
            assert _noalloc(lib, nk, np_, n) == binding.PS_OK
            torch.cuda.synchronize()
            assert np.array_equal(to_host(nk), to_host(rk))
            assert np.array_equal(to_host(np_), to_host(rp))
        # keys only, and the degenerate sizes
        for n in (0, 1, 2, 63, 64, 65, 1000):
            keys = inputs.make("uniform", n, n)
            nk = to_dev(keys)
            assert _noalloc(lib, nk, None, n) == binding.PS_OK
            torch.cuda.synchronize()
            assert np.array_equal(to_host(nk), np.sort(keys))


def test_noalloc_rejects_sizes_above_its_maximum():
    from paper_2605_27147_gb300 import binding

    lib = binding.lib()
    big = torch.zeros(binding.PS_NOALLOC_MAX_N + 1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, big, None, binding.PS_NOALLOC_MAX_N + 1) == binding.PS_EINVAL
