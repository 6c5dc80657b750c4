"""The C ABI without a GPU: the library builds, loads, exports every symbol its
header declares, and rejects bad arguments before touching the device."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

try:
    import torch
    HAVE_GPU = torch.cuda.is_available()
except Exception:  # pragma: no cover
    HAVE_GPU = False


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"PS_API\s+[\w\s\*]+?\b(ps_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_27147_gb300 import binding, build

    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("ps_create", "ps_run", "ps_run_batched", "ps_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2605_27147_gb300 import binding

    names = declared_symbols()
    assert set(names) == set(binding.EXPORTS)
    for name in names:
        assert hasattr(lib, name), f"{name} not exported"


def test_only_declared_symbols_are_exported(lib):
    # the build hides everything else (-fvisibility=hidden); nm lists dynamic symbols
    import subprocess

    from paper_2605_27147_gb300 import binding

    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    ps_syms = {s for s in exported if s.startswith("ps_")}
    assert ps_syms == set(declared_symbols())


def test_status_strings(lib):
    for code in range(7):
        assert lib.ps_status_str(code).startswith(b"PS_")


def test_argument_errors_need_no_gpu(lib):
    from paper_2605_27147_gb300 import binding

    h = ctypes.c_void_p()
    assert lib.ps_create(None, 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    cfg = binding.ps_config(mode=0, want_perm=1, max_n=0)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    cfg = binding.ps_config(mode=0, want_perm=1, max_n=1 << 33)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    cfg = binding.ps_config(mode=0, want_perm=1, max_n=100, max_total=50)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    cfg = binding.ps_config(mode=0, want_perm=1, max_n=100, tile_log2=20)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    cfg = binding.ps_config(mode=7, want_perm=1, max_n=100)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    assert lib.ps_run(None, None, None, 10, None) == binding.PS_EINVAL
    assert lib.ps_run_batched(None, None, None, None, 1, None) == binding.PS_EINVAL
    assert lib.ps_sync(None) == binding.PS_EINVAL
    assert lib.ps_get_runs(None, 0, None, 0, None) == binding.PS_EINVAL
    assert lib.ps_sort_records(None, None, 30, 10, None, None, None) == binding.PS_EINVAL
    assert lib.ps_sort_keys64(None, None, 10, None, 0, None) == binding.PS_EINVAL
    assert lib.ps_gather_rows(None, None, None, 0, 10, None, None, 4) == binding.PS_EINVAL
    assert lib.ps_selftest_wait_timeout(None) == binding.PS_EINVAL
    assert lib.ps_check_guards(None) == binding.PS_EINVAL
    assert lib.ps_server_cancel(None, 0) == binding.PS_EINVAL
    out = ctypes.c_uint64(0)
    assert lib.ps_get_scratch_bytes(None, ctypes.byref(out)) == binding.PS_EINVAL
    cfg = binding.ps_config(mode=0, want_perm=1, max_n=100, key_type=3)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_EINVAL
    lib.ps_destroy(None)


@pytest.mark.skipif(HAVE_GPU, reason="checks the no-GPU failure path")
def test_no_gpu_fails_loudly(lib):
    from paper_2605_27147_gb300 import binding

    h = ctypes.c_void_p()
    cfg = binding.ps_config(mode=0, want_perm=1, max_n=1000)
    assert lib.ps_create(ctypes.byref(cfg), 0, None, ctypes.byref(h)) == binding.PS_ECUDA
    assert not h.value
