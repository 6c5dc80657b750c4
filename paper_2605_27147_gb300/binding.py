"""Thin Python binding of the C ABI in ``include/powersort.h``.

Argument marshalling only: every step of the sort runs in the CUDA kernels
of ``libpowersort.so``.  Device arrays are torch CUDA tensors (torch supplies
device memory and streams); they are passed as raw pointers.  There is no CPU
fallback: if the library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PS_OK, PS_EINVAL, PS_ENOMEM, PS_ECUDA, PS_ETIMEOUT, PS_EINTERNAL, PS_ECANCELED = range(7)
PS_MODE_PINGPONG, PS_MODE_VM = 0, 1

# every symbol include/powersort.h declares
EXPORTS = (
    "ps_status_str", "ps_create", "ps_run", "ps_run_batched", "ps_run_host", "ps_sync",
    "ps_get_phase_times", "ps_get_runs", "ps_get_powers", "ps_get_nodes", "ps_get_instance_stats",
    "ps_destroy", "ps_run_noalloc", "ps_get_round_times", "ps_graph_create_batched",
    "ps_graph_launch", "ps_graph_destroy", "ps_server_create", "ps_server_submit", "ps_server_poll",
    "ps_server_wait", "ps_server_get_stats", "ps_server_destroy", "ps_gather_rows", "ps_sort_records",
    "ps_sort_keys64", "ps_selftest_wait_timeout", "ps_check_guards", "ps_server_cancel",
    "ps_get_scratch_bytes",
)
PS_NOALLOC_MAX_N = 262144
PS_FLAG_TIMING, PS_FLAG_HOST_IO, PS_FLAG_DESCENDING_RUNS, PS_FLAG_RECORDS = 1, 2, 4, 8
PS_FLAG_VM_BATCHED_COPY = 16
PS_KEY_U32, PS_KEY_I32, PS_KEY_F32 = 0, 1, 2
PHASES = ("setup", "runs", "plan", "tiles", "merge_rounds", "finish")


class ps_config(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_uint32),
        ("want_perm", ctypes.c_uint32),
        ("max_n", ctypes.c_uint64),
        ("max_total", ctypes.c_uint64),
        ("max_count", ctypes.c_uint32),
        ("page_log2", ctypes.c_uint32),
        ("tile_log2", ctypes.c_uint32),
        ("pool_pages", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("key_type", ctypes.c_uint32),
        ("merge_lanes", ctypes.c_uint32),
        ("merge_ctas", ctypes.c_uint32),
    ]


class ps_stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("runs", ctypes.c_uint64),
        ("merge_cost", ctypes.c_uint64),
        ("tiles", ctypes.c_uint64),
        ("global_nodes", ctypes.c_uint64),
        ("leaf_moves", ctypes.c_uint64),
        ("scratch_bytes", ctypes.c_uint64),
        ("peak_pages", ctypes.c_uint64),
        ("max_power", ctypes.c_uint32),
        ("rounds", ctypes.c_uint32),
        ("minrun", ctypes.c_uint32),
        ("instances", ctypes.c_uint32),
        ("hbm_merge_elems", ctypes.c_uint64),
        ("launches", ctypes.c_uint32),
        ("pages_spliced", ctypes.c_uint32),
        ("page_size", ctypes.c_uint32),
        ("pool_pages", ctypes.c_uint32),
        ("copy_pages", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class ps_server_config(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_uint64),
        ("max_n", ctypes.c_uint64),
        ("lane_max_total", ctypes.c_uint64),
        ("lane_max_count", ctypes.c_uint32),
        ("lanes", ctypes.c_uint32),
        ("want_perm", ctypes.c_uint32),
        ("device", ctypes.c_uint32),
        ("key_type", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("storage", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class ps_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("failed", ctypes.c_uint64),
        ("elements", ctypes.c_uint64),
        ("batches", ctypes.c_uint64),
        ("queued", ctypes.c_uint64),
        ("device_bytes", ctypes.c_uint64),
        ("lane_max_total", ctypes.c_uint64),
        ("lanes", ctypes.c_uint32),
        ("max_busy_lanes", ctypes.c_uint32),
    ]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class PowersortError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {lib().ps_status_str(status).decode()} ({status})")
        self.status = status


_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    return _build.SO


def lib(build_if_missing: bool = True):
    """The loaded ``libpowersort.so``.  With ``build_if_missing`` the in-tree
    build runs first (a no-op when the library matches the sources), so a
    stale library is never loaded."""
    global _lib
    with _lib_lock:
        if _lib is None:
            _lib = _load(build_if_missing)
    return _lib


def _load(build_if_missing: bool):
    path = _build.SO
    if build_if_missing:
        _build.build()
    elif not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.ps_status_str.restype = ctypes.c_char_p
    L.ps_status_str.argtypes = [ctypes.c_int]
    L.ps_create.restype = ctypes.c_int
    L.ps_create.argtypes = [ctypes.POINTER(ps_config), ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.ps_run.restype = ctypes.c_int
    L.ps_run.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(ps_stats)]
    L.ps_run_batched.restype = ctypes.c_int
    L.ps_run_batched.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.POINTER(ps_stats)]
    L.ps_run_host.restype = ctypes.c_int
    L.ps_run_host.argtypes = [vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(ps_stats)]
    L.ps_get_phase_times.restype = ctypes.c_int
    L.ps_get_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_uint32)]
    L.ps_get_round_times.restype = ctypes.c_int
    L.ps_get_round_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_uint32)]
    L.ps_sync.restype = ctypes.c_int
    L.ps_sync.argtypes = [vp]
    L.ps_selftest_wait_timeout.restype = ctypes.c_int
    L.ps_selftest_wait_timeout.argtypes = [vp]
    L.ps_check_guards.restype = ctypes.c_int
    L.ps_check_guards.argtypes = [vp]
    L.ps_server_cancel.restype = ctypes.c_int
    L.ps_server_cancel.argtypes = [vp, ctypes.c_uint64]
    L.ps_sort_keys64.restype = ctypes.c_int
    L.ps_sort_keys64.argtypes = [vp, vp, ctypes.c_uint64, vp, ctypes.c_uint32, ctypes.POINTER(ps_stats)]
    L.ps_sort_records.restype = ctypes.c_int
    L.ps_sort_records.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint64, vp, vp, ctypes.POINTER(ps_stats)]
    L.ps_gather_rows.restype = ctypes.c_int
    L.ps_gather_rows.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_uint64, vp, vp, ctypes.c_uint32]
    L.ps_graph_create_batched.restype = ctypes.c_int
    L.ps_graph_create_batched.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.POINTER(vp)]
    L.ps_graph_launch.restype = ctypes.c_int
    L.ps_graph_launch.argtypes = [vp]
    L.ps_graph_destroy.restype = None
    L.ps_graph_destroy.argtypes = [vp]
    dp = ctypes.POINTER(ctypes.c_double)
    L.ps_server_create.restype = ctypes.c_int
    L.ps_server_create.argtypes = [ctypes.POINTER(ps_server_config), ctypes.POINTER(vp)]
    L.ps_server_submit.restype = ctypes.c_int
    L.ps_server_submit.argtypes = [vp, vp, vp, vp, ctypes.c_uint64, u64p]
    L.ps_server_poll.restype = ctypes.c_int
    L.ps_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), dp]
    L.ps_server_wait.restype = ctypes.c_int
    L.ps_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, dp]
    L.ps_server_get_stats.restype = ctypes.c_int
    L.ps_server_get_stats.argtypes = [vp, ctypes.POINTER(ps_server_stats)]
    L.ps_server_destroy.restype = None
    L.ps_server_destroy.argtypes = [vp]
    L.ps_get_runs.restype = ctypes.c_int
    L.ps_get_runs.argtypes = [vp, ctypes.c_uint32, u32p, ctypes.c_uint64, u64p]
    L.ps_get_powers.restype = ctypes.c_int
    L.ps_get_powers.argtypes = [vp, ctypes.c_uint32, u8p, ctypes.c_uint64, u64p]
    L.ps_get_nodes.restype = ctypes.c_int
    L.ps_get_nodes.argtypes = [vp, ctypes.c_uint32, u32p, ctypes.c_uint64, u64p]
    L.ps_get_instance_stats.restype = ctypes.c_int
    L.ps_get_instance_stats.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(ps_stats)]
    L.ps_destroy.restype = None
    L.ps_destroy.argtypes = [vp]
    L.ps_get_scratch_bytes.restype = ctypes.c_int
    L.ps_get_scratch_bytes.argtypes = [vp, u64p]
    L.ps_run_noalloc.restype = ctypes.c_int
    L.ps_run_noalloc.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_int, vp]
    return L


def _check(st: int, what: str):
    if st != PS_OK:
        raise PowersortError(st, what)


def _ptr(t) -> int | None:
    """Raw device pointer of a torch tensor (None for None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("device arrays must be contiguous")
    return t.data_ptr()


class Context:
    """One ``ps_ctx``: its stream and every scratch buffer, allocated once."""

    def __init__(self, max_n: int, *, mode: int = PS_MODE_PINGPONG, want_perm: bool = True,
                 max_total: int = 0, max_count: int = 0, tile_log2: int = 0, page_log2: int = 0,
                 pool_pages: int = 0, flags: int = 0, key_type: int = PS_KEY_U32, device: int = 0,
                 stream=None, merge_lanes: int = 0, merge_ctas: int = 0):
        import torch

        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        cfg = ps_config(mode=mode, want_perm=1 if want_perm else 0, max_n=max_n, max_total=max_total,
                        max_count=max_count, page_log2=page_log2, tile_log2=tile_log2,
                        pool_pages=pool_pages, flags=flags, key_type=key_type, merge_lanes=merge_lanes,
                        merge_ctas=merge_ctas)
        h = ctypes.c_void_p()
        _check(lib().ps_create(ctypes.byref(cfg), device, ctypes.c_void_p(self.stream.cuda_stream),
                               ctypes.byref(h)), "ps_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ps_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- calls -------------------------------------------------------------
    def run(self, keys, perm=None, *, stats: bool = False):
        """ps_run: sort ``keys`` (uint32 as torch.int32/uint32 CUDA tensor) in place."""
        st = ps_stats() if stats else None
        _check(lib().ps_run(self._h, _ptr(keys), _ptr(perm), keys.numel(),
                            ctypes.byref(st) if st is not None else None), "ps_run")
        return st.as_dict() if st is not None else None

    def run_batched(self, keys, offsets, perm=None, *, stats: bool = False):
        """ps_run_batched: ``offsets`` is a CUDA int64/uint64 tensor of count + 1 entries."""
        st = ps_stats() if stats else None
        _check(lib().ps_run_batched(self._h, _ptr(keys), _ptr(perm), _ptr(offsets), offsets.numel() - 1,
                                    ctypes.byref(st) if st is not None else None), "ps_run_batched")
        return st.as_dict() if st is not None else None

    def sort_records(self, rec, perm, out=None, *, stats: bool = False):
        """ps_sort_records: ``rec`` is an (n, words) 32-bit tensor; ``perm``
        receives the stable lexicographic order, ``out`` (optional) the rows."""
        st = ps_stats() if stats else None
        n, words = (rec.shape[0], rec.shape[1]) if rec.dim() == 2 else (rec.shape[0], 1)
        _check(lib().ps_sort_records(self._h, _ptr(rec), words, n, _ptr(perm), _ptr(out),
                                     ctypes.byref(st) if st is not None else None), "ps_sort_records")
        return st.as_dict() if st is not None else None

    def check_guards(self):
        """ps_check_guards: raises if a canary word after a device buffer changed."""
        _check(lib().ps_check_guards(self._h), "ps_check_guards")

    def selftest_wait_timeout(self) -> int:
        """ps_selftest_wait_timeout: the status it returns (PS_ETIMEOUT expected)."""
        return int(lib().ps_selftest_wait_timeout(self._h))

    def sort_keys64(self, keys, perm, key_type: int = PS_KEY_U32, *, stats: bool = False):
        """ps_sort_keys64: ``keys`` is a 64-bit tensor sorted in place (as
        unsigned, int64 or float64 per ``key_type``: PS_KEY_U32/I32/F32)."""
        st = ps_stats() if stats else None
        _check(lib().ps_sort_keys64(self._h, _ptr(keys), keys.numel(), _ptr(perm), key_type,
                                    ctypes.byref(st) if st is not None else None), "ps_sort_keys64")
        return st.as_dict() if st is not None else None

    def gather_rows(self, perm, src, dst, *, offsets=None):
        """ps_gather_rows: dst row r = src row perm[r] (rows of src's trailing
        dimensions, any width; per instance when ``offsets`` is given)."""
        rows = src.shape[0] if src.dim() else 0
        row_bytes = (src.numel() // max(rows, 1)) * src.element_size()
        count = offsets.numel() - 1 if offsets is not None else 0
        _check(lib().ps_gather_rows(self._h, _ptr(perm), _ptr(offsets), count, rows, _ptr(src), _ptr(dst),
                                    row_bytes), "ps_gather_rows")

    def graph_batched(self, keys, offsets, perm=None) -> "Graph":
        """Capture ps_run_batched on these arrays into a replayable CUDA graph."""
        h = ctypes.c_void_p()
        _check(lib().ps_graph_create_batched(self._h, _ptr(keys), _ptr(perm), _ptr(offsets), offsets.numel() - 1,
                                             ctypes.byref(h)), "ps_graph_create_batched")
        return Graph(h, self)

    def run_host(self, keys_ptr: int, n: int, perm_ptr: int | None = None, *, stats: bool = False):
        """ps_run_host on raw host pointers (e.g. pinned torch tensors' data_ptr())."""
        st = ps_stats() if stats else None
        _check(lib().ps_run_host(self._h, keys_ptr, perm_ptr, n, ctypes.byref(st) if st is not None else None),
               "ps_run_host")
        return st.as_dict() if st is not None else None

    def phase_times(self) -> dict:
        """Milliseconds per phase of the last call (needs PS_FLAG_TIMING)."""
        buf = (ctypes.c_float * len(PHASES))()
        _check(lib().ps_get_phase_times(self._h, buf, len(PHASES), None), "ps_get_phase_times")
        return {name: float(buf[i]) for i, name in enumerate(PHASES)}

    def round_times(self) -> list:
        """Four times (us since the merge kernel's start) per HBM merge round of
        the last call, as ps_get_round_times describes for each storage."""
        cnt = ctypes.c_uint32()
        _check(lib().ps_get_round_times(self._h, None, 0, ctypes.byref(cnt)), "ps_get_round_times")
        buf = (ctypes.c_float * max(1, cnt.value))()
        _check(lib().ps_get_round_times(self._h, buf, cnt.value, None), "ps_get_round_times")
        v = [float(buf[i]) for i in range(cnt.value)]
        return [tuple(v[i:i + 4]) for i in range(0, len(v), 4)]

    def sync(self):
        _check(lib().ps_sync(self._h), "ps_sync")

    def runs(self, q: int = 0) -> np.ndarray:
        cnt = ctypes.c_uint64()
        _check(lib().ps_get_runs(self._h, q, None, 0, ctypes.byref(cnt)), "ps_get_runs")
        out = np.empty(cnt.value, np.uint32)
        _check(lib().ps_get_runs(self._h, q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), out.size,
                                 None), "ps_get_runs")
        return out

    def powers(self, q: int = 0) -> np.ndarray:
        cnt = ctypes.c_uint64()
        _check(lib().ps_get_powers(self._h, q, None, 0, ctypes.byref(cnt)), "ps_get_powers")
        out = np.empty(cnt.value, np.uint8)
        if out.size:
            _check(lib().ps_get_powers(self._h, q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                       out.size, None), "ps_get_powers")
        return out

    def nodes(self, q: int = 0) -> np.ndarray:
        cnt = ctypes.c_uint64()
        _check(lib().ps_get_nodes(self._h, q, None, 0, ctypes.byref(cnt)), "ps_get_nodes")
        out = np.empty(cnt.value, np.uint32)
        if out.size:
            _check(lib().ps_get_nodes(self._h, q, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                      out.size, None), "ps_get_nodes")
        return out.reshape(-1, 2)

    def scratch_bytes(self) -> int:
        out = ctypes.c_uint64(0)
        _check(lib().ps_get_scratch_bytes(self._h, ctypes.byref(out)), "ps_get_scratch_bytes")
        return int(out.value)

    def instance_stats(self, q: int = 0) -> dict:
        st = ps_stats()
        _check(lib().ps_get_instance_stats(self._h, q, ctypes.byref(st)), "ps_get_instance_stats")
        return st.as_dict()


class Graph:
    """A captured batched sort (ps_graph); launch() replays it on the context's stream."""

    def __init__(self, handle, ctx):
        self._h = handle
        self.ctx = ctx

    def launch(self):
        _check(lib().ps_graph_launch(self._h), "ps_graph_launch")

    def close(self):
        if self._h is not None and self._h.value:
            lib().ps_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """ps_server: continuous batching of host-array sorts under a device-memory budget."""

    def __init__(self, budget_bytes: int, max_n: int, *, lanes: int = 0, lane_max_total: int = 0,
                 lane_max_count: int = 0, want_perm: bool = True, device: int = 0, key_type: int = PS_KEY_U32,
                 flags: int = 0, storage: int = PS_MODE_PINGPONG):
        cfg = ps_server_config(budget_bytes=budget_bytes, max_n=max_n, lane_max_total=lane_max_total,
                               lane_max_count=lane_max_count, lanes=lanes, want_perm=1 if want_perm else 0,
                               device=device, key_type=key_type, flags=flags, storage=storage)
        h = ctypes.c_void_p()
        _check(lib().ps_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ps_server_create")
        self._h = h

    def submit(self, in_ptr: int, keys_out_ptr: int, perm_out_ptr: int | None, n: int) -> int:
        """Queue a sort of host arrays given by raw pointers; returns the ticket."""
        t = ctypes.c_uint64()
        _check(lib().ps_server_submit(self._h, in_ptr, keys_out_ptr, perm_out_ptr, n, ctypes.byref(t)),
               "ps_server_submit")
        return t.value

    def cancel(self, ticket: int) -> bool:
        """ps_server_cancel: True if the request was still queued and is now cancelled."""
        st = lib().ps_server_cancel(self._h, ticket)
        if st not in (PS_OK, PS_EINVAL):
            _check(st, "ps_server_cancel")
        return st == PS_OK

    def poll(self, ticket: int):
        done, lat = ctypes.c_int(), ctypes.c_double()
        _check(lib().ps_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(lat)), "ps_server_poll")
        return bool(done.value), lat.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> float:
        lat = ctypes.c_double()
        _check(lib().ps_server_wait(self._h, ticket, timeout_s, ctypes.byref(lat)), "ps_server_wait")
        return lat.value

    def stats(self) -> dict:
        st = ps_server_stats()
        _check(lib().ps_server_get_stats(self._h, ctypes.byref(st)), "ps_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ps_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def as_u32(t):
    """View an int32 torch tensor holding uint32 bit patterns (torch has limited uint32 support)."""
    import torch

    return t.view(torch.int32) if t.dtype != torch.int32 else t
