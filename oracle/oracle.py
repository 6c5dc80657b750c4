"""ctypes front end of the C oracle in ``powersort_oracle.c``.

TEST INFRASTRUCTURE ONLY: used by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark; never by the library path.

The C file is compiled with gcc into ``oracle/_build/liboracle.so`` on first
use (or by :func:`build`).  Every function here only marshals numpy arrays;
all arithmetic is in the C source, which follows the paper:

* :func:`minrun`       -- Sec. 5, "Algorithm variants" (minimum run length)
* :func:`power`        -- Sec. 2 Theorem (definition of Power)
* :func:`stable_sort`  -- the plain definition of the result (stable order)
* :func:`stable_rank`  -- one output of it: the stable position of one element
* :func:`powersort`    -- Algorithm 1 with Pingpong storage (Sec. 3)
* :func:`powersort_vm` -- Algorithm 1 with virtual-memory storage (Sec. 4)
* :func:`powersort_keys64` -- Algorithm 1 on 64-bit keys ("u64", "i64" or
  "f64": unsigned, two's complement, IEEE 754 binary64 totalOrder)
* :func:`powersort_records`, :func:`stable_sort_records` -- the same for
  records of several 32-bit words ordered lexicographically (the paper's blob
  types, Sec. 5 "Input data types")

``descending_runs=True`` selects the run-detection variant named in Sec. 5
("Algorithm variants"): strictly decreasing runs are accepted too and
reversed in place.  ``key_type`` ("u32", "i32" or "f32") says how the 32-bit
keys are ordered: unsigned, two's complement, or IEEE 754 totalOrder; keys
are always passed as their 32-bit patterns (``arr.view(np.uint32)``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "powersort_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Stats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("runs", ctypes.c_uint64),
        ("merges", ctypes.c_uint64),
        ("merge_cost", ctypes.c_uint64),
        ("comparisons", ctypes.c_uint64),
        ("merge_comparisons", ctypes.c_uint64),
        ("scan_comparisons", ctypes.c_uint64),
        ("insert_comparisons", ctypes.c_uint64),
        ("moves", ctypes.c_uint64),
        ("insert_moves", ctypes.c_uint64),
        ("peak_pages", ctypes.c_uint64),
        ("pool_pages", ctypes.c_uint64),
        ("minrun", ctypes.c_uint32),
        ("max_stack", ctypes.c_uint32),
        ("max_power", ctypes.c_uint32),
        ("page_size", ctypes.c_uint32),
        ("reversed_runs", ctypes.c_uint64),
        ("reverse_moves", ctypes.c_uint64),
    ]


DESCENDING_RUNS = 1   # ORACLE_DESCENDING_RUNS
KEY_ORDER = {"u32": 0, "i32": 2, "f32": 4}   # ORACLE_KEY_I32, ORACLE_KEY_F32


def compile_source(src: str, so: str) -> str:
    """gcc a C source of the oracle into a shared object (plain C, -O2)."""
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, src],
                   check=True)
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            compile_source(_SRC, _SO)
    return _SO


def open_library(so: str):
    """ctypes handle of an oracle shared object with its signatures set."""
    lib = ctypes.CDLL(so)
    _declare(lib)
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = open_library(_SO)
    return _lib


def _declare(lib):
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.oracle_minrun.restype = ctypes.c_uint32
    lib.oracle_minrun.argtypes = [ctypes.c_uint64]
    lib.oracle_power.restype = ctypes.c_uint32
    lib.oracle_power.argtypes = [ctypes.c_uint64] * 4
    lib.oracle_stable_sort.restype = ctypes.c_int
    lib.oracle_stable_sort.argtypes = [u32p, ctypes.c_uint64, u32p, u32p]
    lib.oracle_powersort_keys64.restype = ctypes.c_int
    lib.oracle_powersort_keys64.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64, u32p, u32p, u8p, u32p,
                                            ctypes.c_uint32, ctypes.POINTER(_Stats)]
    lib.oracle_powersort_records.restype = ctypes.c_int
    lib.oracle_powersort_records.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u8p, u32p,
                                             ctypes.c_uint32, ctypes.POINTER(_Stats)]
    lib.oracle_stable_sort_records.restype = ctypes.c_int
    lib.oracle_stable_sort_records.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, u32p]
    lib.oracle_stable_sort_ex.restype = ctypes.c_int
    lib.oracle_stable_rank_ex.restype = ctypes.c_uint64
    lib.oracle_stable_rank_ex.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
    lib.oracle_stable_sort_ex.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, u32p, u32p]
    lib.oracle_powersort.restype = ctypes.c_int
    lib.oracle_powersort.argtypes = [u32p, u32p, ctypes.c_uint64, u32p, u8p, u32p,
                                     ctypes.POINTER(_Stats)]
    lib.oracle_powersort_vm.restype = ctypes.c_int
    lib.oracle_powersort_vm.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_uint64,
                                        u32p, u8p, u32p, ctypes.POINTER(_Stats)]
    lib.oracle_powersort_ex.restype = ctypes.c_int
    lib.oracle_powersort_ex.argtypes = [u32p, u32p, ctypes.c_uint64, u32p, u8p, u32p,
                                        ctypes.c_uint32, ctypes.POINTER(_Stats)]
    lib.oracle_powersort_vm_ex.restype = ctypes.c_int
    lib.oracle_powersort_vm_ex.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_uint64,
                                           u32p, u8p, u32p, ctypes.c_uint32, ctypes.POINTER(_Stats)]


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def minrun(n: int, lib=None) -> int:
    return int((lib or _load()).oracle_minrun(n))


def power(n: int, i: int, j: int, k: int, lib=None) -> int:
    """Power(n, [i,j), [j,k)) from the definition (Sec. 2 Theorem)."""
    return int((lib or _load()).oracle_power(n, i, j, k))


def stable_sort(keys: np.ndarray, key_type: str = "u32"):
    """The definition of the result: (sorted keys, stable permutation)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    n = keys.size
    ko = np.empty(n, np.uint32)
    po = np.empty(n, np.uint32)
    if n:
        rc = _load().oracle_stable_sort_ex(_ptr(keys, ctypes.c_uint32), n, KEY_ORDER[key_type],
                                           _ptr(ko, ctypes.c_uint32), _ptr(po, ctypes.c_uint32))
        if rc:
            raise MemoryError("oracle_stable_sort")
    return ko, po


def stable_rank(keys: np.ndarray, i: int, key_type: str = "u32", lib=None) -> int:
    """One output of the definition: the position of element i in the stable
    order (elements with a smaller key, plus equal keys before it)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    if not 0 <= i < keys.size:
        raise IndexError(i)
    return int((lib or _load()).oracle_stable_rank_ex(_ptr(keys, ctypes.c_uint32), keys.size, KEY_ORDER[key_type], i))


@dataclass
class OracleResult:
    keys: np.ndarray
    perm: np.ndarray
    run_starts: np.ndarray          # runs + 1 entries, last is n
    powers: np.ndarray              # runs - 1 entries (uint8)
    merges: np.ndarray              # (merges, 3) uint32: lo, mid, hi in execution order
    stats: dict = field(default_factory=dict)


def _run(fn_name: str, keys: np.ndarray, page_size: int | None, lib=None, options: int | None = None):
    lib = lib or _load()
    key = np.array(keys, dtype=np.uint32, copy=True)
    n = key.size
    perm = np.empty(n, np.uint32)
    runs = np.empty(n + 2, np.uint32)
    pw = np.zeros(max(n, 1), np.uint8)
    mg = np.empty((max(n, 1), 3), np.uint32)
    st = _Stats()
    args = [_ptr(key, ctypes.c_uint32), _ptr(perm, ctypes.c_uint32), n]
    if page_size is not None:
        args.append(page_size)
    args += [_ptr(runs, ctypes.c_uint32), _ptr(pw, ctypes.c_uint8), _ptr(mg, ctypes.c_uint32)]
    if options is not None:
        args.append(options)
    args.append(ctypes.byref(st))
    rc = getattr(lib, fn_name)(*args)
    if rc:
        raise MemoryError(fn_name)
    stats = {name: int(getattr(st, name)) for name, _ in _Stats._fields_}
    r = stats["runs"]
    return OracleResult(
        keys=key,
        perm=perm,
        run_starts=runs[: r + 1].copy() if n else np.zeros(1, np.uint32),
        powers=pw[: max(r - 1, 0)].copy(),
        merges=mg[: stats["merges"]].copy(),
        stats=stats,
    )


def _options(descending_runs: bool, key_type: str) -> int:
    return (DESCENDING_RUNS if descending_runs else 0) | KEY_ORDER[key_type]


def powersort(keys: np.ndarray, lib=None, descending_runs: bool = False, key_type: str = "u32") -> OracleResult:
    """Algorithm 1 with Pingpong storage, executed literally on one core."""
    opt = _options(descending_runs, key_type)
    if opt:
        return _run("oracle_powersort_ex", keys, None, lib, opt)
    return _run("oracle_powersort", keys, None, lib)


def powersort_vm(keys: np.ndarray, page_size: int, lib=None, descending_runs: bool = False,
                 key_type: str = "u32") -> OracleResult:
    """Algorithm 1 with virtual-memory (paged) storage, on one core."""
    opt = _options(descending_runs, key_type)
    if opt:
        return _run("oracle_powersort_vm_ex", keys, int(page_size), lib, opt)
    return _run("oracle_powersort_vm", keys, int(page_size), lib)


def powersort_records(rec: np.ndarray, lib=None, descending_runs: bool = False) -> OracleResult:
    """Algorithm 1 on records (rows of ``rec``, uint32 words, lexicographic
    order).  ``keys`` and ``perm`` of the result are both the stable order of
    the record indices."""
    lib = lib or _load()
    rec = np.ascontiguousarray(rec, dtype=np.uint32)
    n, words = rec.shape
    perm = np.empty(n, np.uint32)
    runs = np.empty(n + 2, np.uint32)
    pw = np.zeros(max(n, 1), np.uint8)
    mg = np.empty((max(n, 1), 3), np.uint32)
    st = _Stats()
    rc = lib.oracle_powersort_records(_ptr(rec, ctypes.c_uint32), words, n, _ptr(perm, ctypes.c_uint32),
                                      _ptr(runs, ctypes.c_uint32), _ptr(pw, ctypes.c_uint8),
                                      _ptr(mg, ctypes.c_uint32), DESCENDING_RUNS if descending_runs else 0,
                                      ctypes.byref(st))
    if rc:
        raise MemoryError("oracle_powersort_records")
    stats = {name: int(getattr(st, name)) for name, _ in _Stats._fields_}
    r = stats["runs"]
    return OracleResult(
        keys=perm.copy(),
        perm=perm,
        run_starts=runs[: r + 1].copy() if n else np.zeros(1, np.uint32),
        powers=pw[: max(r - 1, 0)].copy(),
        merges=mg[: stats["merges"]].copy(),
        stats=stats,
    )


def stable_sort_records(rec: np.ndarray, lib=None) -> np.ndarray:
    """The definition for records: indices ordered by (row, index)."""
    lib = lib or _load()
    rec = np.ascontiguousarray(rec, dtype=np.uint32)
    n, words = rec.shape
    perm = np.empty(n, np.uint32)
    if n and lib.oracle_stable_sort_records(_ptr(rec, ctypes.c_uint32), words, n, _ptr(perm, ctypes.c_uint32)):
        raise MemoryError("oracle_stable_sort_records")
    return perm


def powersort_keys64(keys: np.ndarray, key_type: str = "u64", lib=None, descending_runs: bool = False) -> OracleResult:
    """Algorithm 1 on 64-bit keys given as their bit patterns (uint64)."""
    lib = lib or _load()
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.size
    perm = np.empty(n, np.uint32)
    runs = np.empty(n + 2, np.uint32)
    pw = np.zeros(max(n, 1), np.uint8)
    mg = np.empty((max(n, 1), 3), np.uint32)
    st = _Stats()
    opt = {"u64": 0, "i64": 2, "f64": 4}[key_type] | (DESCENDING_RUNS if descending_runs else 0)
    rc = lib.oracle_powersort_keys64(keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n,
                                     _ptr(perm, ctypes.c_uint32), _ptr(runs, ctypes.c_uint32), _ptr(pw, ctypes.c_uint8),
                                     _ptr(mg, ctypes.c_uint32), opt, ctypes.byref(st))
    if rc:
        raise MemoryError("oracle_powersort_keys64")
    stats = {name: int(getattr(st, name)) for name, _ in _Stats._fields_}
    r = stats["runs"]
    return OracleResult(
        keys=keys[perm],
        perm=perm,
        run_starts=runs[: r + 1].copy() if n else np.zeros(1, np.uint32),
        powers=pw[: max(r - 1, 0)].copy(),
        merges=mg[: stats["merges"]].copy(),
        stats=stats,
    )
