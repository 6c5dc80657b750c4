"""CPU oracle for Powersort (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library path never does.
"""
from .oracle import (  # noqa: F401
    build,
    minrun,
    power,
    stable_sort,
    stable_rank,
    powersort,
    powersort_keys64,
    powersort_records,
    stable_sort_records,
    powersort_vm,
    OracleResult,
)
