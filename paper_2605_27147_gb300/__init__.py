"""GB300-native Powersort (Virtual-Memory Powersort, Moltmann/Nakajima/Wild).

The sort runs in hand-written sm_103a CUDA kernels behind a C ABI
(``include/powersort.h``); :mod:`paper_2605_27147_gb300.binding` is the thin
Python binding over it.  Importing this package loads nothing; the binding
loads ``libpowersort.so`` on first use and raises if it is missing.
"""
__all__ = ["binding", "inputs"]
