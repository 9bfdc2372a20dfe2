"""GB300 (sm_103a) statically condensed spectral-element Helmholtz solver.

The compute path is the CUDA library libsemgb.so behind the C ABI of
include/sem.h; ``paper_1601_08179_gb300.sem`` is its thin ctypes binding.
Nothing is imported eagerly: the library is loaded on first use and a missing
build raises an error instead of falling back to the CPU.
"""
