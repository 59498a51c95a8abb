"""GB300-native exhaustive Goldbach range verification (segmented double sieve).

The compute path lives in the CUDA shared library ``libgoldbach_gb300.so``
built from ``csrc/``; ``binding`` is a thin ctypes layer over its C ABI.
"""
