"""CPU oracle for the Goldbach p_min computation -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it.
"""
from .oracle import (  # noqa: F401
    OracleRecord,
    build,
    is_prime_td,
    isqrt,
    pi,
    pmin_range,
    pmin_single,
    primes_upto,
)
