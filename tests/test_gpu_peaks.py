"""The unit microbenchmarks behind the measured roofline (gb_measure_peaks).

Each figure must be positive and physically possible for the GPU that ran
it: no more than its SMs x 128 lanes x a 3 GHz clock.  The popcount and
shared-atomic units are narrower than the integer logic pipe, so their rates
must be below its rate.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_unit_peaks_are_plausible():
    from paper_2603_07850_gb300 import binding, build
    build.build()
    binding.load()
    p = binding.gb_measure_peaks()
    ceiling = p["sms"] * 128 * 3.0e9
    for k in ("int_logic_ops", "int_mad_ops", "popc_ops", "smem_atomic_ops"):
        assert 0 < p[k] <= ceiling, (k, p[k], ceiling)
    assert p["popc_ops"] < p["int_logic_ops"]
    assert p["smem_atomic_ops"] < p["int_logic_ops"]
    # a second measurement agrees within a factor of two (no broken timing)
    q = binding.gb_measure_peaks()
    for k in ("int_logic_ops", "smem_atomic_ops"):
        assert 0.5 < q[k] / p[k] < 2.0
