"""The deposits' fixed-point conversions (32-bit instructions only) against CUDA's direct
64-bit conversions, bit for bit, on the device (weights in [0, 1] with both ends, counts
of every magnitude, exact rounding ties)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fixed_point_conversions_are_bit_identical(seed):
    import paper_2003_04925_gb300 as sc
    assert sc.scola_selftest_conversions(1 << 24, seed) == 0
