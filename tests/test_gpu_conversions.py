"""The integer-only number conversions that replace FP64 conversion
instructions in the kernels (GB300 runs FP64 arithmetic and conversions at
1/64 of the FP32 rate): double -> float with round-to-nearest-even and
float -> double compared bit for bit with the CUDA conversions, and the
double -> double-float split within its 2^-47 bound, over 2^24 seeded inputs
(every exponent, ties, zeros, subnormals, infinities, NaN)."""
import pytest

from paper_1706_06844_gb300 import fde

pytestmark = pytest.mark.gpu


def test_integer_conversions_match_cuda():
    import torch
    assert torch.cuda.is_available()
    assert fde.fde_conversion_selftest(1 << 24) == 0


def test_conversion_selftest_rejects_bad_arguments():
    with pytest.raises(fde.FDEError):
        fde.fde_conversion_selftest(0)
