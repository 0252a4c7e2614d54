"""The measured fused multiply-add ceilings (the compute side of the step's
roofline) are positive, ordered as the hardware's pipes are, and in the range
of the device's nominal rates."""
import pytest

from paper_1106_0785_gb300 import mrtlb as M

pytestmark = pytest.mark.gpu


def test_fma_ceilings(cuda):
    fp32 = M.mrtlb_measure_peak(M.MRTLB_PEAK_FP32)
    pair = M.mrtlb_measure_peak(M.MRTLB_PEAK_FP32_PAIR)
    fp64 = M.mrtlb_measure_peak(M.MRTLB_PEAK_FP64)
    assert 10.0 < fp32 < 400.0, fp32
    assert 0.5 * fp32 < pair < 2.5 * fp32, (fp32, pair)
    assert 0.0 < fp64 < fp32, (fp64, fp32)


def test_unknown_kind_is_an_argument_error(cuda):
    with pytest.raises(M.MrtlbError):
        M.mrtlb_measure_peak(7)
