"""ps_fma_peak: the measured FMA rate that the FP64 step is held against."""
import pytest
import torch

from paper_2002_08642_gb300 import binding as B
from paper_2002_08642_gb300 import build as pbuild

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    pbuild.build()
    s = torch.cuda.current_stream().cuda_stream
    f64 = B.ps_fma_peak(B.PS_FP64, 2000, s)
    f32 = B.ps_fma_peak(B.PS_FP32, 20000, s)
    print("FMA rate: FP64 %.3f TFLOP/s, FP32 %.1f TFLOP/s" % (f64 / 1e12, f32 / 1e12))
    # below the nominal 2 x 128 lanes x 152 SMs x 2.07 GHz = 80.5 TFLOP/s FP32
    assert 1e10 < f64 < f32 < 8.2e13
    with pytest.raises(B.PsError):
        B.ps_fma_peak(7, 10, s)
